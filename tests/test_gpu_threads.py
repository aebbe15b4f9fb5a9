"""Two host threads, each with its own context on device 0 and its own CUDA
stream, run BF16 DeepClean forwards (the whole-network tensor-core kernel)
and BBHnet scores (the per-layer tensor-core kernel) at the same time; every
result equals, bit for bit, the one computed alone.  This covers the launch
state that is per device (kernel attributes, the multiprocessor count) or
per thread (the failure-path test hook) rather than per process."""
import threading

import numpy as np
import pytest
import torch

from paper_2108_12430_gb300 import gwstream as G, synth

pytestmark = pytest.mark.gpu

B, L, STRIDE = 4, 4096, 512


def make_inputs():
    x = synth.witness_channels(5, 21, L + (B - 1) * STRIDE).astype(np.float32)
    xb = np.random.default_rng(6).standard_normal((B, 2, 2048)).astype(np.float32)
    return x, xb


def run_once(ctx, x_d, xb_d, stream):
    dc = G.gw_model_create(ctx, G.GW_MODEL_DEEPCLEAN, G.GW_BF16, 21, synth.flatten_params(synth.deepclean_params(3)))
    layers, head = synth.bbhnet_params(4)
    bb = G.gw_model_create(ctx, G.GW_MODEL_BBHNET, G.GW_BF16, 2, synth.flatten_params(layers, head))
    return dc, bb


def forward(dc, bb, x_d, xb_d, y, logits, stream):
    h = stream.cuda_stream
    G.gw_deepclean_forward(dc, x_d.data_ptr(), x_d.shape[1], STRIDE, B, L, y.data_ptr(), h)
    G.gw_bbhnet_score(bb, xb_d.data_ptr(), B, 2048, logits.data_ptr(), h)
    stream.synchronize()


def test_two_contexts_on_two_threads_bf16(gpu_lib):
    x, xb = make_inputs()
    x_d, xb_d = torch.from_numpy(x).cuda(), torch.from_numpy(xb).cuda()
    ctx0 = G.gw_ctx_create(0, 0)
    try:
        s0 = torch.cuda.Stream()
        dc, bb = run_once(ctx0, x_d, xb_d, s0)
        y_ref, l_ref = torch.zeros(B, L, device="cuda"), torch.zeros(B, device="cuda")
        forward(dc, bb, x_d, xb_d, y_ref, l_ref, s0)
        y_ref, l_ref = y_ref.cpu(), l_ref.cpu()
        assert torch.isfinite(y_ref).all() and torch.isfinite(l_ref).all()
        G.gw_model_destroy(dc)
        G.gw_model_destroy(bb)
    finally:
        G.gw_ctx_destroy(ctx0)

    errors = []
    start = threading.Barrier(2)

    def worker(tid):
        try:
            ctx = G.gw_ctx_create(0, 0)
            try:
                st = torch.cuda.Stream()
                dc, bb = run_once(ctx, x_d, xb_d, st)
                y, lg = torch.zeros(B, L, device="cuda"), torch.zeros(B, device="cuda")
                start.wait(timeout=60)
                for it in range(25):
                    forward(dc, bb, x_d, xb_d, y, lg, st)
                    if not (torch.equal(y.cpu(), y_ref) and torch.equal(lg.cpu(), l_ref)):
                        errors.append(f"thread {tid} iteration {it}: result differs from the one computed alone")
                        break
                assert G.gw_model_status(dc, st.cuda_stream) in (G.GW_OK, None)
                G.gw_model_destroy(dc)
                G.gw_model_destroy(bb)
            finally:
                G.gw_ctx_destroy(ctx)
        except Exception as e:  # reported to the main thread
            errors.append(f"thread {tid}: {type(e).__name__}: {e}")

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not any(t.is_alive() for t in threads), "a worker thread did not finish"
    assert not errors, errors
