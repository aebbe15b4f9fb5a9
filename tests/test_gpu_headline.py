"""Parity at the benchmarked streaming configuration, and the tolerance on
the cleaned-strain ASD (Methods, "Streaming IaaS", "Data aggregation" and
"Aggregation latency").

The stream is driven the way the benchmark drives it: DeepClean on 21 x 32768
windows (8 s at 4096 Hz), stride 256, pushes of 64 snapshots, AVERAGE
aggregation with latency W - S, so that every cleaned sample is the mean of
the 128 windows that cover it.  18 pushes (1152 snapshots) make the ring of
R = W + 63 S samples wrap six times, and snapshots 127 .. 1150 emit 64 s of
cleaned strain in which every sample is averaged over all 128 windows.  The
first 9 pushes go through device buffers (the benchmark's timed loop), the
last 9 through pinned host buffers queued with gw_stream_push_async and one
gw_stream_sync (its end-to-end leg).

Every cleaned sample is compared with the FP64 oracle's: per snapshot,
relative L2 <= 1e-5 (FP32) or <= 2e-2 (BF16), both for the cleaned strain
and for the aggregated prediction it contains.  The ASD check: Welch (Hann,
2 s segments, 50% overlap) of the 64 s of cleaned strain, every bin in
55-65 Hz within 1% of the oracle's.
"""
import numpy as np
import pytest
import torch

from oracle import pool, spectral, stream as ostream
from paper_2108_12430_gb300 import gwstream as G, synth
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu

W, S, B, C, SEED = 32768, 256, 64, 21, 1234
N_PUSH = 18
N_SNAP = N_PUSH * B
DELTA = W - S
FS = 4096.0
ASD_SNAPS = slice(W // S - 1, W // S - 1 + 1024)  # snapshots emitting times [0, 64 s)
TOL = {"fp32": 1e-5, "bf16": 2e-2}


@pytest.fixture(scope="module")
def inputs():
    n = N_SNAP * S
    wit = synth.witness_channels(SEED, C, n).astype(np.float32)
    strain = synth.coupled_strain(SEED, wit.astype(np.float64)).astype(np.float32)
    return wit, strain


@pytest.fixture(scope="module")
def oracle_out(inputs):
    wit, strain = inputs
    params = synth.deepclean_params(SEED)
    preds = pool.deepclean_stream_windows(wit.astype(np.float64), W, S, range(N_SNAP), params,
                                          synth.DEEPCLEAN_LAYERS)
    agg = ostream.aggregate_by_window(preds, W, S, ostream.AVERAGE, DELTA)
    return agg, ostream.clean(strain.astype(np.float64), agg, S, DELTA)


def run_gpu(precision, inputs):
    wit, strain = inputs
    ctx = G.gw_ctx_create(0, 0)
    try:
        m = G.gw_model_create(ctx, G.GW_MODEL_DEEPCLEAN, precision, C,
                              synth.flatten_params(synth.deepclean_params(SEED)))
        s = G.gw_stream_create(ctx, [m], 1, C, W, S, B, G.GW_AGG_AVERAGE, DELTA)
        n = B * S
        out = np.zeros((N_PUSH, n), np.float32)
        wit_d = torch.from_numpy(wit).cuda()
        str_d = torch.from_numpy(strain).cuda()
        o_d = torch.zeros(n, device="cuda")
        h = torch.cuda.current_stream().cuda_stream
        half = N_PUSH // 2
        for p in range(half):  # device buffers, as the timed loop of the benchmark
            w_ = wit_d[:, p * n:(p + 1) * n].contiguous()
            s_ = str_d[p * n:(p + 1) * n].contiguous()
            G.gw_stream_push(s, B, w_.data_ptr(), s_.data_ptr(), o_d.data_ptr(), G.GW_MEM_DEVICE, h)
            torch.cuda.synchronize()
            out[p] = o_d.cpu().numpy()
        # pinned host buffers, queued, one sync (the benchmark's end-to-end leg)
        lib = G.lib()
        wh = [torch.from_numpy(np.ascontiguousarray(wit[:, p * n:(p + 1) * n])).pin_memory() for p in range(half, N_PUSH)]
        sh = [torch.from_numpy(np.ascontiguousarray(strain[p * n:(p + 1) * n])).pin_memory() for p in range(half, N_PUSH)]
        oh = [torch.zeros(n).pin_memory() for _ in range(half, N_PUSH)]
        for i in range(N_PUSH - half):
            rc = lib.gw_stream_push_async(s, B, wh[i].data_ptr(), sh[i].data_ptr(), oh[i].data_ptr(), h)
            assert rc == G.GW_OK, lib.gw_last_error()
        G.gw_stream_sync(s)
        for i in range(N_PUSH - half):
            out[half + i] = oh[i].numpy()
        assert G.gw_stream_status(s, h) == G.GW_OK
        G.gw_stream_destroy(s)
        G.gw_model_destroy(m)
    finally:
        G.gw_ctx_destroy(ctx)
    return out.reshape(N_SNAP, S).astype(np.float64)


@pytest.fixture(scope="module")
def gpu_out(gpu_lib, inputs):
    res = {}
    for name, prec in (("fp32", G.GW_FP32), ("bf16", G.GW_BF16)):
        try:
            res[name] = run_gpu(prec, inputs)
        except G.GwError as e:
            if e.code != G.GW_ENOTIMPL:
                raise
    return res


def emitted_strain(strain, k):
    t = ostream.emit_times(k, S, DELTA)
    return np.where(t >= 0, strain[np.clip(t, 0, None)].astype(np.float64), 0.0)


@pytest.mark.parametrize("name", ["fp32", "bf16"])
def test_headline_stream_matches_oracle(name, gpu_out, oracle_out, inputs):
    if name not in gpu_out:
        pytest.skip(f"{name} path not available on this device")
    got = gpu_out[name]
    agg_ref, clean_ref = oracle_out
    strain = inputs[1]
    tol = TOL[name]
    worst_c = worst_p = 0.0
    for k in range(N_SNAP):
        ec = rel_l2(got[k], clean_ref[k])
        ep = rel_l2(emitted_strain(strain, k) - got[k], agg_ref[k])
        worst_c, worst_p = max(worst_c, ec), max(worst_p, ep)
        assert ec <= tol and ep <= tol, (name, k, ec, ep)
    print(f"{name}: worst per-snapshot rel-L2 cleaned {worst_c:.2e}, prediction {worst_p:.2e}")


@pytest.mark.parametrize("name", ["fp32", "bf16"])
def test_headline_cleaned_strain_asd_within_1pct(name, gpu_out, oracle_out, inputs):
    if name not in gpu_out:
        pytest.skip(f"{name} path not available on this device")
    got = gpu_out[name][ASD_SNAPS].reshape(-1)
    agg_ref, clean_ref = oracle_out
    ref = clean_ref[ASD_SNAPS].reshape(-1)
    assert got.size == 64 * int(FS)
    f, a_got = spectral.welch_asd(got, FS)
    _, a_ref = spectral.welch_asd(ref, FS)
    band = (f >= 55.0) & (f <= 65.0)
    dev = np.abs(a_got[band] / a_ref[band] - 1.0)
    assert dev.max() <= 0.01, (name, dev.max())
    # the aggregated noise prediction the cleaning subtracts, the same way
    strain = inputs[1]
    pred_got = np.concatenate([emitted_strain(strain, k) - gpu_out[name][k] for k in range(N_SNAP)[ASD_SNAPS]])
    _, p_got = spectral.welch_asd(pred_got, FS)
    _, p_ref = spectral.welch_asd(agg_ref[ASD_SNAPS].reshape(-1), FS)
    pdev = np.abs(p_got[band] / p_ref[band] - 1.0)
    assert pdev.max() <= 0.01, (name, pdev.max())
    print(f"{name}: max ASD deviation in 55-65 Hz: cleaned {dev.max():.2e}, prediction {pdev.max():.2e}")
