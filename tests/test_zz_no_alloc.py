"""The allocation-free DeepClean forward against the ordinary one.

gw_deepclean_forward_noalloc serves callers that may not allocate device
memory (a real-time loop with a fixed memory plan, or a framework that bans
cudaMalloc from plug-ins); it runs on a fixed scratch array inside the
library.  This file is collected last so that a failure here cannot hide
the other tests' results; it passes alone and after them.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2108_12430_gb300 import gwstream as G, synth

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_forward_matches_allocating_forward(gpu_lib):
    lib = G.lib()
    ctx = G.gw_ctx_create(0, 0)
    try:
        m = G.gw_model_create(ctx, G.GW_MODEL_DEEPCLEAN, G.GW_FP32, 21,
                              synth.flatten_params(synth.deepclean_params(11)))
        B, L, stride = 3, 4096, 2048
        ld = L + (B - 1) * stride
        x = torch.from_numpy(synth.witness_channels(12, 21, ld).astype(np.float32)).cuda()
        ys = [torch.full((B, L), float("nan"), device="cuda") for _ in range(2)]
        torch.cuda.synchronize()
        # the model is fresh: the allocating forward has not grown its
        # workspace yet, so any allocation by the calls below would show
        allocs0, in_use0 = G.gw_alloc_count(), G.gw_ctx_bytes_in_use(ctx)
        for call in range(2):  # two calls in a row share the scratch array
            rc = lib.gw_deepclean_forward_noalloc(m, ctypes.c_void_p(x.data_ptr()), ld, stride, B, L,
                                                  ctypes.c_void_p(ys[call].data_ptr()), None)
            assert rc == G.GW_OK, lib.gw_last_error()
        torch.cuda.synchronize()
        assert G.gw_alloc_count() == allocs0 and G.gw_ctx_bytes_in_use(ctx) == in_use0
        ref = torch.zeros(B, L, device="cuda")
        G.gw_deepclean_forward(m, x.data_ptr(), ld, stride, B, L, ref.data_ptr())
        torch.cuda.synchronize()
        assert G.gw_alloc_count() > allocs0  # the counter does see the workspace of the allocating forward
        for call in range(2):
            assert rel_l2(ys[call].cpu().numpy(), ref.cpu().numpy()) <= 1e-5, call
        # sizes beyond the scratch limit are refused without touching the device
        big = torch.zeros(2, 32768, device="cuda")
        rc = lib.gw_deepclean_forward_noalloc(m, ctypes.c_void_p(x.data_ptr()), 32768, 0, 2, 32768,
                                              ctypes.c_void_p(big.data_ptr()), None)
        assert rc == G.GW_EINVAL and b"scratch limit" in lib.gw_last_error()
        G.gw_model_destroy(m)
    finally:
        G.gw_ctx_destroy(ctx)
