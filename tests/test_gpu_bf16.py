"""BF16 tensor-core path parity against the FP64 oracle.

Tolerances (stated for the BF16 path): relative L2 <= 2e-2 per output
tensor, BBHnet logits within 0.05 absolute.  The first test is the smallest
case (one 1 s window) so that a problem shows on a tiny launch.
"""
import numpy as np
import pytest
import torch

from oracle import nets
from paper_2108_12430_gb300 import gwstream as G, synth
from tests.gpu_util import Ctx, dev, rel_l2
from tests.test_gpu_f32 import oracle_dc, run_stream_case

pytestmark = pytest.mark.gpu
TOL16 = 2e-2


@pytest.fixture
def ctx(gpu_lib):
    c = Ctx()
    yield c
    c.close()


def test_deepclean_config1_bf16(ctx):
    x = synth.witness_channels(0, 21, 4096)[None]
    m = ctx.deepclean(0, G.GW_BF16)
    y = torch.zeros(1, 4096, device="cuda")
    G.gw_deepclean_forward(m, dev(x[0]).data_ptr(), 4096, 0, 1, 4096, y.data_ptr())
    torch.cuda.synchronize()
    G.gw_model_status(m)
    err = rel_l2(y.cpu().numpy(), oracle_dc(x, 0))
    print("config-1 BF16 rel-L2", err)
    assert err <= TOL16


def test_bf16_deepclean_is_one_whole_network_launch(ctx):
    """A BF16 DeepClean model runs the whole-network kernel, one launch per
    forward.  The per-layer kernels give results within the same tolerance,
    so only the launch list shows a model that fell back to them."""
    x = synth.witness_channels(1, 21, 4096)
    m = ctx.deepclean(0, G.GW_BF16)
    xd = dev(x)
    y = torch.zeros(1, 4096, device="cuda")
    G.gw_deepclean_forward(m, xd.data_ptr(), 4096, 0, 1, 4096, y.data_ptr())  # the workspace is made here
    torch.cuda.synchronize()
    G.gw_profile_enable(True)
    try:
        G.gw_deepclean_forward(m, xd.data_ptr(), 4096, 0, 1, 4096, y.data_ptr())
        prof = G.gw_profile_read()
    finally:
        G.gw_profile_enable(False)
    assert prof.get("deepclean_fused", (0.0, 0))[1] == 1, prof
    assert not any(k.startswith("conv_tc") for k in prof), prof


@pytest.mark.parametrize("B,L,stride", [(3, 1000, 1000), (5, 2056, 264), (2, 8, 8), (1, 4104, 0)])
def test_deepclean_ragged_and_views_bf16(ctx, B, L, stride):
    ld = L + (B - 1) * stride
    xs = synth.witness_channels(3, 21, ld) * 2.0 + 0.5
    mean, std = np.full(21, 0.5), np.full(21, 2.0)
    m = ctx.deepclean(1, G.GW_BF16, mean=mean, std=std)
    y = torch.zeros(B, L, device="cuda")
    G.gw_deepclean_forward(m, dev(xs).data_ptr(), ld, stride, B, L, y.data_ptr())
    torch.cuda.synchronize()
    G.gw_model_status(m)
    wins = np.stack([xs[:, b * stride:b * stride + L] for b in range(B)])
    ref = oracle_dc(wins, 1, mean, std)
    for b in range(B):
        assert rel_l2(y[b].cpu().numpy(), ref[b]) <= TOL16, b


def test_deepclean_full_window_batch_sampled_bf16(ctx):
    W, S, B = 32768, 256, 64
    ld = W + (B - 1) * S
    xs = synth.witness_channels(4, 21, ld)
    m = ctx.deepclean(2, G.GW_BF16)
    y = torch.zeros(B, W, device="cuda")
    G.gw_deepclean_forward(m, dev(xs).data_ptr(), ld, S, B, W, y.data_ptr())
    torch.cuda.synchronize()
    G.gw_model_status(m)
    for b in (0, 41, 63):
        ref = oracle_dc(xs[None, :, b * S:b * S + W], 2)[0]
        assert rel_l2(y[b].cpu().numpy(), ref) <= TOL16, b


def test_bf16_matches_fp32_path_closely(ctx):
    # same inputs through both GPU paths: BF16 error stays at bf16 level
    x = synth.witness_channels(8, 21, 8192)
    m32, m16 = ctx.deepclean(5), ctx.deepclean(5, G.GW_BF16)
    y32 = torch.zeros(1, 8192, device="cuda")
    y16 = torch.zeros(1, 8192, device="cuda")
    xd = dev(x)
    G.gw_deepclean_forward(m32, xd.data_ptr(), 8192, 0, 1, 8192, y32.data_ptr())
    G.gw_deepclean_forward(m16, xd.data_ptr(), 8192, 0, 1, 8192, y16.data_ptr())
    torch.cuda.synchronize()
    assert rel_l2(y16.cpu().numpy(), y32.cpu().numpy()) <= TOL16


@pytest.mark.parametrize("mode,delta", [(G.GW_AGG_LATEST, 0), (G.GW_AGG_AVERAGE, 1024 - 128),
                                        (G.GW_AGG_AVERAGE, 200)])
def test_stream_matches_oracle_bf16(ctx, mode, delta):
    W, S = 1024, 128
    for g, ref in run_stream_case(ctx, W, S, [3, 1, 5, 4, 2, 5], mode, delta, precision=G.GW_BF16):
        assert g.shape == ref.shape
        assert rel_l2(g, ref) <= TOL16


def test_stream_post_processing_bf16(ctx):
    W, S = 1024, 128
    for g, ref in run_stream_case(ctx, W, S, [2, 5, 1, 4], G.GW_AGG_AVERAGE, W - S, seed=9, precision=G.GW_BF16,
                                  post_taps=257):
        assert g.shape == ref.shape
        assert rel_l2(g, ref) <= TOL16


def test_bulk_stride_half_window_bf16(ctx):
    # offline bulk mode: snapshots at 1/4 Hz with 8 s windows, i.e. S = W / 2,
    # every sample averaged over the two windows that cover it
    W, S = 2048, 1024
    for g, ref in run_stream_case(ctx, W, S, [4, 2, 5], G.GW_AGG_AVERAGE, W - S, seed=6, precision=G.GW_BF16):
        assert g.shape == ref.shape
        assert rel_l2(g, ref) <= TOL16


def test_stream_two_detectors_bf16(ctx):
    W, S = 512, 64
    for g, ref in run_stream_case(ctx, W, S, [2, 6, 1, 8], G.GW_AGG_AVERAGE, W - S, seed=3, n_det=2,
                                  precision=G.GW_BF16):
        assert rel_l2(g, ref) <= TOL16


def test_stream_standardised_input_bf16(ctx):
    W, S = 1024, 128
    for g, ref in run_stream_case(ctx, W, S, [2, 3, 1, 4], G.GW_AGG_AVERAGE, W - S, seed=4, n_det=2,
                                  precision=G.GW_BF16, standardise=True):
        assert rel_l2(g, ref) <= TOL16


@pytest.mark.parametrize("B,L", [(3, 2048), (2, 512), (1, 16)])
def test_bbhnet_bf16(ctx, B, L):
    x = np.random.default_rng(B * 1000 + L).standard_normal((B, 2, L))
    m = ctx.bbhnet(0, G.GW_BF16)
    out = torch.zeros(B, device="cuda")
    G.gw_bbhnet_score(m, dev(x).data_ptr(), B, L, out.data_ptr())
    torch.cuda.synchronize()
    G.gw_model_status(m)
    params, head = synth.bbhnet_params(0)
    ref = nets.bbhnet_forward(x, params, head, synth.bbhnet_layers())
    np.testing.assert_allclose(out.cpu().numpy(), ref, atol=0.05)
    assert rel_l2(out.cpu().numpy(), ref) <= TOL16 or np.abs(out.cpu().numpy() - ref).max() <= 0.05


def test_bbhnet_batch256_sampled_bf16(ctx):
    x, label, snr = synth.injected_strain(9, 256, 2048)
    m = ctx.bbhnet(1, G.GW_BF16)
    out = torch.zeros(256, device="cuda")
    G.gw_bbhnet_score(m, dev(x).data_ptr(), 256, 2048, out.data_ptr())
    torch.cuda.synchronize()
    G.gw_model_status(m)
    params, head = synth.bbhnet_params(1)
    idx = [0, 1, 100, 255]
    ref = nets.bbhnet_forward(x[idx], params, head, synth.bbhnet_layers())
    np.testing.assert_allclose(out.cpu().numpy()[idx], ref, atol=0.05)


@pytest.mark.parametrize("B,C,L_in", [(256, 2, 4096), (3, 1, 2056), (2, 2, 6144)])
def test_whiten_bf16(ctx, B, C, L_in):
    # the FIR runs as an 8 -> 8 channel tensor-core conv on the space-to-depth
    # view of the signal; compared with the oracle's valid-mode FIR
    from oracle import fir as ofir
    fs, nfft = 2048.0, 8192
    f, psd = synth.psd_grid(fs, nfft)
    fh = G.gw_fir_create_whitening(ctx.h, psd, fs, 2049, G.GW_BF16)
    ctx.objs.append((G.gw_fir_destroy, fh))
    x = synth.colored_noise(B + L_in, L_in, fs, n_ch=B * C).reshape(B, C, L_in)
    lout = L_in - 2048
    y = torch.zeros(B, C, lout, device="cuda")
    G.gw_whiten(fh, dev(x).data_ptr(), B, C, L_in, y.data_ptr())
    torch.cuda.synchronize()
    h = ofir.whitening_fir(psd, fs, nfft, 2049)
    xr = x.reshape(B * C, L_in)
    yr = y.reshape(B * C, lout).cpu().numpy()
    for r in sorted({0, B * C // 2, B * C - 1}):
        assert rel_l2(yr[r], ofir.fir_valid(xr[r], h)) <= TOL16, r


def test_bounded_wait_runs_out_and_context_survives(ctx):
    # failure detection without a GPU fault: one CTA of the first layer never
    # arms an input stage, its MMA thread's bounded wait (about 1 s) runs out,
    # the launch unwinds, the host reads GW_ETIMEOUT; afterwards the same model
    # and context run a normal forward that matches one from a fresh model
    m = ctx.deepclean(0, G.GW_BF16)
    assert G.gw_model_test_wait_timeout(m) == G.GW_ETIMEOUT
    G.gw_model_status(m)  # the flag was cleared and stays clear
    x = torch.randn(21, 4096, device="cuda", generator=torch.Generator(device="cuda").manual_seed(5))
    y = torch.empty(4096, device="cuda")
    G.gw_deepclean_forward(m, x.data_ptr(), 4096, 0, 1, 4096, y.data_ptr())
    m2 = ctx.deepclean(0, G.GW_BF16)
    y2 = torch.empty(4096, device="cuda")
    G.gw_deepclean_forward(m2, x.data_ptr(), 4096, 0, 1, 4096, y2.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(y, y2)
    G.gw_model_status(m)
