"""FP32 path parity against the FP64 oracle (relative L2 <= 1e-5).

Shapes span several CTA tiles with ragged tails; full-size cases (21 x 32768
windows, batch 256 BBHnet) are checked on sampled items the oracle computes
one by one.
"""
import numpy as np
import pytest
import torch

from oracle import fir as ofir, nets, stream as ostream
from paper_2108_12430_gb300 import gwstream as G, synth
from tests.gpu_util import Ctx, dev, rel_l2

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture
def ctx(gpu_lib):
    c = Ctx()
    yield c
    c.close()


def oracle_dc(x, seed, mean=None, std=None):
    return nets.deepclean_forward(x, synth.deepclean_params(seed), synth.DEEPCLEAN_LAYERS, mean, std)


def test_deepclean_config1_fp32(ctx):
    # 1 x 21 x 4096 (1 s at 4096 Hz)
    x = synth.witness_channels(0, 21, 4096)[None]
    m = ctx.deepclean(0)
    y = torch.zeros(1, 4096, device="cuda")
    xd = dev(x[0])
    G.gw_deepclean_forward(m, xd.data_ptr(), 4096, 0, 1, 4096, y.data_ptr())
    torch.cuda.synchronize()
    assert rel_l2(y.cpu().numpy(), oracle_dc(x, 0)) <= TOL32


@pytest.mark.parametrize("B,L,stride", [(3, 1000, 1000), (5, 2056, 264), (2, 8, 8), (1, 4104, 0)])
def test_deepclean_ragged_and_views_fp32(ctx, B, L, stride):
    ld = L + (B - 1) * stride
    xs = synth.witness_channels(3, 21, ld) * 2.0 + 0.5
    mean, std = np.full(21, 0.5), np.full(21, 2.0)
    m = ctx.deepclean(1, mean=mean, std=std)
    y = torch.zeros(B, L, device="cuda")
    G.gw_deepclean_forward(m, dev(xs).data_ptr(), ld, stride, B, L, y.data_ptr())
    torch.cuda.synchronize()
    wins = np.stack([xs[:, b * stride:b * stride + L] for b in range(B)])
    ref = oracle_dc(wins, 1, mean, std)
    for b in range(B):
        assert rel_l2(y[b].cpu().numpy(), ref[b]) <= TOL32, b


def test_deepclean_full_window_batch_sampled_fp32(ctx):
    # config-2 shape: 64 consecutive 21 x 32768 windows at stride 256; the
    # oracle checks two sampled windows.
    W, S, B = 32768, 256, 64
    ld = W + (B - 1) * S
    xs = synth.witness_channels(4, 21, ld)
    m = ctx.deepclean(2)
    y = torch.zeros(B, W, device="cuda")
    G.gw_deepclean_forward(m, dev(xs).data_ptr(), ld, S, B, W, y.data_ptr())
    torch.cuda.synchronize()
    for b in (0, 37):
        ref = oracle_dc(xs[None, :, b * S:b * S + W], 2)[0]
        assert rel_l2(y[b].cpu().numpy(), ref) <= TOL32, b


@pytest.mark.parametrize("B,L", [(3, 2048), (2, 512), (1, 16)])
def test_bbhnet_fp32(ctx, B, L):
    x = np.random.default_rng(B * 1000 + L).standard_normal((B, 2, L))
    m = ctx.bbhnet(0)
    out = torch.zeros(B, device="cuda")
    G.gw_bbhnet_score(m, dev(x).data_ptr(), B, L, out.data_ptr())
    torch.cuda.synchronize()
    layers = synth.bbhnet_layers()
    params, head = synth.bbhnet_params(0)
    ref = nets.bbhnet_forward(x, params, head, layers)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-4, atol=1e-4)
    assert rel_l2(out.cpu().numpy(), ref) <= TOL32 * 10


def test_bbhnet_batch256_sampled_fp32(ctx):
    x, label, snr = synth.injected_strain(9, 256, 2048)
    m = ctx.bbhnet(1)
    out = torch.zeros(256, device="cuda")
    G.gw_bbhnet_score(m, dev(x).data_ptr(), 256, 2048, out.data_ptr())
    torch.cuda.synchronize()
    params, head = synth.bbhnet_params(1)
    idx = [0, 17, 255]
    ref = nets.bbhnet_forward(x[idx], params, head, synth.bbhnet_layers())
    np.testing.assert_allclose(out.cpu().numpy()[idx], ref, rtol=1e-4, atol=1e-4)


def test_whitening_design_matches_oracle(ctx):
    fs, nfft = 2048.0, 8192
    f, psd = synth.psd_grid(fs, nfft)
    fh = G.gw_fir_create_whitening(ctx.h, psd, fs, 2049)
    ctx.objs.append((G.gw_fir_destroy, fh))
    taps = G.gw_fir_taps(fh)
    ref = ofir.whitening_fir(psd, fs, nfft, 2049)
    np.testing.assert_allclose(taps, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("B,C,L_in", [(256, 2, 4096), (3, 1, 2049), (2, 2, 5000)])
def test_whiten_fp32(ctx, B, C, L_in):
    fs, nfft = 2048.0, 8192
    f, psd = synth.psd_grid(fs, nfft)
    fh = G.gw_fir_create_whitening(ctx.h, psd, fs, 2049)
    ctx.objs.append((G.gw_fir_destroy, fh))
    x = synth.colored_noise(B + L_in, L_in, fs, n_ch=B * C).reshape(B, C, L_in)
    lout = L_in - 2048
    y = torch.zeros(B, C, lout, device="cuda")
    G.gw_whiten(fh, dev(x).data_ptr(), B, C, L_in, y.data_ptr())
    torch.cuda.synchronize()
    h = ofir.whitening_fir(psd, fs, nfft, 2049)
    rows = [0, B * C - 1] if B * C > 4 else range(B * C)
    xr = x.reshape(B * C, L_in)
    yr = y.reshape(B * C, lout).cpu().numpy()
    for r in rows:
        assert rel_l2(yr[r], ofir.fir_valid(xr[r], h)) <= TOL32


def stream_standardisation(seed, d):
    r = np.random.default_rng(1000 + seed + d)
    return r.normal(0, 0.2, 21).astype(np.float32), r.uniform(0.7, 1.4, 21).astype(np.float32)


def run_stream_case(ctx, W, S, pushes, mode, delta, seed=0, n_det=1, precision=G.GW_FP32, standardise=False,
                    post_taps=0):
    """Push the given batch sizes through a stream; compare with the oracle.
    With standardise, the models carry input mean / std, and the missing past
    before time 0 is a zero input sample that the model standardises."""
    n_total = sum(pushes)
    wit = [synth.witness_channels(seed + 10 * d, 21, n_total * S) for d in range(n_det)]
    strn = [synth.coupled_strain(seed + 10 * d, wit[d]) for d in range(n_det)]
    ms = [stream_standardisation(seed, d) if standardise else (None, None) for d in range(n_det)]
    models = [ctx.deepclean(seed + d, precision, *ms[d]) for d in range(n_det)]
    post, taps = None, None
    if post_taps:
        post = G.gw_fir_create_bandpass(ctx.h, 4096.0, 8192, post_taps)
        # the stream applies the taps in FP32
        taps = G.gw_fir_taps(post).astype(np.float32).astype(np.float64)
    s = G.gw_stream_create(ctx.h, models, n_det, 21, W, S, max(pushes), mode, delta, post)
    if post:
        G.gw_fir_destroy(post)  # the stream keeps its own copy of the taps
    ctx.objs.append((G.gw_stream_destroy, s))
    got = [[] for _ in range(n_det)]
    t = 0
    for n in pushes:
        w_in = np.ascontiguousarray(np.stack([wit[d][:, t * S:(t + n) * S] for d in range(n_det)]), np.float32)
        s_in = np.ascontiguousarray(np.stack([strn[d][t * S:(t + n) * S] for d in range(n_det)]), np.float32)
        out = np.zeros((n_det, n * S), np.float32)
        G.gw_stream_push(s, n, w_in, s_in, out)
        for d in range(n_det):
            got[d].append(out[d].reshape(n, S))
        t += n
    assert G.gw_stream_head(s) == n_total * S
    res = []
    for d in range(n_det):
        g = np.concatenate(got[d])
        # the oracle sees the same float32-rounded inputs
        w32 = wit[d].astype(np.float32).astype(np.float64)
        s32 = strn[d].astype(np.float32).astype(np.float64)
        params = synth.deepclean_params(seed + d)
        mean, std = [None if a is None else a.astype(np.float64) for a in ms[d]]
        fwd = lambda wins: nets.deepclean_forward(wins, params, synth.DEEPCLEAN_LAYERS, mean, std)
        snaps = None
        if mode == ostream.LATEST:
            snaps = list(range(n_total))
        _, ref = ostream.run_deepclean_stream(fwd, w32, s32, W, S, n_total, mode, delta, snaps, post=taps)
        res.append((g, ref))
    return res


@pytest.mark.parametrize("mode,delta", [(G.GW_AGG_LATEST, 0), (G.GW_AGG_AVERAGE, 1024 - 128),
                                        (G.GW_AGG_AVERAGE, 200)])
def test_stream_post_processing_fp32(ctx, mode, delta):
    # the aggregated prediction goes through a 129-tap band-pass before it is
    # subtracted; outputs arrive 64 samples later; two detectors
    W, S = 1024, 128
    for g, ref in run_stream_case(ctx, W, S, [3, 1, 5, 4, 2], mode, delta, seed=8, n_det=2, post_taps=129):
        assert g.shape == ref.shape
        assert rel_l2(g, ref) <= TOL32
        np.testing.assert_allclose(g, ref, rtol=1e-4, atol=1e-4)


def test_bandpass_design_matches_oracle(ctx):
    h = G.gw_fir_create_bandpass(ctx.h, 4096.0, 8192, 2049)
    try:
        np.testing.assert_allclose(G.gw_fir_taps(h), ofir.bandpass_fir(4096.0, 8192, 2049), rtol=0, atol=1e-13)
    finally:
        G.gw_fir_destroy(h)


def test_bulk_stride_half_window_fp32(ctx):
    # offline bulk mode (S = W / 2, two windows per sample)
    W, S = 2048, 1024
    for g, ref in run_stream_case(ctx, W, S, [4, 2, 5], G.GW_AGG_AVERAGE, W - S, seed=6):
        assert g.shape == ref.shape
        assert rel_l2(g, ref) <= TOL32


@pytest.mark.parametrize("mode,delta", [(G.GW_AGG_LATEST, 0), (G.GW_AGG_LATEST, 300),
                                        (G.GW_AGG_AVERAGE, 0), (G.GW_AGG_AVERAGE, 1024 - 128),
                                        (G.GW_AGG_AVERAGE, 200), (G.GW_AGG_AVERAGE, 202)])
def test_stream_matches_oracle_fp32(ctx, mode, delta):
    # (latency 202 is not a multiple of 4: the aggregation's one-time-per-lane form)
    W, S = 1024, 128
    for g, ref in run_stream_case(ctx, W, S, [3, 1, 5, 4, 2, 5], mode, delta):
        assert g.shape == ref.shape
        assert rel_l2(g, ref) <= TOL32
        np.testing.assert_allclose(g, ref, rtol=1e-4, atol=1e-4)


def test_stream_two_detectors_fp32(ctx):
    W, S = 512, 64
    for g, ref in run_stream_case(ctx, W, S, [2, 6, 1, 8], G.GW_AGG_AVERAGE, W - S, seed=3, n_det=2):
        assert rel_l2(g, ref) <= TOL32


@pytest.mark.parametrize("mode,delta", [(G.GW_AGG_LATEST, 0), (G.GW_AGG_AVERAGE, 1024 - 128)])
def test_stream_standardised_input_fp32(ctx, mode, delta):
    W, S = 1024, 128
    for g, ref in run_stream_case(ctx, W, S, [2, 3, 1, 4], mode, delta, seed=4, n_det=2, standardise=True):
        assert rel_l2(g, ref) <= TOL32


def test_stream_batch_equals_single_pushes_fp32(ctx):
    # The same stream pushed one snapshot at a time and 6 at a time gives the
    # same cleaned samples (state carried on the device between pushes).
    W, S = 1024, 128
    a = run_stream_case(ctx, W, S, [1] * 12, G.GW_AGG_AVERAGE, W - S, seed=5)[0][0]
    b = run_stream_case(ctx, W, S, [6, 6], G.GW_AGG_AVERAGE, W - S, seed=5)[0][0]
    np.testing.assert_allclose(a, b, rtol=2e-6, atol=2e-6)


def test_stream_errors(ctx):
    m = ctx.deepclean(0)
    with pytest.raises(G.GwError) as e:
        G.gw_stream_create(ctx.h, [m], 1, 21, 1000, 128, 4, G.GW_AGG_LATEST, 0)
    assert e.value.code == G.GW_EINVAL
    with pytest.raises(G.GwError) as e:
        G.gw_stream_create(ctx.h, [m], 1, 21, 1024, 128, 4, G.GW_AGG_AVERAGE, 1000)
    assert e.value.code == G.GW_EINVAL
    s = G.gw_stream_create(ctx.h, [m], 1, 21, 1024, 128, 4, G.GW_AGG_LATEST, 0)
    ctx.objs.append((G.gw_stream_destroy, s))
    w = np.zeros((1, 21, 128), np.float32)
    st = np.zeros((1, 128), np.float32)
    out = np.zeros((1, 128), np.float32)
    with pytest.raises(G.GwError) as e:
        G.gw_stream_push(s, 5, np.zeros((1, 21, 640), np.float32), np.zeros((1, 640), np.float32),
                         np.zeros((1, 640), np.float32))
    assert e.value.code == G.GW_EINVAL
    w[0, 3, 7] = np.nan
    with pytest.raises(G.GwError) as e:
        G.gw_stream_push(s, 1, w, st, out)
    assert e.value.code == G.GW_ENONFINITE
    assert G.gw_stream_head(s) == 0


@pytest.mark.parametrize("prec", [G.GW_FP32, G.GW_BF16])
def test_rejected_push_leaves_state_unchanged(ctx, prec):
    # a push with a non-finite witness or strain sample changes nothing: the
    # valid pushes that follow give exactly what a fresh stream gives
    m = ctx.deepclean(0, prec)
    rng = np.random.default_rng(7)
    W, S, n = 1024, 128, 3
    w = rng.standard_normal((1, 21, n * S)).astype(np.float32)
    x = rng.standard_normal((1, n * S)).astype(np.float32)

    def run(reject_first):
        s = G.gw_stream_create(ctx.h, [m], 1, 21, W, S, 4, G.GW_AGG_AVERAGE, W - S)
        ctx.objs.append((G.gw_stream_destroy, s))
        if reject_first:
            for bad_w in (True, False):
                wb, xb = w[:, :, :S].copy(), x[:, :S].copy()
                if bad_w:
                    wb[0, 20, S - 1] = np.inf
                else:
                    xb[0, 5] = np.nan
                with pytest.raises(G.GwError) as e:
                    G.gw_stream_push(s, 1, wb, xb, np.zeros((1, S), np.float32))
                assert e.value.code == G.GW_ENONFINITE
                assert G.gw_stream_head(s) == 0
        out = np.zeros((1, n * S), np.float32)
        for k in range(n):
            o = np.zeros((1, S), np.float32)
            G.gw_stream_push(s, 1, np.ascontiguousarray(w[:, :, k * S:(k + 1) * S]),
                             np.ascontiguousarray(x[:, k * S:(k + 1) * S]), o)
            out[:, k * S:(k + 1) * S] = o
        assert G.gw_stream_head(s) == n * S
        return out

    assert np.array_equal(run(True), run(False))


def test_budget_refusal(gpu_lib):
    c = Ctx(budget=4 << 20)
    try:
        m = c.deepclean(0)  # ~0.3 MB of weights fits
        with pytest.raises(G.GwError) as e:
            G.gw_stream_create(c.h, [m], 1, 21, 32768, 256, 64, G.GW_AGG_AVERAGE, 32768 - 256)
        assert e.value.code == G.GW_EBUDGET
        used = G.gw_ctx_bytes_in_use(c.h)
        assert used < 4 << 20
    finally:
        c.close()
