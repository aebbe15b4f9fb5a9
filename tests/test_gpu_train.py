"""Training path (DeepClean forward with tape, band-limited PSD-weighted loss,
hand-written backward, Adam) against the FP64 oracle's analytic gradient and
FP64 central finite differences.

Tolerances: FP32 path, relative L2 <= 1e-5 on the loss, the prediction and
every parameter group's gradient against the oracle; <= 1e-4 against finite
differences on sampled parameters (21 x 512 instance).
"""
import numpy as np
import pytest
import torch

from oracle import fir as ofir, grad as ograd
from paper_2108_12430_gb300 import autograd as GA, gwstream as G, synth
from tests.gpu_util import Ctx, dev, rel_l2

pytestmark = pytest.mark.gpu
TOL32 = 1e-5
C = 21
KEYS = ("w", "b", "gamma", "beta")


@pytest.fixture
def ctx(gpu_lib):
    c = Ctx()
    yield c
    c.close()


def case(B, L, seed=5, ntaps=129, nfft=2048):
    params = synth.deepclean_params(seed)
    x = np.stack([synth.witness_channels(6 + b, C, L) for b in range(B)]).astype(np.float32)
    s = (np.random.default_rng(seed).standard_normal((B, L)) * 0.3).astype(np.float32)
    r = np.random.default_rng(100 + seed)
    mean = r.normal(0, 0.1, C).astype(np.float32)
    std = r.uniform(0.8, 1.25, C).astype(np.float32)
    _, psd = synth.psd_grid(4096.0, nfft)
    return params, x, s, mean, std, psd, ntaps, nfft


def oracle(params, x, s, mean, std, psd, ntaps, nfft):
    g = ofir.band_loss_fir(psd, 4096.0, nfft, ntaps)
    xs = (x.astype(np.float64) - mean.astype(np.float64)[None, :, None]) / std.astype(np.float64)[None, :, None]
    return ograd.deepclean_loss_and_grad(xs, s.astype(np.float64), params, synth.DEEPCLEAN_LAYERS, g)


def flat_grads(grads):
    """Oracle gradients in the library's flat order (running stats: 0)."""
    parts = []
    for gr, spec in zip(grads, synth.DEEPCLEAN_LAYERS):
        for k in synth.PARAM_ORDER:
            if k in gr:
                parts.append(np.asarray(gr[k], np.float64).ravel())
            elif k in ("mean", "var") and spec[8]:
                parts.append(np.zeros(spec[2]))
    return np.concatenate(parts)


def check_grads(dp, ref, params, tol=TOL32):
    """Every layer's gradient (w, b, gamma, beta together) within tol, and every
    group within tol when its exact norm is at least 1e-3 of its layer's.  A
    smaller group is a sum that cancels to far below its terms (the output
    bias gradient is sum dL/dy_hat, proportional to the loss filter's DC gain,
    about 1e-10 here), so FP32 rounding of the terms decides its error."""
    worst = 0.0
    by_layer = {}
    for li, k, sl in groups(params):
        if k in ("mean", "var"):
            assert not dp[sl].any()
            continue
        by_layer.setdefault(li, []).append((k, sl))
    for li, gs in by_layer.items():
        idx = np.concatenate([np.arange(sl.start, sl.stop) for _, sl in gs])
        e = rel_l2(dp[idx], ref[idx])
        assert e <= tol, (li, e)
        worst = max(worst, e)
        ln = np.linalg.norm(ref[idx])
        for k, sl in gs:
            if np.linalg.norm(ref[sl]) >= 1e-3 * ln:
                e = rel_l2(dp[sl], ref[sl])
                assert e <= tol, (li, k, e)
                worst = max(worst, e)
    return worst


def groups(params):
    """(layer, key, slice) of every parameter group in the flat vector."""
    out, o = [], 0
    for li, p in enumerate(params):
        for k in synth.PARAM_ORDER:
            if k in p:
                n = np.asarray(p[k]).size
                out.append((li, k, slice(o, o + n)))
                o += n
    return out


class Run:
    """A trainer, a loss FIR and device buffers for one case."""

    def __init__(self, ctx, params, x, s, mean, std, psd, ntaps, nfft, checkpoint=0, B_max=None, precision=G.GW_FP32,
                 tc_data=0):
        B, _, L = x.shape
        self.B, self.L = B, L
        self.t = G.gw_trainer_create(ctx.h, C, B_max or B, L, checkpoint, mean, std, precision=precision,
                                     tc_data=tc_data)
        ctx.objs.append((G.gw_trainer_destroy, self.t))
        self.g = G.gw_fir_create_band_loss(ctx.h, psd, 4096.0, ntaps)
        ctx.objs.append((G.gw_fir_destroy, self.g))
        self.K = ntaps
        self.p = dev(synth.flatten_params(params))
        assert self.p.numel() == G.gw_trainer_param_count(self.t)
        self.x, self.s = dev(x), dev(s)

    def step(self, B=None, x=None, s=None):
        B = B or self.B
        x = self.x if x is None else x
        s = self.s if s is None else s
        y = torch.empty(B, self.L, device="cuda")
        loss = torch.empty(1, device="cuda")
        r = torch.empty(B, self.L - self.K + 1, device="cuda")
        dy = torch.empty(B, self.L, device="cuda")
        dp = torch.empty_like(self.p)
        G.gw_trainer_forward(self.t, self.p.data_ptr(), x.data_ptr(), B, y.data_ptr())
        G.gw_band_loss(self.g, s.data_ptr(), y.data_ptr(), B, self.L, loss.data_ptr(), r.data_ptr())
        G.gw_band_loss_backward(self.g, r.data_ptr(), B, self.L, 0, dy.data_ptr())
        G.gw_trainer_backward(self.t, dy.data_ptr(), dp.data_ptr())
        torch.cuda.synchronize()
        return float(loss.item()), y.cpu().numpy(), dp.cpu().numpy()


def test_band_loss_design_matches_oracle(ctx):
    _, psd = synth.psd_grid(4096.0, 8192)
    f = G.gw_fir_create_band_loss(ctx.h, psd, 4096.0, 2049)
    ctx.objs.append((G.gw_fir_destroy, f))
    ref = ofir.band_loss_fir(psd, 4096.0, 8192, 2049)
    np.testing.assert_allclose(G.gw_fir_taps(f), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("checkpoint", [0, 1])
def test_loss_and_gradient_match_oracle_fp32(ctx, checkpoint):
    c = case(2, 512)
    loss_ref, y_ref, grads_ref = oracle(*c)
    loss, y, dp = Run(ctx, *c, checkpoint=checkpoint).step()
    assert abs(loss - loss_ref) <= TOL32 * abs(loss_ref)
    assert rel_l2(y, y_ref) <= TOL32
    worst = check_grads(dp, flat_grads(grads_ref), c[0])
    print("worst gradient rel-L2", worst)


def test_gradient_matches_finite_differences(ctx):
    # FP32 GPU gradient against FP64 central differences of the oracle loss
    c = case(1, 512)
    params, x, s, mean, std, psd, ntaps, nfft = c
    _, _, dp = Run(ctx, *c).step()
    g = ofir.band_loss_fir(psd, 4096.0, nfft, ntaps)
    xs = (x.astype(np.float64) - mean[None, :, None]) / std[None, :, None]
    rr = np.random.default_rng(11)
    fd, an = [], []
    for li, k, sl in groups(params):
        if k not in KEYS:
            continue
        for _ in range(2):
            j = int(rr.integers(0, sl.stop - sl.start))
            eps = 1e-5 * max(1.0, abs(float(np.asarray(params[li][k]).ravel()[j])))
            vals = []
            for sign in (1, -1):
                q = [dict((kk, np.array(v, np.float64)) for kk, v in p.items()) for p in params]
                flat = q[li][k].reshape(-1)
                flat[j] += sign * eps
                vals.append(ograd.deepclean_loss(xs, s.astype(np.float64), q, synth.DEEPCLEAN_LAYERS, g))
            fd.append((vals[0] - vals[1]) / (2 * eps))
            an.append(dp[sl.start + j])
    fd, an = np.array(fd), np.array(an)
    err = rel_l2(an, fd)
    print("sampled gradient vs finite differences rel-L2", err)
    assert err <= 1e-4


# BF16 weight gradients: rounding both operands of every product to BF16
# bounds its relative error by about 2^-8 = 3.9e-3; sums whose terms partly
# cancel can exceed that by a small factor, hence 1e-2 (the data gradients,
# bias gradients and the loss stay FP32).
TOL_WG16 = 1e-2


@pytest.mark.parametrize("B,L,ntaps,nfft", [(2, 512, 129, 2048), (2, 8192, 2049, 8192)])
def test_tensor_core_weight_gradients_match_oracle(ctx, B, L, ntaps, nfft):
    c = case(B, L, ntaps=ntaps, nfft=nfft)
    loss_ref, y_ref, grads_ref = oracle(*c)
    run = Run(ctx, *c, precision=G.GW_BF16)
    loss, y, dp = run.step()
    G.gw_trainer_status(run.t)
    assert abs(loss - loss_ref) <= TOL32 * abs(loss_ref)
    assert rel_l2(y, y_ref) <= TOL32
    worst = check_grads(dp, flat_grads(grads_ref), c[0], tol=TOL_WG16)
    print("BF16 weight gradients: worst rel-L2", worst)
    # the FP32 trainer on the same case stays within the same bound of it
    _, _, dp32 = Run(ctx, *c).step()
    assert rel_l2(dp, dp32) <= TOL_WG16


# Forward convs and data gradients on the tensor cores too: the prediction
# carries the BF16 path's error (bound 2e-2, as for inference); a gradient
# combines that forward error with the BF16 rounding of the backward operands,
# so its bound is twice that, 4e-2.
TOL_TC16_Y, TOL_TC16_G = 2e-2, 4e-2


@pytest.mark.parametrize("B,L,ntaps,nfft", [(2, 512, 129, 2048), (2, 8192, 2049, 8192)])
def test_tensor_core_training_step_matches_oracle(ctx, B, L, ntaps, nfft):
    c = case(B, L, ntaps=ntaps, nfft=nfft)
    loss_ref, y_ref, grads_ref = oracle(*c)
    run = Run(ctx, *c, precision=G.GW_BF16, tc_data=1)
    loss, y, dp = run.step()
    G.gw_trainer_status(run.t)
    print(f"tensor-core step: loss rel err {abs(loss - loss_ref) / abs(loss_ref):.2e}, y rel-L2 {rel_l2(y, y_ref):.2e}")
    assert abs(loss - loss_ref) <= TOL_TC16_Y * abs(loss_ref)
    assert rel_l2(y, y_ref) <= TOL_TC16_Y
    print("worst gradient rel-L2", check_grads(dp, flat_grads(grads_ref), c[0], tol=TOL_TC16_G))
    # checkpointing recomputes through the same kernels: identical bits
    b = Run(ctx, *c, precision=G.GW_BF16, tc_data=1, checkpoint=1).step()
    assert b[0] == loss and np.array_equal(b[1], y) and np.array_equal(b[2], dp)


def test_full_length_gradient_and_batch_mean_property(ctx):
    # Windows of the training configuration's length (8192): a batch of 2
    # against the oracle, then a batch of 8 equals the mean of its four
    # 2-window batches (the loss is a mean over samples).
    c = case(8, 8192, ntaps=2049, nfft=8192)
    params, x, s = c[0], c[1], c[2]
    run = Run(ctx, *c, B_max=8)
    c2 = (params, x[:2], s[:2]) + c[3:]
    loss_ref, _, grads_ref = oracle(*c2)
    loss2, _, dp2 = run.step(2, dev(x[:2]), dev(s[:2]))
    assert abs(loss2 - loss_ref) <= TOL32 * abs(loss_ref)
    print("full-length worst gradient rel-L2", check_grads(dp2, flat_grads(grads_ref), params))
    loss8, _, dp8 = run.step()
    parts = [run.step(2, dev(x[i:i + 2]), dev(s[i:i + 2])) for i in range(0, 8, 2)]
    assert abs(loss8 - np.mean([p[0] for p in parts])) <= 1e-5 * abs(loss8)
    assert rel_l2(dp8, np.mean([p[2] for p in parts], axis=0)) <= 1e-5


def test_checkpointing_gives_identical_gradients(ctx):
    c = case(3, 1024)
    a = Run(ctx, *c, checkpoint=0).step()
    b = Run(ctx, *c, checkpoint=1).step()
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_autograd_functions(ctx):
    c = case(2, 512)
    run = Run(ctx, *c)
    _, _, dp = run.step()
    params = run.p.clone().requires_grad_(True)
    y = GA.DeepCleanFn.apply(run.x, params, run.t)
    loss = GA.BandLossFn.apply(run.s, y, run.g)
    loss.backward()
    assert np.array_equal(params.grad.cpu().numpy(), dp)


def test_fir_backward_is_the_adjoint(ctx):
    _, psd = synth.psd_grid(2048.0, 1024)
    f = G.gw_fir_create_whitening(ctx.h, psd, 2048.0, 257)
    ctx.objs.append((G.gw_fir_destroy, f))
    h = G.gw_fir_taps(f).astype(np.float32).astype(np.float64)
    r = np.random.default_rng(3)
    B, Cc, L = 2, 3, 3000
    x = r.standard_normal((B, Cc, L)).astype(np.float32)
    dy = r.standard_normal((B, Cc, L - 256)).astype(np.float32)
    xd = dev(x).requires_grad_(True)
    y = GA.FirFn.apply(xd, f)
    y.backward(dev(dy))
    dx = xd.grad.cpu().numpy()
    # the full convolution of dy with h, written out by the numpy library routine
    ref = np.stack([[np.convolve(dy[b, c].astype(np.float64), h) for c in range(Cc)] for b in range(B)])
    assert rel_l2(dx, ref) <= TOL32
    lhs = float(np.sum(y.detach().cpu().numpy().astype(np.float64) * dy))
    rhs = float(np.sum(x.astype(np.float64) * dx))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_adam_step(ctx):
    r = np.random.default_rng(4)
    n = 10001
    p0, g = r.standard_normal(n).astype(np.float32), r.standard_normal(n).astype(np.float32)
    m0, v0 = (r.standard_normal(n) * 0.1).astype(np.float32), np.abs(r.standard_normal(n) * 0.1).astype(np.float32)
    p, m, v, gd = dev(p0), dev(m0), dev(v0), dev(g)
    G.gw_adam_step(p.data_ptr(), gd.data_ptr(), m.data_ptr(), v.data_ptr(), n, 3, 1e-3)
    torch.cuda.synchronize()
    # Adam (Kingma & Ba 2015, Algorithm 1) in float64
    mm = 0.9 * m0 + 0.1 * g.astype(np.float64)
    vv = 0.999 * v0 + 0.001 * g.astype(np.float64) ** 2
    pp = p0 - 1e-3 * (mm / (1 - 0.9 ** 3)) / (np.sqrt(vv / (1 - 0.999 ** 3)) + 1e-8)
    assert rel_l2(m.cpu().numpy(), mm) <= 1e-6 and rel_l2(v.cpu().numpy(), vv) <= 1e-6
    assert np.abs(p.cpu().numpy() - pp).max() <= 1e-6


def test_adam_step_with_device_step_count(ctx):
    # three updates with the count on the device against three with the count from the host
    r = np.random.default_rng(5)
    n = 4099
    p0, m0 = r.standard_normal(n).astype(np.float32), (r.standard_normal(n) * 0.1).astype(np.float32)
    v0 = np.abs(r.standard_normal(n) * 0.1).astype(np.float32)
    grads = [dev(r.standard_normal(n).astype(np.float32)) for _ in range(3)]
    a = [dev(p0), dev(m0), dev(v0)]
    b = [dev(p0), dev(m0), dev(v0)]
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    for it, gd in enumerate(grads, 1):
        G.gw_adam_step(a[0].data_ptr(), gd.data_ptr(), a[1].data_ptr(), a[2].data_ptr(), n, it, 1e-3)
        G.gw_adam_step_dev(b[0].data_ptr(), gd.data_ptr(), b[1].data_ptr(), b[2].data_ptr(), n, step.data_ptr(), 1e-3)
    torch.cuda.synchronize()
    assert int(step.item()) == 3
    for x, y in zip(a, b):
        # the bias corrections come from the device's powf instead of the host's
        assert rel_l2(y.cpu().numpy(), x.cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("precision,tc_data", [(G.GW_FP32, 0), (G.GW_BF16, 1)])
def test_training_step_replays_as_a_cuda_graph(ctx, precision, tc_data):
    # forward, loss, backward and Adam (device step count) captured once and
    # replayed: two replays give the parameters of two eager steps exactly
    c = case(2, 1024)
    runs = [Run(ctx, *c, precision=precision, tc_data=tc_data) for _ in range(2)]
    bufs = []
    for run in runs:
        B, L, K = run.B, run.L, run.K
        bufs.append(dict(y=torch.empty(B, L, device="cuda"), loss=torch.empty(1, device="cuda"),
                         r=torch.empty(B, L - K + 1, device="cuda"), dy=torch.empty(B, L, device="cuda"),
                         dp=torch.empty_like(run.p), m=torch.zeros_like(run.p), v=torch.zeros_like(run.p),
                         step=torch.zeros(1, dtype=torch.int32, device="cuda")))

    def step(run, b, st):
        G.gw_trainer_forward(run.t, run.p.data_ptr(), run.x.data_ptr(), run.B, b["y"].data_ptr(), st)
        G.gw_band_loss(run.g, run.s.data_ptr(), b["y"].data_ptr(), run.B, run.L, b["loss"].data_ptr(),
                       b["r"].data_ptr(), st)
        G.gw_band_loss_backward(run.g, b["r"].data_ptr(), run.B, run.L, 0, b["dy"].data_ptr(), st)
        G.gw_trainer_backward(run.t, b["dy"].data_ptr(), b["dp"].data_ptr(), st)
        G.gw_adam_step_dev(run.p.data_ptr(), b["dp"].data_ptr(), b["m"].data_ptr(), b["v"].data_ptr(),
                           run.p.numel(), b["step"].data_ptr(), 1e-3, stream=st)

    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        for _ in range(2):
            step(runs[0], bufs[0], side.cuda_stream)
    side.synchronize()
    # a warm-up eager step on the graph run's own buffers first (lazy set-up
    # happens outside the capture), then its parameters and moments reset
    p_init = runs[1].p.clone()
    with torch.cuda.stream(side):
        step(runs[1], bufs[1], side.cuda_stream)
    side.synchronize()
    runs[1].p.copy_(p_init)
    for k in ("m", "v", "step"):
        bufs[1][k].zero_()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step(runs[1], bufs[1], torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    assert int(bufs[1]["step"].item()) == 2
    assert torch.equal(runs[0].p, runs[1].p)
    assert torch.equal(bufs[0]["m"], bufs[1]["m"]) and torch.equal(bufs[0]["v"], bufs[1]["v"])


@pytest.mark.parametrize("precision,tc_data", [(G.GW_FP32, 0), (G.GW_BF16, 0), (G.GW_BF16, 1)])
def test_training_reduces_the_loss(ctx, precision, tc_data):
    c = case(4, 1024)
    run = Run(ctx, *c, precision=precision, tc_data=tc_data)
    m = torch.zeros_like(run.p)
    v = torch.zeros_like(run.p)
    losses = []
    for it in range(1, 31):
        loss, _, dp = run.step()
        losses.append(loss)
        g = dev(dp)
        G.gw_adam_step(run.p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), run.p.numel(), it, 1e-2)
    print("loss", losses[0], "->", losses[-1])
    assert losses[-1] < 0.5 * losses[0]
