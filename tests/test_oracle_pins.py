"""Pins for the FP64 oracle against things other than itself (CPU only).

Each test ties an oracle function to a library routine (PyTorch float64 on
CPU), a closed form, an invariant or finite differences, so that a dropped
term, wrong sign or index, or transposed operand in the oracle fails here.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import fir, grad, layers as Lyr, nets, spectral, stream
from paper_2108_12430_gb300 import synth

rng = np.random.default_rng(12345)


def t64(a):
    return torch.from_numpy(np.asarray(a, np.float64))


# ----------------------------------------------------------------------------
# Layers: library special cases, impulse response, adjoint identity
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("cin,cout,K,s,pl,pr,L", [
    (3, 5, 7, 1, 3, 3, 40), (4, 2, 7, 2, 3, 3, 33), (2, 3, 16, 1, 7, 8, 50),
    (5, 4, 1, 2, 0, 0, 17), (21, 8, 7, 1, 3, 3, 64)])
def test_conv1d_matches_torch(cin, cout, K, s, pl, pr, L):
    x = rng.standard_normal((2, cin, L))
    w = rng.standard_normal((cout, cin, K))
    b = rng.standard_normal(cout)
    ref = F.conv1d(F.pad(t64(x), (pl, pr)), t64(w), t64(b), stride=s).numpy()
    np.testing.assert_allclose(Lyr.conv1d(x, w, b, s, pl, pr), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("cin,cout,K,s,p,op,L", [
    (4, 3, 7, 2, 3, 1, 9), (64, 32, 7, 2, 3, 1, 16), (2, 5, 5, 3, 1, 2, 7), (3, 3, 7, 1, 3, 0, 12)])
def test_conv_transpose1d_matches_torch(cin, cout, K, s, p, op, L):
    x = rng.standard_normal((2, cin, L))
    w = rng.standard_normal((cin, cout, K))
    b = rng.standard_normal(cout)
    ref = F.conv_transpose1d(t64(x), t64(w), t64(b), stride=s, padding=p, output_padding=op).numpy()
    got = Lyr.conv_transpose1d(x, w, b, s, p, op)
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_conv1d_delta_impulse_reproduces_kernel():
    cin, cout, K, p, L, t0, i0 = 3, 4, 7, 3, 32, 15, 1
    w = rng.standard_normal((cout, cin, K))
    x = np.zeros((1, cin, L))
    x[0, i0, t0] = 1.0
    y = Lyr.conv1d(x, w, np.zeros(cout), 1, p, p)
    for k in range(K):
        np.testing.assert_array_equal(y[0, :, t0 + p - k], w[:, i0, k])
    mask = np.ones(L, bool)
    mask[t0 + p - K + 1:t0 + p + 1] = False
    assert np.all(y[0][:, mask] == 0.0)


def test_conv_transpose1d_delta_impulse():
    cin, cout, K, s, p, op, L, t0 = 2, 3, 7, 2, 3, 1, 10, 4
    w = rng.standard_normal((cin, cout, K))
    x = np.zeros((1, cin, L))
    x[0, 1, t0] = 1.0
    y = Lyr.conv_transpose1d(x, w, np.zeros(cout), s, p, op)
    for k in range(K):
        np.testing.assert_array_equal(y[0, :, s * t0 + k - p], w[1, :, k])


def test_conv_transpose_is_adjoint_of_strided_conv():
    # <convT(x; w), y> = <x, conv(y; w)>: the transposed conv is the adjoint of
    # the strided conv with the same taps (crop <-> zero-pad).
    cin, cout, K, s, p, op, L = 5, 3, 7, 2, 3, 1, 11
    w = rng.standard_normal((cin, cout, K))
    x = rng.standard_normal((1, cin, L))
    lout = (L - 1) * s - 2 * p + K + op
    y = rng.standard_normal((1, cout, lout))
    lhs = np.sum(Lyr.conv_transpose1d(x, w, np.zeros(cout), s, p, op) * y)
    z = Lyr.conv1d(y, w, np.zeros(cin), s, p, p - op)
    assert z.shape == x.shape
    rhs = np.sum(x * z)
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def test_bn_fold_equals_unfolded():
    for kind, axis in (("conv", 0), ("convT", 1)):
        cin, cout = 6, 4
        shape = (cout, cin, 7) if kind == "conv" else (cin, cout, 7)
        w = rng.standard_normal(shape)
        b = rng.standard_normal(cout)
        g, bt = rng.uniform(0.5, 1.5, cout), rng.standard_normal(cout)
        m, v = rng.standard_normal(cout), rng.uniform(0.5, 2, cout)
        x = rng.standard_normal((2, cin, 20))
        if kind == "conv":
            ref = Lyr.batchnorm_eval(Lyr.conv1d(x, w, b, 1, 3, 3), g, bt, m, v)
            w2, b2 = Lyr.fold_bn(w, b, g, bt, m, v, out_axis=axis)
            got = Lyr.conv1d(x, w2, b2, 1, 3, 3)
        else:
            ref = Lyr.batchnorm_eval(Lyr.conv_transpose1d(x, w, b, 2, 3, 1), g, bt, m, v)
            w2, b2 = Lyr.fold_bn(w, b, g, bt, m, v, out_axis=axis)
            got = Lyr.conv_transpose1d(x, w2, b2, 2, 3, 1)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
        tbn = torch.nn.BatchNorm1d(cout, eps=Lyr.BN_EPS).double().eval()
        with torch.no_grad():
            tbn.weight.copy_(t64(g)); tbn.bias.copy_(t64(bt))
            tbn.running_mean.copy_(t64(m)); tbn.running_var.copy_(t64(v))
        z = rng.standard_normal((2, cout, 9))
        np.testing.assert_allclose(Lyr.batchnorm_eval(z, g, bt, m, v), tbn(t64(z)).detach().numpy(), rtol=1e-12)


# ----------------------------------------------------------------------------
# Networks against a PyTorch float64 module stack (a library special case)
# ----------------------------------------------------------------------------

def torch_layer(spec, p):
    kind, cin, cout, k, s, pl, pr, op, bn, act = spec
    mods = []
    if kind == "conv":
        if pl != pr:
            mods.append(torch.nn.ConstantPad1d((pl, pr), 0.0))
            c = torch.nn.Conv1d(cin, cout, k, stride=s, padding=0)
        else:
            c = torch.nn.Conv1d(cin, cout, k, stride=s, padding=pl)
    else:
        c = torch.nn.ConvTranspose1d(cin, cout, k, stride=s, padding=pl, output_padding=op)
    c = c.double()
    with torch.no_grad():
        c.weight.copy_(t64(p["w"])); c.bias.copy_(t64(p["b"]))
    mods.append(c)
    if bn:
        m = torch.nn.BatchNorm1d(cout, eps=1e-5).double().eval()
        with torch.no_grad():
            m.weight.copy_(t64(p["gamma"])); m.bias.copy_(t64(p["beta"]))
            m.running_mean.copy_(t64(p["mean"])); m.running_var.copy_(t64(p["var"]))
        mods.append(m)
    if act == "tanh":
        mods.append(torch.nn.Tanh())
    elif act == "relu":
        mods.append(torch.nn.ReLU())
    return torch.nn.Sequential(*mods).eval()


def test_deepclean_matches_torch_modules():
    params = synth.deepclean_params(0)
    x = synth.witness_channels(1, 21, 4096)[None]
    model = torch.nn.Sequential(*[torch_layer(s, p) for s, p in zip(synth.DEEPCLEAN_LAYERS, params)])
    ref = model(t64(x)).detach().numpy()[:, 0]
    got = nets.deepclean_forward(x, params, synth.DEEPCLEAN_LAYERS)
    assert got.shape == (1, 4096)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12)


def test_deepclean_standardisation():
    params = synth.deepclean_params(3)
    x = rng.standard_normal((1, 21, 256)) * 3.0 + 2.0
    mu, sd = np.full(21, 2.0), np.full(21, 3.0)
    a = nets.deepclean_forward(x, params, synth.DEEPCLEAN_LAYERS, mu, sd)
    b = nets.deepclean_forward((x - 2.0) / 3.0, params, synth.DEEPCLEAN_LAYERS)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_bbhnet_matches_torch_modules():
    layers = synth.bbhnet_layers()
    params, head = synth.bbhnet_params(0)
    x = rng.standard_normal((3, 2, 2048))
    mods = [torch_layer(s, p) for s, p in zip(layers, params)]
    h = mods[0](t64(x))
    for i in range(1, len(mods), 3):
        h = torch.relu(mods[i + 1](mods[i](h)) + mods[i + 2](h))
    ref = (h.mean(-1) @ t64(head["w"]) + float(head["b"][0])).detach().numpy()
    got = nets.bbhnet_forward(x, params, head, layers)
    assert h.shape[-1] == 128
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-10)


# ----------------------------------------------------------------------------
# FIR design: invariants of the designed filters
# ----------------------------------------------------------------------------

def test_whitening_flattens_coloured_noise():
    fs, nfft = 2048.0, 8192
    f, psd = synth.psd_grid(fs, nfft)
    h = fir.whitening_fir(psd, fs, nfft, 2049)
    x = synth.colored_noise(11, 1 << 18, fs)[0]
    y = fir.fir_valid(x, h)
    assert abs(np.var(y) - 1.0) < 0.02
    from scipy import signal
    ff, pyy = signal.welch(y, fs=fs, nperseg=int(2 * fs), noverlap=int(fs), window="hann")
    # flat ASD sqrt(2/fs): PSD averaged over 20 Hz sub-bands (40 bins x ~127
    # Welch segments each, so the estimator's own scatter is ~1.5%)
    for lo in np.arange(30.0, 900.0, 20.0):
        band = (ff >= lo) & (ff < lo + 20.0)
        assert abs(np.sqrt(pyy[band].mean()) / np.sqrt(2.0 / fs) - 1.0) < 0.05, lo


def test_whitening_sinusoid_amplitude_and_linearity():
    fs, nfft = 2048.0, 8192
    f, psd = synth.psd_grid(fs, nfft)
    h = fir.whitening_fir(psd, fs, nfft, 2049)
    n = np.arange(8192)
    for f0 in (40.0, 100.25, 300.0):
        x = np.cos(2 * np.pi * f0 * n / fs)
        y = fir.fir_valid(x, h)
        # closed-form DTFT magnitude of the taps
        np.testing.assert_allclose(np.max(np.abs(y)), fir.freq_response(h, f0, fs)[0], rtol=2e-3)
        # and the design target sqrt(2 / (fs S)) away from the band edge
        np.testing.assert_allclose(fir.freq_response(h, f0, fs)[0],
                                   np.sqrt(2.0 / (fs * synth.aligo_psd(f0))), rtol=0.03)
    a, b = rng.standard_normal(4096), rng.standard_normal(4096)
    np.testing.assert_allclose(fir.fir_valid(2 * a - 3 * b, h),
                               2 * fir.fir_valid(a, h) - 3 * fir.fir_valid(b, h), rtol=1e-9, atol=1e-12)


def test_whitening_taps_symmetric_and_direct_dft():
    # zero-phase design => symmetric taps; compare the direct DFT with numpy's irfft
    fs, nfft = 2048.0, 8192
    f, psd = synth.psd_grid(fs, nfft)
    h = fir.whitening_fir(psd, fs, nfft, 2049)
    np.testing.assert_allclose(h, h[::-1], rtol=1e-10, atol=1e-14 * np.abs(h).max())
    h0 = np.fft.irfft(np.sqrt(2.0 / (fs * psd)), n=nfft)
    ref = np.concatenate([h0[-1024:], h0[:1025]]) * fir.hann(2049)
    np.testing.assert_allclose(h, ref, rtol=1e-9, atol=1e-12 * np.abs(h).max())


def test_lowpass_response():
    h = fir.lowpass_fir(127, 900.0, 4096.0)
    assert abs(fir.freq_response(h, 0.0, 4096.0)[0] - 1.0) < 1e-12
    assert np.all(np.abs(fir.freq_response(h, np.linspace(0, 700, 50), 4096.0) - 1.0) < 0.01)
    assert np.all(fir.freq_response(h, np.linspace(1150, 2048, 60), 4096.0) < 2e-3)


def test_band_loss_filter_response():
    fs, nfft = 4096.0, 16384
    f, psd = synth.psd_grid(fs, nfft)
    g = fir.band_loss_fir(psd, fs, nfft, 2049)
    r = fir.freq_response(g, [59.0, 60.0, 61.0], fs)
    ref = np.sqrt(synth.aligo_psd(60.0) / synth.aligo_psd(np.array([59.0, 60.0, 61.0])))
    np.testing.assert_allclose(r, ref, rtol=0.03)
    assert np.all(fir.freq_response(g, np.array([20.0, 40.0, 80.0, 200.0, 1000.0]), fs) < 0.01)


def test_bandpass_response():
    fs = 4096.0
    # long enough for the 6 Hz flat top: within 1% of 1 on [58, 62] Hz
    h = fir.bandpass_fir(fs, 16384, 8191)
    assert np.allclose(h, h[::-1], atol=1e-15)
    np.testing.assert_allclose(fir.freq_response(h, np.linspace(58.0, 62.0, 9), fs), 1.0, atol=0.01)
    assert np.all(fir.freq_response(h, np.array([0.0, 20.0, 45.0, 50.0, 70.0, 80.0, 200.0, 1000.0]), fs) < 1e-3)
    # the 2049-tap version used online (0.25 s delay): unit gain at 60 Hz, the
    # Hann window widens the ramps to about 8 Hz
    h = fir.bandpass_fir(fs, 8192, 2049)
    np.testing.assert_allclose(fir.freq_response(h, [60.0], fs), 1.0, atol=0.01)
    assert np.all(fir.freq_response(h, np.array([0.0, 20.0, 45.0, 75.0, 80.0, 200.0, 1000.0]), fs) < 0.01)


def test_clean_post_one_tap_is_plain_subtraction():
    # with a single unit tap the post-processed path subtracts the aggregated
    # prediction itself; before time 0 both strain and prediction count as 0
    x = rng.standard_normal(3000)
    agg = rng.standard_normal((6, 128))
    for delta in (0, 100):
        got = stream.clean_post(x, agg, 128, delta, np.ones(1)).reshape(-1)
        want = stream.clean(x, agg, 128, delta).reshape(-1)
        t = np.arange(-delta, 6 * 128 - delta)
        np.testing.assert_array_equal(got[t >= 0], want[t >= 0])
        assert np.all(got[t < 0] == 0.0)


def test_clean_post_is_a_delayed_convolution():
    # brute force: the emitted prediction series (zero before time 0), full
    # convolution with the symmetric taps, read c samples late
    S, n, delta, K = 64, 9, 40, 31
    h = np.hanning(K + 2)[1:-1]
    x = rng.standard_normal(n * S + 100)
    agg = rng.standard_normal((n, S))
    got = stream.clean_post(x, agg, S, delta, h)
    c = (K - 1) // 2
    t = np.arange(-delta, n * S - delta)  # emitted times
    p = np.where(t >= 0, agg.reshape(-1), 0.0)
    # q(t') = sum_j h[j] p(t' + j - c) on t' = t - c; p(u) = 0 for u < -delta
    pad = np.concatenate([np.zeros(2 * c), p])  # index i <-> time i - 2 c - delta
    q = np.convolve(pad, h[::-1], mode="valid")  # q[i] = sum_j h[j] pad[i + j] <-> t' = i - c - delta
    tq = np.arange(q.size) - c - delta
    want = np.where(tq >= 0, x[np.clip(tq, 0, None)], 0.0) - q
    np.testing.assert_allclose(got.reshape(-1), want[:n * S], atol=1e-12)


def test_decimate_alignment():
    h = fir.lowpass_fir()
    x = np.cos(2 * np.pi * 50.0 * np.arange(4096) / 4096.0)
    y = fir.decimate2(x, h, first=32)
    m = 32 + np.arange(y.shape[-1])
    np.testing.assert_allclose(y, np.cos(2 * np.pi * 50.0 * (2 * m) / 4096.0) * fir.freq_response(h, 50.0, 4096)[0],
                               atol=1e-9)


# ----------------------------------------------------------------------------
# Streaming: windows and aggregation against direct statements
# ----------------------------------------------------------------------------

def test_window_is_slice_of_stream():
    x = rng.standard_normal((3, 5000))
    W, S = 1024, 128
    for k in (0, 3, 7, 20, 30):
        w = stream.window(x, W, S, k)
        end = (k + 1) * S
        ref = np.zeros((3, W))
        if end >= W:
            ref = x[:, end - W:end]
        else:
            ref[:, W - end:] = x[:, :end]
        np.testing.assert_array_equal(w, ref)


def test_aggregation_identity_model():
    # A model that returns its input channel 0 predicts the same value for a
    # time in every window, so AVERAGE == LATEST == the signal itself.
    W, S, n = 512, 64, 20
    x = rng.standard_normal((2, n * S))
    s = rng.standard_normal(n * S)
    fwd = lambda wins: wins[:, 0, :]
    for mode in (stream.LATEST, stream.AVERAGE):
        for delta in (0, 64, 100, W - S):
            _, cl = stream.run_deepclean_stream(fwd, x, s, W, S, n, mode, delta)
            for k in range(n):
                t = stream.emit_times(k, S, delta)
                ok = t >= 0
                np.testing.assert_allclose(cl[k][ok], s[t[ok]] - x[0, t[ok]], atol=1e-12)


def test_average_is_mean_of_covering_windows():
    W, S, n = 256, 32, 16
    preds = rng.standard_normal((n, W))
    delta = W - S
    agg = stream.aggregate(preds, W, S, stream.AVERAGE, delta)
    # full overlap-add: once the stream is long enough each emitted sample is
    # the average of exactly W/S windows (k - W/S + 1 .. k)
    k = n - 1
    for i in range(S):
        tau = k * S - delta + i
        vals = [preds[j, tau - ((j + 1) * S - W)] for j in range(k - W // S + 1, k + 1)]
        assert len(vals) == W // S
        assert abs(agg[k, i] - sum(vals) / len(vals)) < 1e-12
    np.testing.assert_allclose(stream.aggregate(preds, W, S, stream.AVERAGE, 0),
                               stream.aggregate(preds, W, S, stream.LATEST, 0))


@pytest.mark.parametrize("W,S", [(256, 32), (128, 64), (64, 64), (96, 8)])
def test_aggregate_by_window_equals_per_sample_definition(W, S):
    # the per-window form used for long streams against the per-sample
    # statement (brute force on short streams), every mode and latency
    n = 3 * W // S + 2
    preds = rng.standard_normal((n, W))
    for mode in (stream.LATEST, stream.AVERAGE):
        for delta in sorted({0, 3, S // 2, W // 2, W - S} & set(range(0, W - S + 1))):
            ref = stream.aggregate(preds, W, S, mode, delta)
            np.testing.assert_allclose(stream.aggregate_by_window(preds, W, S, mode, delta), ref, atol=1e-12)
            ks = [0, n // 2, n - 1]
            np.testing.assert_allclose(stream.aggregate_by_window(preds, W, S, mode, delta, ks), ref[ks], atol=1e-12)


def test_aggregate_by_window_full_overlap_count():
    # with delta = W - S a sample emitted once the stream holds W samples is
    # the mean of exactly W / S windows: a prediction equal to the window
    # index j gives the mean of k - W/S + 1 .. k
    W, S, n = 512, 64, 30
    preds = np.repeat(np.arange(n, dtype=np.float64)[:, None], W, 1)
    agg = stream.aggregate_by_window(preds, W, S, stream.AVERAGE, W - S)
    for k in range(W // S, n):
        np.testing.assert_allclose(agg[k], np.full(S, k - (W // S - 1) / 2.0), atol=1e-12)


# ----------------------------------------------------------------------------
# Welch ASD (cleaning-quality measure of Methods, "Aggregation latency")
# ----------------------------------------------------------------------------

def test_welch_matches_scipy():
    from scipy.signal import welch
    x = rng.standard_normal(4096 * 12)
    f, p = spectral.welch_psd(x, 4096.0)
    f2, p2 = welch(x, fs=4096.0, window="hann", nperseg=8192, noverlap=4096)
    np.testing.assert_allclose(f, f2)
    np.testing.assert_allclose(p, p2, rtol=1e-10)


def test_welch_pure_tone_peak_closed_form():
    # A sin(2 pi f0 t) with f0 on a bin: the windowed DFT at f0 is A/2 sum w,
    # so the one-sided density there is A^2 (sum w)^2 / (2 fs sum w^2); for
    # the periodic Hann window sum w = N/2 and sum w^2 = 3N/8, giving A^2 N / (3 fs)
    fs, N, A = 4096.0, 8192, 0.7
    f0 = 60.0  # 120 bins at df = 0.5 Hz
    t = np.arange(10 * N) / fs
    f, p = spectral.welch_psd(A * np.sin(2 * np.pi * f0 * t + 0.3), fs)
    j = int(round(f0 / (fs / N)))
    assert abs(p[j] / (A * A * N / (3 * fs)) - 1) < 1e-6
    # the two neighbouring bins hold a quarter of the amplitude each, and the
    # density integrates to the tone's power A^2 / 2
    np.testing.assert_allclose(p[j - 1:j + 2:2], p[j] / 4, rtol=1e-6)
    assert abs(p.sum() * (fs / N) - A * A / 2) < 1e-6


def test_welch_white_noise_flat_and_scaling():
    # white noise of variance s2 has the flat one-sided density 2 s2 / fs;
    # the ASD of a scaled series is the scaled ASD, so ratios of scaled series
    # are exact
    fs, s = 4096.0, 1.7
    x = rng.standard_normal(4096 * 64) * s
    f, a = spectral.welch_asd(x, fs)
    inner = (f > 10) & (f < 2000)
    assert abs(np.mean(a[inner] ** 2) / (2 * s * s / fs) - 1) < 0.01
    _, r = spectral.asd_ratio(0.25 * x, x, fs)
    np.testing.assert_allclose(r, 0.25, rtol=1e-12)


def test_frac_bins_off():
    f = np.arange(0, 100, 0.5)
    off = np.ones_like(f)
    on = np.ones_like(f)
    band = (f >= 50) & (f <= 70)
    idx = np.flatnonzero(band)
    on[idx[:8]] = 1.2   # 8 bins 20% off
    on[idx[8:12]] = 1.05  # within 10%
    on[f < 50] = 3.0    # outside the band: ignored
    assert spectral.frac_bins_off(on, off, f) == pytest.approx(8 / band.sum())


def test_streamed_equals_full_pass_for_local_model():
    # For a conv model of half-width 3, a window's prediction away from its
    # edges equals the same conv over the whole stream; LATEST(delta >= 3)
    # therefore reproduces the full-stream pass exactly.
    W, S, n = 512, 64, 24
    C = 4
    x = rng.standard_normal((C, n * S))
    w = rng.standard_normal((1, C, 7))
    fwd = lambda wins: Lyr.conv1d(wins, w, np.zeros(1), 1, 3, 3)[:, 0]
    full = Lyr.conv1d(x[None], w, np.zeros(1), 1, 3, 3)[0, 0]
    zero = np.zeros(n * S)
    for delta in (3, 64, 200):
        _, cl = stream.run_deepclean_stream(fwd, x, zero, W, S, n, stream.LATEST, delta)
        for k in range(W // S, n):
            t = stream.emit_times(k, S, delta)
            np.testing.assert_allclose(-cl[k], full[t], atol=1e-12)


def test_pipeline_timing_with_delta_filters():
    # With a model that predicts zero, cleaned = strain; with a decimator that
    # is a unit impulse at its centre tap and a whitening filter that is a unit
    # impulse at its centre tap, w[n] = d[n] = c[2n] = strain[2n].  The BBHnet
    # input of snapshot k is then strain at even times ending at 2 n_end_k, and
    # its logit must equal BBHnet applied to that window directly.
    from oracle import pipeline
    W, S, n, Lb = 256, 64, 12, 128
    layers = synth.bbhnet_layers()
    params, head = synth.bbhnet_params(4)
    strain = [rng.standard_normal(n * S) for _ in range(2)]
    wit = [np.zeros((3, n * S)) for _ in range(2)]
    zero = lambda wins: np.zeros((wins.shape[0], wins.shape[-1]))
    f_dec = np.zeros(127); f_dec[63] = 1.0
    h = np.zeros(33); h[16] = 1.0
    delta = 40
    cl, logits = pipeline.run_pipeline(wit, strain, W, S, n, stream.AVERAGE, delta, [zero, zero], f_dec, h,
                                       params, head, layers, Lb=Lb)
    for k in range(n):
        t = stream.emit_times(k, S, delta)
        ok = t >= 0
        np.testing.assert_allclose(cl[0, k][ok], strain[0][t[ok]], atol=1e-12)
        me = pipeline.m_end(k, S, delta)
        ne = me - 16
        win = np.zeros((1, 2, Lb))
        for i, nn in enumerate(range(ne - Lb, ne)):
            if nn >= 0:
                win[0, :, i] = [strain[0][2 * nn], strain[1][2 * nn]]
        assert abs(logits[k] - nets.bbhnet_forward(win, params, head, layers)[0]) < 1e-9


def test_pipeline_post_processing_timing():
    # A post-processing FIR that is a unit impulse at its centre tap leaves the
    # cleaned series unchanged but delays it by c samples; with c = S every
    # output of snapshot k (cleaned samples and the BBHnet input window, hence
    # the logit) is the plain pipeline's output of snapshot k - 1.  A one-tap
    # FIR [1] changes nothing.
    from oracle import pipeline
    W, S, n, Lb, delta = 256, 64, 10, 128, 40
    layers = synth.bbhnet_layers()
    params, head = synth.bbhnet_params(5)
    r = np.random.default_rng(12)
    wit = [r.standard_normal((21, n * S)) for _ in range(2)]
    strain = [r.standard_normal(n * S) for _ in range(2)]
    dc = synth.deepclean_params(13)
    fwd = lambda wins: nets.deepclean_forward(wins, dc, synth.DEEPCLEAN_LAYERS) * 0.05
    f_dec = r.standard_normal(127) * 0.1
    h = r.standard_normal(33) * 0.2
    args = (wit, strain, W, S, n, stream.AVERAGE, delta, [fwd, fwd], f_dec, h, params, head, layers)
    cl0, lg0 = pipeline.run_pipeline(*args, Lb=Lb)
    # emitted times before the stream start: the plain pipeline gives minus the
    # prediction there, the post-processed one reads the prediction at
    # negative times as zero (there is no data), so both give their own values
    t = np.stack([stream.emit_times(k, S, delta) for k in range(n)])
    cl1, lg1 = pipeline.run_pipeline(*args, Lb=Lb, post=np.array([1.0]))
    ok = np.broadcast_to(t >= 0, cl0.shape)
    np.testing.assert_array_equal(cl1[ok], cl0[ok])
    assert np.abs(cl1[~ok]).max() == 0.0
    np.testing.assert_array_equal(lg1, lg0)
    imp = np.zeros(2 * S + 1)
    imp[S] = 1.0
    cl2, lg2 = pipeline.run_pipeline(*args, Lb=Lb, post=imp)
    ok1 = np.broadcast_to(t[:-1] >= 0, cl0[:, :-1].shape)
    np.testing.assert_allclose(cl2[:, 1:][ok1], cl0[:, :-1][ok1], atol=1e-12)
    assert np.abs(cl2[:, 1:][~ok1]).max() == 0.0 and np.abs(cl2[:, 0]).max() == 0.0
    np.testing.assert_allclose(lg2[1:], lg0[:-1], atol=1e-9)


# ----------------------------------------------------------------------------
# Gradient: central finite differences and PyTorch autograd in float64
# ----------------------------------------------------------------------------

def _small_training_case():
    params = synth.deepclean_params(5)
    L = 512
    x = synth.witness_channels(6, 21, L * 2)[None, :, :L]
    s = rng.standard_normal((1, L)) * 0.3
    f, psd = synth.psd_grid(4096.0, 2048)
    g = fir.band_loss_fir(psd, 4096.0, 2048, 129)
    return params, x, s, g


def test_gradient_matches_finite_differences():
    params, x, s, g = _small_training_case()
    layers = synth.DEEPCLEAN_LAYERS
    loss, _, grads = grad.deepclean_loss_and_grad(x, s, params, layers, g)
    assert abs(loss - grad.deepclean_loss(x, s, params, layers, g)) < 1e-12 * abs(loss)
    r = np.random.default_rng(7)
    for li in range(len(layers)):
        for key in ("w", "b", "gamma", "beta"):
            if key not in params[li]:
                continue
            P = params[li][key]
            for _ in range(2):
                idx = tuple(r.integers(0, d) for d in P.shape)
                eps = 1e-5
                pp = [dict((k, np.array(v, np.float64)) for k, v in q.items()) for q in params]
                pm = [dict((k, np.array(v, np.float64)) for k, v in q.items()) for q in params]
                pp[li][key][idx] += eps
                pm[li][key][idx] -= eps
                fd = (grad.deepclean_loss(x, s, pp, layers, g) - grad.deepclean_loss(x, s, pm, layers, g)) / (2 * eps)
                an = grads[li][key][idx]
                assert abs(fd - an) <= 1e-4 * max(abs(fd), 1e-3 * np.abs(grads[li][key]).max()), (li, key, idx, fd, an)


def test_gradient_matches_torch_autograd():
    params, x, s, g = _small_training_case()
    layers = synth.DEEPCLEAN_LAYERS
    loss, _, grads = grad.deepclean_loss_and_grad(x, s, params, layers, g)
    mods = [torch_layer(sp, p) for sp, p in zip(layers, params)]
    model = torch.nn.Sequential(*mods)
    y = model(t64(x))[:, 0]
    r = F.conv1d((t64(s) - y)[:, None], t64(g)[None, None])
    tl = (r ** 2).mean()
    tl.backward()
    assert abs(tl.item() - loss) < 1e-12 * abs(loss)
    for li, m in enumerate(mods):
        conv = [c for c in m if isinstance(c, (torch.nn.Conv1d, torch.nn.ConvTranspose1d))][0]
        np.testing.assert_allclose(grads[li]["w"], conv.weight.grad.numpy(), rtol=1e-9, atol=1e-14)
        np.testing.assert_allclose(grads[li]["b"], conv.bias.grad.numpy(), rtol=1e-9, atol=1e-14)
        bns = [c for c in m if isinstance(c, torch.nn.BatchNorm1d)]
        if bns:
            np.testing.assert_allclose(grads[li]["gamma"], bns[0].weight.grad.numpy(), rtol=1e-9, atol=1e-14)
            np.testing.assert_allclose(grads[li]["beta"], bns[0].bias.grad.numpy(), rtol=1e-9, atol=1e-14)


# ----------------------------------------------------------------------------
# Narrow casts against PyTorch's own rounding
# ----------------------------------------------------------------------------

def test_quant_bf16_matches_torch():
    from oracle import quant
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        [0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5]])
    x32 = x.astype(np.float32)
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(quant.to_bf16(x32), ref)


def test_quant_e4m3_matches_torch_in_range():
    from oracle import quant
    x = np.concatenate([rng.uniform(-440, 440, 20000), rng.standard_normal(5000) * 1e-2,
                        [0.0, 0.5 * 2 ** -9, 1.5 * 2 ** -9, 1.0 + 2 ** -4, 1.0 + 3 * 2 ** -4]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(quant.to_e4m3(x.astype(np.float32)), ref)
    assert quant.to_e4m3(1e4) == 448.0 and quant.to_e4m3(-1e4) == -448.0


# ----------------------------------------------------------------------------
# The oracle's process pool: distribution only
# ----------------------------------------------------------------------------

def test_pool_returns_each_windows_serial_forward_in_order():
    """Worker processes (spawned, one BLAS thread each) return, in the order
    asked, what the serial oracle gives for each snapshot window, including a
    window that starts before t = 0 (zero fill) and repeated indices."""
    from oracle import pool
    W, S = 256, 64
    x = rng.standard_normal((21, W + 7 * S))
    params = synth.deepclean_params(3)
    ks = [5, 0, 7, 2, 5, 3]
    got = pool.deepclean_stream_windows(x, W, S, ks, params, synth.DEEPCLEAN_LAYERS, workers=2, chunk=1)
    ref = np.stack([nets.deepclean_forward(stream.window(x, W, S, k)[None], params, synth.DEEPCLEAN_LAYERS)[0]
                    for k in ks])
    assert got.shape == (len(ks), W)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
