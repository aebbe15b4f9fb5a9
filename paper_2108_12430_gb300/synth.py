"""Seeded synthetic inputs shaped like the detector data of arXiv 2108.12430.

This module produces *inputs only*: witness channels, coloured strain,
chirp injections, the analytic noise PSD and randomly initialised network
parameters.  It holds none of the method's arithmetic (no convolution layer,
no filter design, no aggregation); the FP64 oracle and the CUDA library both
consume the arrays it returns, so both sides see bit-identical inputs.

The paper's own data (O2/O3 frame files, trained DeepClean / BBHnet weights)
is not available; these generators stand in for it with the paper's shapes:
21 witness channels (Sec. 1), f_s = 4096 Hz (Methods, offline deployment),
8 s windows (Methods, aggregation latency) and two detectors (Methods,
end-to-end ensemble).

Every function takes an explicit ``seed`` (numpy PCG64) and is deterministic.
"""
from __future__ import annotations

import math

import numpy as np

# Strain is expressed in units of 1e-21 so that samples are O(1); the PSD is
# scaled by the square of that factor accordingly.
STRAIN_SCALE = 1.0e21
F_LOW_CLAMP = 15.0  # Hz: the analytic PSD is held constant below this


def aligo_psd(f):
    """One-sided analytic aLIGO-like noise PSD in (scaled strain)^2 / Hz.

    Zero-detuned high-power design fit of Ajith (2011),
    S(f) = S0 [x^-4.14 - 5 x^-2 + 111 (1 - x^2 + x^4/2) / (1 + x^2/2)],
    x = f / 215 Hz, S0 = 1e-49 / Hz, held at S(15 Hz) below 15 Hz so that it
    is finite down to DC.  Multiplied by STRAIN_SCALE**2.
    """
    f = np.asarray(f, dtype=np.float64)
    fc = np.maximum(f, F_LOW_CLAMP)
    x = fc / 215.0
    s = x ** -4.14 - 5.0 * x ** -2 + 111.0 * (1.0 - x ** 2 + 0.5 * x ** 4) / (1.0 + 0.5 * x ** 2)
    return 1.0e-49 * STRAIN_SCALE ** 2 * s


def psd_grid(fs: float, nfft: int):
    """(frequencies, PSD) on the rfft grid f_j = j fs / nfft, j = 0..nfft/2."""
    f = np.arange(nfft // 2 + 1, dtype=np.float64) * (fs / nfft)
    return f, aligo_psd(f)


def colored_noise(seed: int, n: int, fs: float, n_ch: int = 1):
    """Gaussian noise with one-sided PSD aligo_psd, shape (n_ch, n), float64.

    White N(0,1) samples (one-sided PSD 2/fs) are coloured in the frequency
    domain by sqrt(S(f) fs / 2).  The result is circular (periodic in n).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((n_ch, n))
    f = np.fft.rfftfreq(n, 1.0 / fs)
    amp = np.sqrt(aligo_psd(f) * fs / 2.0)
    return np.fft.irfft(np.fft.rfft(w, axis=-1) * amp, n=n, axis=-1)


def _band_rms(x, fs, f1, f2):
    """RMS of x after a brick-wall frequency-domain band limit to [f1, f2]."""
    n = x.shape[-1]
    X = np.fft.rfft(x, axis=-1)
    f = np.fft.rfftfreq(n, 1.0 / fs)
    X[..., (f < f1) | (f > f2)] = 0.0
    return float(np.sqrt(np.mean(np.fft.irfft(X, n=n, axis=-1) ** 2)))


def witness_channels(seed: int, n_ch: int, n: int, fs: float = 4096.0,
                     n_line: int = 3, burn_in: int = 4096):
    """Witness channels, shape (n_ch, n), float64, each with unit variance.

    Every channel is seeded Gaussian noise through a 4th-order Butterworth
    low-pass at 256 Hz (zero initial state, ``burn_in`` samples discarded).
    The first ``n_line`` channels also carry a 60 Hz mains line with a
    random-walk phase plus 58-62 Hz band noise: these are the channels that
    couple into strain.
    """
    from scipy import signal

    rng = np.random.Generator(np.random.PCG64(seed))
    b, a = signal.butter(4, 256.0 / (fs / 2.0))
    raw = rng.standard_normal((n_ch, n + burn_in))
    x = signal.lfilter(b, a, raw, axis=-1)[:, burn_in:]
    t = np.arange(n) / fs
    for c in range(min(n_line, n_ch)):
        phase = np.cumsum(rng.standard_normal(n)) * 2.0e-3 + rng.uniform(0, 2 * np.pi)
        line = (1.0 + 0.5 * c) * np.sin(2 * np.pi * 60.0 * t + phase)
        bn = rng.standard_normal(n)
        B = np.fft.rfft(bn)
        f = np.fft.rfftfreq(n, 1.0 / fs)
        B[(f < 58.0) | (f > 62.0)] = 0.0
        band = np.fft.irfft(B, n=n)
        band *= 0.5 / max(np.std(band), 1e-30)
        x[c] = x[c] / np.std(x[c]) * 0.3 + line + band
    x -= x.mean(axis=-1, keepdims=True)
    x /= x.std(axis=-1, keepdims=True)
    return x


def coupled_strain(seed: int, witness, fs: float = 4096.0, snr: float = 20.0,
                   n_couple: int = 3, ntap: int = 33):
    """Strain = coloured aLIGO-like noise + linear coupling of witnesses.

    The coupling is sum_k a_k (c_k * w_k) over the first ``n_couple``
    witnesses with seeded ``ntap``-tap FIRs c_k (full convolution, truncated
    causally).  Its overall gain is set so that the RMS of the coupled part
    over the RMS of the background, both limited to 55-65 Hz by a
    frequency-domain brick wall, equals ``snr``.  Returns float64 (n,).
    """
    n = witness.shape[-1]
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    bg = colored_noise(seed, n, fs)[0]
    coup = np.zeros(n)
    for k in range(n_couple):
        c = rng.standard_normal(ntap) * np.hanning(ntap + 2)[1:-1]
        coup += rng.uniform(0.5, 1.5) * np.convolve(witness[k], c)[:n]
    r_c = _band_rms(coup, fs, 55.0, 65.0)
    r_b = _band_rms(bg, fs, 55.0, 65.0)
    return bg + coup * (snr * r_b / max(r_c, 1e-30))


def chirp(seed: int, n: int, fs: float = 2048.0):
    """A frequency-sweeping sinusoid with a Gaussian envelope, shape (n,).

    f(t) = 30 Hz ((t_c - t) / (t_c - t0))^(-3/8), capped at 300 Hz, with t_c
    uniform in the central half of the segment; envelope width U(0.1, 0.3) s.
    Unit peak amplitude; SNR scaling is done by ``injected_strain``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.arange(n) / fs
    T = n / fs
    tc = rng.uniform(0.25 * T, 0.75 * T)
    tau0 = 0.5
    tau = np.maximum(tc - t, 1e-4)
    f = np.minimum(30.0 * (tau / tau0) ** (-3.0 / 8.0), 300.0)
    phase = 2 * np.pi * np.cumsum(f) / fs + rng.uniform(0, 2 * np.pi)
    width = rng.uniform(0.1, 0.3)
    env = np.exp(-0.5 * ((t - tc) / width) ** 2)
    return env * np.sin(phase)


def _whitened_norm(x, fs):
    """||x_w|| with x whitened in the frequency domain by 1/sqrt(S fs / 2)."""
    n = x.shape[-1]
    f = np.fft.rfftfreq(n, 1.0 / fs)
    X = np.fft.rfft(x, axis=-1) / np.sqrt(aligo_psd(f) * fs / 2.0)
    return float(np.sqrt(np.sum(np.fft.irfft(X, n=n, axis=-1) ** 2)))


def injected_strain(seed: int, batch: int, n: int, fs: float = 2048.0,
                    frac: float = 0.5, snr_range=(8.0, 20.0)):
    """Two-detector coloured strain with chirps in a fraction of windows.

    Returns (x float64 (batch, 2, n), label int (batch,), snr float (batch,)).
    An injected window carries the same chirp in both detectors with a time
    shift of at most 10 ms and amplitude factors U(0.5, 1), scaled so that
    the network SNR sqrt(sum_det ||h_w||^2) of the frequency-domain-whitened
    injection equals a U(snr_range) draw.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x = colored_noise(seed + 1, n, fs, n_ch=2 * batch).reshape(batch, 2, n)
    label = (rng.uniform(size=batch) < frac).astype(np.int64)
    snr = np.zeros(batch)
    for b in range(batch):
        if not label[b]:
            continue
        h = chirp(int(rng.integers(1 << 30)), n, fs)
        shift = int(round(rng.uniform(-0.01, 0.01) * fs))
        h2 = np.stack([h * rng.uniform(0.5, 1.0), np.roll(h, shift) * rng.uniform(0.5, 1.0)])
        norm = math.sqrt(sum(_whitened_norm(h2[d], fs) ** 2 for d in range(2)))
        snr[b] = rng.uniform(*snr_range)
        x[b] += h2 * (snr[b] / max(norm, 1e-30))
    return x, label, snr


# ----------------------------------------------------------------------------
# Network parameters (random initialisation; the paper's weights are not
# public).  Layer specifications are plain data: (kind, c_in, c_out, k,
# stride, pad_left, pad_right, out_pad, bn, act).
# ----------------------------------------------------------------------------

DEEPCLEAN_LAYERS = (
    ("conv", 21, 8, 7, 1, 3, 3, 0, True, "tanh"),
    ("conv", 8, 16, 7, 2, 3, 3, 0, True, "tanh"),
    ("conv", 16, 32, 7, 2, 3, 3, 0, True, "tanh"),
    ("conv", 32, 64, 7, 2, 3, 3, 0, True, "tanh"),
    ("convT", 64, 32, 7, 2, 3, 3, 1, True, "tanh"),
    ("convT", 32, 16, 7, 2, 3, 3, 1, True, "tanh"),
    ("convT", 16, 8, 7, 2, 3, 3, 1, True, "tanh"),
    ("conv", 8, 1, 7, 1, 3, 3, 0, False, "none"),
)


def bbhnet_layers(c_in: int = 2):
    """BBHnet-shaped layer list: stem, 4 residual blocks, then GAP + linear.

    Each block is (conv1 k7 s2, conv2 k7 s1, shortcut k1 s2); the order in
    the flat parameter vector follows this list.
    """
    L = [("conv", c_in, 32, 16, 1, 7, 8, 0, True, "relu")]
    cin = 32
    for cout in (32, 64, 128, 256):
        L.append(("conv", cin, cout, 7, 2, 3, 3, 0, True, "relu"))
        L.append(("conv", cout, cout, 7, 1, 3, 3, 0, True, "none"))
        L.append(("conv", cin, cout, 1, 2, 0, 0, 0, True, "none"))
        cin = cout
    return tuple(L)


def _layer_params(rng, spec):
    kind, cin, cout, k, s, pl, pr, op, bn, act = spec
    if kind == "conv":
        shape, fan_in = (cout, cin, k), cin * k
    else:
        shape, fan_in = (cin, cout, k), cin * k / s
    p = {
        "w": (rng.standard_normal(shape) * math.sqrt(2.0 / fan_in)).astype(np.float32),
        "b": (rng.standard_normal(cout) * 0.05).astype(np.float32),
    }
    if bn:
        p["gamma"] = rng.uniform(0.5, 1.5, cout).astype(np.float32)
        p["beta"] = (rng.standard_normal(cout) * 0.1).astype(np.float32)
        p["mean"] = (rng.standard_normal(cout) * 0.1).astype(np.float32)
        p["var"] = rng.uniform(0.5, 2.0, cout).astype(np.float32)
    return p


def deepclean_params(seed: int):
    """He-initialised DeepClean parameters: list of per-layer dicts (FP32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [_layer_params(rng, s) for s in DEEPCLEAN_LAYERS]


def bbhnet_params(seed: int, c_in: int = 2):
    """He-initialised BBHnet parameters: (list of conv-layer dicts, head dict)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    layers = [_layer_params(rng, s) for s in bbhnet_layers(c_in)]
    head = {
        "w": (rng.standard_normal(256) * math.sqrt(1.0 / 256)).astype(np.float32),
        "b": np.float32(rng.standard_normal() * 0.05).reshape(1),
    }
    return layers, head


PARAM_ORDER = ("w", "b", "gamma", "beta", "mean", "var")


def flatten_params(layers, head=None):
    """Flat FP32 vector in the library's canonical order.

    For each layer in order: w (PyTorch layout: conv (C_out, C_in, K),
    transposed conv (C_in, C_out, K)), b, then gamma, beta, running mean,
    running var when the layer has BatchNorm; then the head's w, b.
    """
    parts = []
    for p in layers:
        for key in PARAM_ORDER:
            if key in p:
                parts.append(np.asarray(p[key], np.float32).ravel())
    if head is not None:
        parts.append(np.asarray(head["w"], np.float32).ravel())
        parts.append(np.asarray(head["b"], np.float32).ravel())
    return np.concatenate(parts)
