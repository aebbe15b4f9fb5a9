"""FIR design and application in float64 (test infrastructure).

The paper feeds BBHnet with DeepClean-cleaned strain from two detectors
(Methods, offline deployment, end-to-end ensemble) after a "postprocess"
step it does not specify, at a rate it does not state.  Readings taken:

* Whitening: a linear-phase FIR of ``ntaps`` (2049) taps designed from the
  one-sided PSD S sampled on the grid f_j = j fs / nfft (nfft = 8192 at
  fs = 2048 Hz).  Target amplitude A_j = sqrt(2 / (fs S_j)): noise of PSD S
  comes out with PSD 2/fs, i.e. unit variance.  The zero-phase impulse
  response is the real inverse DFT of A (evaluated directly, O(N ntaps)),
  centred on tap (ntaps-1)/2, truncated and multiplied by a Hann window.
  Applied in valid mode: y[n] = sum_k h[k] x[n + k].
* Resampling 4096 -> 2048 Hz: 127-tap Hann-windowed sinc low-pass with
  cut-off 900 Hz and unit DC gain, followed by keeping every second sample.
* Training loss weight: the same zero-phase design with target amplitude
  sqrt(T(f) S(60 Hz) / S(f)), T a Tukey taper equal to 1 on [57, 63] Hz and
  falling to 0 at 55 and 65 Hz (a time-domain form of the inverse-PSD
  weighted 55-65 Hz mean-square error).
* Post-processing of the prediction before subtraction (Methods, online
  deployment: the noise estimate is post-processed, then subtracted): the
  same zero-phase design with target amplitude T(f), a band-pass that keeps
  the band the network was trained on.
"""
from __future__ import annotations

import numpy as np


def hann(n):
    """Hann window with zero end points: 0.5 (1 - cos(2 pi k / (n - 1)))."""
    k = np.arange(n, dtype=np.float64)
    return 0.5 * (1.0 - np.cos(2.0 * np.pi * k / (n - 1)))


def zero_phase_fir(amp, nfft, ntaps):
    """Centred, Hann-windowed truncation of the inverse real DFT of ``amp``.

    amp: real amplitudes on j = 0..nfft/2.  The zero-phase response is
    h0[n] = (1/nfft) [A_0 + A_{nfft/2} (-1)^n + 2 sum_{j=1}^{nfft/2-1} A_j cos(2 pi j n / nfft)]
    for n = -(ntaps-1)/2 .. (ntaps-1)/2, computed as a direct sum.
    """
    amp = np.asarray(amp, np.float64)
    assert amp.shape == (nfft // 2 + 1,) and ntaps % 2 == 1 and ntaps <= nfft
    c = (ntaps - 1) // 2
    n = np.arange(-c, c + 1, dtype=np.float64)
    j = np.arange(1, nfft // 2, dtype=np.float64)
    cosm = np.cos(2.0 * np.pi * np.outer(n, j) / nfft)  # (ntaps, nfft/2 - 1)
    h0 = (amp[0] + amp[-1] * np.cos(np.pi * n) + 2.0 * cosm @ amp[1:-1]) / nfft
    return h0 * hann(ntaps)


def whitening_fir(psd, fs, nfft, ntaps=2049):
    """Whitening filter taps (ntaps,) from a one-sided PSD on the rfft grid."""
    A = np.sqrt(2.0 / (fs * np.asarray(psd, np.float64)))
    return zero_phase_fir(A, nfft, ntaps)


def lowpass_fir(ntaps=127, fc=900.0, fs=4096.0):
    """Hann-windowed sinc low-pass, unit DC gain (anti-alias for decimation)."""
    c = (ntaps - 1) / 2.0
    k = np.arange(ntaps, dtype=np.float64) - c
    h = (2.0 * fc / fs) * np.sinc(2.0 * fc / fs * k) * hann(ntaps)
    return h / h.sum()


def tukey_band(f, f1=55.0, f2=65.0, ramp=2.0):
    """1 on [f1+ramp, f2-ramp], raised-cosine ramps to 0 at f1 and f2."""
    f = np.asarray(f, np.float64)
    T = np.zeros_like(f)
    inner = (f >= f1 + ramp) & (f <= f2 - ramp)
    T[inner] = 1.0
    lo = (f > f1) & (f < f1 + ramp)
    T[lo] = 0.5 * (1.0 - np.cos(np.pi * (f[lo] - f1) / ramp))
    hi = (f > f2 - ramp) & (f < f2)
    T[hi] = 0.5 * (1.0 - np.cos(np.pi * (f2 - f[hi]) / ramp))
    return T


def band_loss_fir(psd, fs, nfft, ntaps=2049, f1=55.0, f2=65.0, f_ref=60.0):
    """Loss-weight filter g with |G(f)|^2 = T(f) S(f_ref) / S(f)."""
    psd = np.asarray(psd, np.float64)
    f = np.arange(nfft // 2 + 1) * (fs / nfft)
    s_ref = np.interp(f_ref, f, psd)
    amp = np.sqrt(tukey_band(f, f1, f2) * s_ref / psd)
    return zero_phase_fir(amp, nfft, ntaps)


def bandpass_fir(fs, nfft, ntaps, f1=55.0, f2=65.0, ramp=2.0):
    """Zero-phase band-pass with target amplitude T(f) (Tukey band)."""
    f = np.arange(nfft // 2 + 1) * (fs / nfft)
    return zero_phase_fir(tukey_band(f, f1, f2, ramp), nfft, ntaps)


def fir_valid(x, h):
    """Valid-mode correlation along the last axis: y[n] = sum_k h[k] x[n+k]."""
    x = np.asarray(x, np.float64)
    h = np.asarray(h, np.float64)
    K = h.shape[0]
    n_out = x.shape[-1] - K + 1
    y = np.zeros(x.shape[:-1] + (n_out,))
    for k in range(K):
        y += h[k] * x[..., k:k + n_out]
    return y


def decimate2(x, h, first):
    """Decimated low-pass: y[m] = sum_k h[k] x[2 (first + m) + k - (K-1)/2].

    Only output indices whose support lies inside x are produced, starting at
    output index ``first`` (an index on the 2048 Hz grid, time 2*first on the
    input grid).
    """
    x = np.asarray(x, np.float64)
    K = h.shape[0]
    c = (K - 1) // 2
    out = []
    m = first
    while 2 * m + c < x.shape[-1]:
        lo = 2 * m - c
        assert lo >= 0
        out.append(x[..., lo:lo + K] @ h)
        m += 1
    return np.stack(out, axis=-1) if out else np.zeros(x.shape[:-1] + (0,))


def freq_response(h, f, fs):
    """|H(f)| = |sum_k h[k] exp(-2 pi i f k / fs)| (closed-form DTFT)."""
    k = np.arange(len(h))
    return np.abs(np.exp(-2j * np.pi * np.outer(np.atleast_1d(f), k) / fs) @ h)
