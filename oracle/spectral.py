"""Welch amplitude spectral density and the aggregation-latency metrics in
float64 (test infrastructure; see the package header).

Methods, "Aggregation latency": cleaning quality is judged by the ratio of
the amplitude spectral density (ASD) of the cleaned strain to that of the
raw strain, and an online scheme by the fraction of frequency bins in
[50, 70] Hz where its ratio is more than 10% away from the offline one.  The
paper does not give the spectral estimator; the reading here (also the one
for the benchmark spec's tolerance on the cleaned-strain ASD) is Welch's method:

* segments of nperseg = seg_seconds * fs samples, advanced by
  nperseg * (1 - overlap) (Hann, 2 s, 50% overlap by default);
* each segment minus its own mean, times the periodic Hann window
  w[n] = 0.5 - 0.5 cos(2 pi n / nperseg);
* one-sided periodogram P_j = 2 |X_j|^2 / (fs sum_n w[n]^2), with the DC and
  Nyquist bins not doubled, X = the DFT of the windowed segment;
* the PSD is the mean of the segments' periodograms, the ASD its square
  root, on the grid f_j = j fs / nperseg.

The DFT is numpy's rfft (a library primitive).
"""
from __future__ import annotations

import numpy as np


def hann_periodic(n):
    return 0.5 - 0.5 * np.cos(2.0 * np.pi * np.arange(n) / n)


def welch_psd(x, fs, seg_seconds=2.0, overlap=0.5):
    """(f, one-sided PSD) of the 1-D series x by Welch's method (see header)."""
    x = np.asarray(x, np.float64)
    nper = int(round(seg_seconds * fs))
    step = int(round(nper * (1.0 - overlap)))
    assert 0 < step <= nper <= x.size
    w = hann_periodic(nper)
    scale = fs * np.sum(w * w)
    starts = range(0, x.size - nper + 1, step)
    acc = np.zeros(nper // 2 + 1)
    for s0 in starts:
        seg = x[s0:s0 + nper]
        X = np.fft.rfft((seg - seg.mean()) * w)
        p = np.abs(X) ** 2 / scale
        p[1:] *= 2.0
        if nper % 2 == 0:
            p[-1] /= 2.0  # the Nyquist bin has no negative-frequency twin
        acc += p
    return np.arange(nper // 2 + 1) * (fs / nper), acc / len(starts)


def welch_asd(x, fs, seg_seconds=2.0, overlap=0.5):
    """(f, ASD) = (f, sqrt(Welch PSD))."""
    f, p = welch_psd(x, fs, seg_seconds, overlap)
    return f, np.sqrt(p)


def asd_ratio(cleaned, raw, fs, seg_seconds=2.0, overlap=0.5):
    """(f, ASD(cleaned) / ASD(raw)): the paper's cleaning-quality curve."""
    f, a = welch_asd(cleaned, fs, seg_seconds, overlap)
    _, b = welch_asd(raw, fs, seg_seconds, overlap)
    return f, a / b


def frac_bins_off(ratio_online, ratio_offline, f, f1=50.0, f2=70.0, rel=0.1):
    """Fraction of bins with f1 <= f <= f2 in which the online ratio differs
    from the offline one by more than `rel` of the offline value."""
    band = (f >= f1) & (f <= f2)
    return float(np.mean(np.abs(np.asarray(ratio_online)[band] / np.asarray(ratio_offline)[band] - 1.0) > rel))
