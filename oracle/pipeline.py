"""End-to-end streaming pipeline per stream in float64 (test infrastructure).

The paper's end-to-end ensemble cleans the strain of two detectors with
DeepClean, combines and post-processes it and scores it with BBHnet (Methods,
offline deployment); online, each request brings S new samples and returns
the newest cleaned samples (Methods, "Streaming IaaS", "Data aggregation").
Readings of the unspecified timing, sample for sample:

* cleaned c[tau] (4096 Hz) for tau >= 0 is the aggregated, subtracted strain of
  ``oracle.stream`` (times tau < 0 count as 0); after snapshot k (0-based) it
  is known up to c_end_k = (k+1) S - delta (exclusive).
* decimated d[m] = sum_{j=0}^{126} f[j] c[2m + j - 63] (2048 Hz), m >= 0;
  known after snapshot k for m < m_end_k = floor((c_end_k - 64) / 2) + 1.
* whitened w[n] = sum_{j=0}^{2048} h[j] d[n + j - 1024], n >= 0 (d[m < 0] = 0);
  known for n < n_end_k = m_end_k - 1024.
* the BBHnet input at snapshot k is w[n_end_k - Lb, n_end_k) of each detector
  (w at negative n = 0), Lb = 2048 (1 s at 2048 Hz); the score is its logit.
* with post-processing (the online pipeline's band-pass of the noise estimate
  before subtraction, ``oracle.stream.clean_post``), the FIR of K taps needs
  the aggregated prediction c = (K - 1) / 2 samples past an output time, so the
  cleaned series after snapshot k is known up to (k+1) S - delta - c, and every
  later stage follows it: c_end_k, m_end_k and n_end_k are those of delta + c.
"""
from __future__ import annotations

import numpy as np

from . import fir, nets, stream


def _floordiv(a, b):
    return -((-a) // b) if a < 0 else a // b


def m_end(k, S, delta):
    c_end = (k + 1) * S - delta
    return max(0, (c_end - 64) // 2 + 1) if c_end >= 64 else 0


def run_pipeline(witness, strain, W, S, n_snap, mode, delta, dc_fwd, f_dec, h_wht, bbh_params, bbh_head,
                 bbh_layers, Lb=2048, post=None):
    """One stream of n_det detectors.

    witness: list (per detector) of (C, n_snap*S); strain: list of (n_snap*S,).
    dc_fwd: per-detector callables mapping (B, C, W) windows to (B, W).
    post: optional post-processing FIR taps (odd length) of the aggregated
    prediction.
    Returns (cleaned (n_det, n_snap, S), logits (n_snap,)); with post, row k of
    cleaned holds the times emitted by snapshot k shifted by c.
    """
    n_det = len(witness)
    c_post = (len(post) - 1) // 2 if post is not None else 0
    cleaned = []
    cstreams = []
    for d in range(n_det):
        _, cl = stream.run_deepclean_stream(dc_fwd[d], witness[d], strain[d], W, S, n_snap, mode, delta, post=post)
        cleaned.append(cl)
        # continuous cleaned series c[tau], tau >= 0 (emitted times kS - delta + i)
        total = n_snap * S
        c = np.zeros(total)
        for k in range(n_snap):
            t = stream.emit_times(k, S, delta) - c_post
            ok = (t >= 0) & (t < total)
            c[t[ok]] = cl[k][ok]
        cstreams.append(c)
    K = len(f_dec)
    Kw = len(h_wht)
    logits = np.zeros(n_snap)
    for k in range(n_snap):
        me = m_end(k, S, delta + c_post)
        ne = me - (Kw - 1) // 2
        wins = np.zeros((1, n_det, Lb))
        for d in range(n_det):
            c = cstreams[d]
            cpad = np.concatenate([np.zeros(64), c, np.zeros(4096)])  # c[tau] at cpad[tau + 64]
            # d[m] for m < me
            dm = np.zeros(max(me, 0))
            for m in range(me):
                lo = 2 * m - (K - 1) // 2
                dm[m] = cpad[lo + 64:lo + 64 + K] @ f_dec
            for i, n in enumerate(range(ne - Lb, ne)):
                if n < 0:
                    continue
                acc = 0.0
                lo = n - (Kw - 1) // 2
                seg = np.zeros(Kw)
                a = max(lo, 0)
                b = min(lo + Kw, me)
                if b > a:
                    seg[a - lo:b - lo] = dm[a:b]
                acc = seg @ h_wht
                wins[0, d, i] = acc
        logits[k] = nets.bbhnet_forward(wins, bbh_params, bbh_head, bbh_layers)[0]
    return np.stack(cleaned), logits
