"""Snapshot windows and output aggregation in float64 (test infrastructure).

Methods, "Streaming IaaS": a stream sampled at f_s is processed in fixed
length snapshots; each request carries floor(f_s / r) = S strictly new
samples, and the snapshot state moves forward by S, so snapshot k (k = 0, 1,
...) is the window of the last W samples ending at time (k+1) S:

    window_k = x[(k+1) S - W, (k+1) S)     (zero before the stream starts).

Methods, "Data aggregation" and "Aggregation latency": a model whose output
is itself a W-sample series returns, per snapshot, S samples of cleaned
data.  With aggregation latency delta (in samples) the samples emitted at
snapshot k are the times

    [k S - delta, k S + S - delta).

* LATEST(delta): the newest window's prediction on those times, i.e. the
  slice pred_k[W - S - delta, W - delta).  delta = 0 is the paper's
  "fully-online" / causal scheme (keep the most recent S samples).
* AVERAGE(delta): the mean, over every window j <= k already pushed (j >= 0)
  that covers a time, of that window's prediction there -- the overlapping
  predictions the paper says could be aggregated.  delta = W - S averages
  each sample over all W / S windows that cover it (full overlap-add).

Cleaned strain is strain minus the aggregated prediction (Sec. 1, DeepClean
predicts and subtracts noise); strain before time 0 is taken as zero.
"""
from __future__ import annotations

import numpy as np

LATEST = 0
AVERAGE = 1


def window(x_total, W, S, k):
    """Snapshot window k of a (C, N) stream -> (C, W), zero-filled before t=0."""
    x_total = np.asarray(x_total, np.float64)
    C = x_total.shape[0]
    end = (k + 1) * S
    out = np.zeros((C, W))
    lo = end - W
    src_lo = max(lo, 0)
    out[:, src_lo - lo:] = x_total[:, src_lo:end]
    return out


def emit_times(k, S, delta):
    return np.arange(k * S - delta, k * S + S - delta)


def aggregate(preds, W, S, mode, delta):
    """Aggregated predictions per snapshot: preds (n, W) -> (n, S)."""
    preds = np.asarray(preds, np.float64)
    n = preds.shape[0]
    assert 0 <= delta <= W - S
    out = np.zeros((n, S))
    for k in range(n):
        if mode == LATEST:
            out[k] = preds[k, W - S - delta:W - delta]
            continue
        for i, tau in enumerate(emit_times(k, S, delta)):
            vals = []
            for j in range(0, k + 1):  # windows already pushed, in order
                start = (j + 1) * S - W
                if start <= tau < start + W:
                    vals.append(preds[j, tau - start])
            out[k, i] = np.mean(vals)
    return out


def clean(strain_total, agg, S, delta):
    """cleaned = strain - aggregated prediction on the emitted times (n, S)."""
    strain_total = np.asarray(strain_total, np.float64)
    n = agg.shape[0]
    out = np.zeros((n, S))
    for k in range(n):
        t = emit_times(k, S, delta)
        s = np.where(t >= 0, strain_total[np.clip(t, 0, None)], 0.0)
        out[k] = s - agg[k]
    return out


def clean_post(strain_total, agg, S, delta, h):
    """Cleaned strain with the aggregated prediction post-processed by the FIR h
    (K odd taps, c = (K - 1) / 2) before subtraction (Methods, online
    deployment: the noise estimate is post-processed, then subtracted):

        cleaned[t] = strain[t] - sum_k h[k] p[t + k - c],

    p the aggregated prediction on its emitted times (zero before time 0).
    Snapshot k then delivers the times [k S - delta - c, k S + S - delta - c):
    the FIR needs p up to c samples after the output time.  Returns (n, S)."""
    strain_total = np.asarray(strain_total, np.float64)
    h = np.asarray(h, np.float64)
    n = agg.shape[0]
    K = h.shape[0]
    c = (K - 1) // 2
    # p on the times [-delta, n S - delta); times before 0 count as zero
    t_first = -delta
    p = np.asarray(agg, np.float64).reshape(-1).copy()
    p[np.arange(p.size) + t_first < 0] = 0.0
    out = np.zeros((n, S))
    j = np.arange(K)
    for k in range(n):
        for i, t in enumerate(emit_times(k, S, delta) - c):
            u = t + j - c  # prediction times, at most the last one emitted
            ok = u >= 0
            q = h[ok] @ p[u[ok] - t_first]
            out[k, i] = (strain_total[t] if t >= 0 else 0.0) - q
    return out


def run_deepclean_stream(forward, witness_total, strain_total, W, S, n_snap,
                         mode, delta, snaps=None, post=None):
    """Push n_snap snapshots; returns (predictions (n, W), cleaned (n, S)).

    ``forward`` maps a (B, C, W) batch of windows to (B, W) predictions.
    ``snaps`` restricts the windows evaluated (others are not needed by
    LATEST); by default every snapshot is evaluated.  ``post``: optional
    post-processing FIR taps (see ``clean_post``).
    """
    ks = range(n_snap) if snaps is None else snaps
    wins = np.stack([window(witness_total, W, S, k) for k in ks])
    preds = np.zeros((n_snap, W))
    preds[list(ks)] = forward(wins)
    agg = aggregate(preds, W, S, mode, delta)
    if post is not None:
        return preds, clean_post(strain_total, agg, S, delta, post)
    return preds, clean(strain_total, agg, S, delta)


def aggregate_by_window(preds, W, S, mode, delta, ks=None):
    """The aggregation of ``aggregate`` written per window instead of per
    sample, for long streams: for each emitted snapshot k (all of them, or
    those in ``ks``) the S emitted times are handled together, and the loop
    runs over the windows j = 0 .. k in order, adding window j's prediction
    wherever its span [(j+1) S - W, (j+1) S) holds an emitted time.  The mean
    is that sum over the number of covering windows.  preds (n, W) holds
    every window's prediction; returns (len(ks), S)."""
    preds = np.asarray(preds, np.float64)
    n = preds.shape[0]
    assert 0 <= delta <= W - S
    ks = list(range(n)) if ks is None else list(ks)
    out = np.zeros((len(ks), S))
    for r, k in enumerate(ks):
        if mode == LATEST:
            out[r] = preds[k, W - S - delta:W - delta]
            continue
        tau = emit_times(k, S, delta)
        total = np.zeros(S)
        count = np.zeros(S)
        # windows ending (at (j+1) S) before the first emitted time k S - delta
        # cover none of it; starting the loop a little earlier than that
        # changes nothing
        for j in range(max(0, k - (W + delta) // S - 1), k + 1):
            start = (j + 1) * S - W
            cover = (tau >= start) & (tau < start + W)
            if not cover.any():
                continue
            total[cover] += preds[j, tau[cover] - start]
            count[cover] += 1
        out[r] = total / count
    return out
