"""Aggregation-latency study (Methods, "Aggregation latency"; the figure on
DeepClean performance against aggregation latency).

DeepClean is trained with the library's training step (band-limited
PSD-weighted loss, hand-written backward, Adam) on a synthetic recording in
which three witnesses carry a 60 Hz line that couples linearly into the
strain.  A held-out segment is then cleaned

  * offline: the whole segment as one window, so that only its two ends see
    the network's zero padding;
  * online: through a stream (8 s windows, stride S) in the causal scheme
    LATEST(delta), which keeps the S newest samples of every window that lie
    delta samples before the window's end - the aggregation latency delta
    moves the kept samples away from the window edge.

Optionally (post_taps > 0) the prediction is post-processed before it is
subtracted, as in the paper's online pipeline: a zero-phase 55-65 Hz
band-pass (gw_fir_create_bandpass), offline through the library's FIR,
online inside the stream (the outputs arrive (post_taps - 1) / 2 samples
later).

The quantity compared is the paper's: the ratio of the amplitude spectral
density (Welch, Hann, 2 s segments, 50% overlap) of the cleaned data to that
of the uncleaned data, and the fraction of frequency bins in [50, 70] Hz in
which an online ratio differs from the offline ratio by more than 10%.

Everything runs through the public API of the library; numpy/scipy only
compute the spectra.  Device buffers are torch tensors.
"""
import numpy as np

from . import gwstream as G, synth

FS = 4096


def _asd(x):
    from scipy.signal import welch
    f, p = welch(x, fs=FS, window="hann", nperseg=2 * FS, noverlap=FS)
    return f, np.sqrt(p)


def aggregation_latency_study(device=0, seed=11, train_s=192, eval_s=64, steps=1000, lr=1e-3, batch=32,
                              train_len=8192, window_s=8, stride=256, deltas_s=(0.0, 0.5, 0.75),
                              precision=G.GW_FP32, post_taps=0, return_series=False):
    """Runs the study; returns a dict of the training losses, the offline ASD
    ratio near 60 Hz and outside the band, and per aggregation latency the
    fraction of [50, 70] Hz bins off the offline ratio by more than 10%.
    return_series: also the raw, offline-cleaned and online-cleaned series
    over the span the spectra are taken on (key "series")."""
    import torch
    C = 21
    W = window_s * FS
    n_tr, n_ev = train_s * FS, eval_s * FS
    # training part, W of stream history, the evaluation segment, W of look-ahead
    wit = synth.witness_channels(seed, C, n_tr + n_ev + 2 * W)
    strain = synth.coupled_strain(seed, wit)
    mean = wit[:, :n_tr].mean(1).astype(np.float32)
    std = wit[:, :n_tr].std(1).astype(np.float32)
    ctx = G.gw_ctx_create(device, 0)
    out = {"seed": seed, "train_seconds": train_s, "eval_seconds": eval_s, "steps": steps, "lr": lr,
           "window_seconds": window_s, "stride": stride, "post_taps": post_taps}
    c = (post_taps - 1) // 2 if post_taps else 0
    try:
        # ---- training (rows a9, a10) ----
        t = G.gw_trainer_create(ctx, C, batch, train_len, 0, mean, std)
        _, psd = synth.psd_grid(4096.0, 8192)
        g = G.gw_fir_create_band_loss(ctx, psd, 4096.0, 2049)
        ntap = G.gw_fir_ntaps(g)
        wd = torch.from_numpy(wit[:, :n_tr].astype(np.float32)).cuda()
        sd = torch.from_numpy(strain[:n_tr].astype(np.float32)).cuda()
        p = torch.from_numpy(synth.flatten_params(synth.deepclean_params(seed))).cuda()
        m1, m2, dp = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
        x = torch.empty(batch, C, train_len, device="cuda")
        s = torch.empty(batch, train_len, device="cuda")
        y, dy = torch.empty(batch, train_len, device="cuda"), torch.empty(batch, train_len, device="cuda")
        r = torch.empty(batch, train_len - ntap + 1, device="cuda")
        loss = torch.empty(1, device="cuda")
        gen = torch.Generator(device="cuda").manual_seed(seed)
        ar = torch.arange(train_len, device="cuda")
        losses = []
        for it in range(1, steps + 1):
            st = torch.randint(0, n_tr - train_len, (batch,), device="cuda", generator=gen)
            idx = st[:, None] + ar[None, :]
            x.copy_(wd[:, idx].permute(1, 0, 2))
            s.copy_(sd[idx])
            G.gw_trainer_forward(t, p.data_ptr(), x.data_ptr(), batch, y.data_ptr())
            G.gw_band_loss(g, s.data_ptr(), y.data_ptr(), batch, train_len, loss.data_ptr(), r.data_ptr())
            G.gw_band_loss_backward(g, r.data_ptr(), batch, train_len, 0, dy.data_ptr())
            G.gw_trainer_backward(t, dy.data_ptr(), dp.data_ptr())
            G.gw_adam_step(p.data_ptr(), dp.data_ptr(), m1.data_ptr(), m2.data_ptr(), p.numel(), it, lr)
            if it == 1 or it % 100 == 0 or it == steps:
                losses.append((it, float(loss.item())))
        G.gw_trainer_destroy(t)
        G.gw_fir_destroy(g)
        out["loss_first"], out["loss_last"] = losses[0][1], losses[-1][1]
        out["losses"] = losses
        params = p.cpu().numpy()
        m = G.gw_model_create(ctx, G.GW_MODEL_DEEPCLEAN, precision, C, params, mean, std)
        post = G.gw_fir_create_bandpass(ctx, float(FS), 8192, post_taps) if post_taps else None

        # ---- offline: the evaluation segment as one window ----
        e0 = n_tr + W
        xe = torch.from_numpy(np.ascontiguousarray(wit[:, e0:e0 + n_ev]).astype(np.float32)).cuda()
        ye = torch.empty(n_ev, device="cuda")
        G.gw_deepclean_forward(m, xe.data_ptr(), n_ev, 0, 1, n_ev, ye.data_ptr())
        torch.cuda.synchronize()
        raw = strain[e0:e0 + n_ev]
        pred = ye.cpu().numpy().astype(np.float64)
        if post:
            # valid-mode FIR: output i sits at time i + c of the segment
            q = torch.empty(n_ev - post_taps + 1, device="cuda")
            G.gw_whiten(post, ye.data_ptr(), 1, 1, n_ev, q.data_ptr())
            torch.cuda.synchronize()
            pred = np.zeros(n_ev)
            pred[c:n_ev - c] = q.cpu().numpy()
        offline = raw - pred
        # spectra over a common span: the offline segment's own padded ends
        # and the FIR's edges are excluded
        lo, hi = 2 * FS + c, n_ev - 2 * FS - c
        series = {"raw": raw[lo:hi], "offline": offline[lo:hi], "online": {}}
        f, a_raw = _asd(raw[lo:hi])
        _, a_off = _asd(offline[lo:hi])
        rat_off = a_off / a_raw
        band = (f >= 50) & (f <= 70)
        line = (f >= 59) & (f <= 61)
        out["offline_ratio_59_61Hz"] = float(rat_off[line].mean())
        out["offline_ratio_20_45Hz"] = float(rat_off[(f >= 20) & (f <= 45)].mean())
        out["offline_ratio_80_200Hz"] = float(rat_off[(f >= 80) & (f <= 200)].mean())

        # ---- online: causal scheme with aggregation latency delta ----
        per = {}
        for dsec in deltas_s:
            delta = int(round(dsec * FS))
            sm = G.gw_stream_create(ctx, [m], 1, C, W, stride, 1, G.GW_AGG_LATEST, delta, post)
            total = W + n_ev + delta + c + stride
            cleaned = np.zeros(total, np.float32)
            k = 0
            while (k + 1) * stride <= total:
                a = n_tr + k * stride
                w_in = np.ascontiguousarray(wit[None, :, a:a + stride], np.float32)
                s_in = np.ascontiguousarray(strain[None, a:a + stride], np.float32)
                o = np.zeros((1, stride), np.float32)
                G.gw_stream_push(sm, 1, w_in, s_in, o)
                t0 = k * stride - delta - c  # emitted times [k S - delta - c, k S + S - delta - c)
                if t0 >= 0:
                    cleaned[t0:t0 + stride] = o[0]
                k += 1
            G.gw_stream_destroy(sm)
            on = cleaned[W:W + n_ev].astype(np.float64)
            series["online"][f"{dsec:g}s"] = on[lo:hi]
            _, a_on = _asd(on[lo:hi])
            rat_on = a_on / a_raw
            per[f"{dsec:g}s"] = {
                "frac_50_70Hz_off_by_10pct": float(np.mean(np.abs(rat_on[band] / rat_off[band] - 1) > 0.1)),
                "ratio_59_61Hz": float(rat_on[line].mean())}
        out["online"] = per
        if return_series:
            out["series"] = series
        if post:
            G.gw_fir_destroy(post)
        G.gw_model_destroy(m)
    finally:
        G.gw_ctx_destroy(ctx)
    return out
