"""DeepClean training loss and its exact gradient in float64 (test infrastructure).

The paper retrains DeepClean on recent data (Main text, model validity and
retraining) but gives no loss.  Reading taken: the band-limited,
inverse-PSD-weighted mean-square error

    L = (1 / N) sum_{b, n} r[b, n]^2,   r = g (*) (s - y_hat)   (valid mode),

with g the 55-65 Hz loss-weight FIR of ``oracle.fir.band_loss_fir``, s the
strain, y_hat the network's noise prediction and N the number of valid
output samples.  BatchNorm runs in eval mode (running statistics fixed), so
the trainable parameters per layer are the raw w, b, gamma, beta.

The gradient is reverse-mode written out layer by layer:

* conv  u = b + sum_k w[:, :, k] x_pad[:, s t + k]:
  dW[:, :, k] = sum_{b,t} du[:, t] x_pad[:, s t + k]^T, db = sum du,
  dx_pad[:, s t + k] += w[:, :, k]^T du[:, t].
* convT u[:, s t + k - p] += w[:, :, k]^T x[:, t]:
  dW[:, :, k] = sum x[:, t] du[:, s t + k - p]^T, dx[:, t] = sum_k w[:, :, k] du[:, s t + k - p].
* BN + act: v = (u - mu) a gamma' ... with a = 1 / sqrt(var + eps):
  dv = dy * act'(v), dgamma = sum dv (u - mu) a, dbeta = sum dv, du = dv gamma a.
"""
from __future__ import annotations

import numpy as np

from . import layers as Lyr
from .fir import fir_valid


def _conv_fwd(x, spec, p):
    kind, cin, cout, k, s, pl, pr, op, bn, act = spec
    if kind == "conv":
        return Lyr.conv1d(x, p["w"], p["b"], stride=s, pad_l=pl, pad_r=pr)
    return Lyr.conv_transpose1d(x, p["w"], p["b"], stride=s, pad=pl, out_pad=op)


def _conv_bwd(x, du, spec, p):
    """Gradients of a conv / convT layer: returns (dx, dw, db)."""
    kind, cin, cout, K, s, pl, pr, op, bn, act = spec
    w = np.asarray(p["w"], np.float64)
    B, _, L = x.shape
    db = du.sum(axis=(0, 2))
    dw = np.zeros_like(w)
    if kind == "conv":
        lout = du.shape[-1]
        xp = np.zeros((B, cin, L + pl + pr))
        xp[:, :, pl:pl + L] = x
        dxp = np.zeros_like(xp)
        idx = s * np.arange(lout)
        for k in range(K):
            cols = xp[:, :, idx + k]                      # (B, cin, lout)
            dw[:, :, k] = np.einsum("bot,bit->oi", du, cols)
            dxp[:, :, idx + k] += np.matmul(w[:, :, k].T, du)
        return dxp[:, :, pl:pl + L], dw, db
    # transposed conv: output index s t + k - p for input index t
    lout = du.shape[-1]
    full = np.zeros((B, cout, (L - 1) * s + K + op))
    full[:, :, pl:pl + lout] = du
    t = np.arange(L)
    dx = np.zeros((B, cin, L))
    for k in range(K):
        g = full[:, :, s * t + k]                          # (B, cout, L)
        dw[:, :, k] = np.einsum("bit,bot->io", x, g)
        dx += np.matmul(w[:, :, k], g)
    return dx, dw, db


def deepclean_loss_and_grad(x, strain, params, layers, g):
    """Loss and gradients w.r.t. raw (w, b, gamma, beta) of every layer.

    x (B, C, L) standardised witness windows, strain (B, L), g loss FIR.
    Returns (loss, y_hat (B, L), grads list of dicts).
    """
    h = np.asarray(x, np.float64)
    tape = []
    for spec, p in zip(layers, params):
        u = _conv_fwd(h, spec, p)
        v = u
        if spec[8]:
            a = 1.0 / np.sqrt(np.asarray(p["var"], np.float64) + Lyr.BN_EPS)
            v = (u - np.asarray(p["mean"], np.float64)[None, :, None]) * (a * p["gamma"])[None, :, None] \
                + np.asarray(p["beta"], np.float64)[None, :, None]
        y = Lyr.activation(v, spec[9])
        tape.append((h, u, y))
        h = y
    y_hat = h[:, 0, :]
    e = np.asarray(strain, np.float64) - y_hat
    r = fir_valid(e, g)
    N = r.size
    loss = float(np.sum(r ** 2) / N)
    # d loss / d e[m] = sum_n (2 r[n] / N) g[m - n]
    dr = 2.0 * r / N
    K = len(g)
    de = np.zeros_like(e)
    for k in range(K):
        de[:, k:k + r.shape[-1]] += g[k] * dr
    dh = -de[:, None, :]
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        spec, p = layers[li], params[li]
        h_in, u, y = tape[li]
        act = spec[9]
        if act == "tanh":
            dv = dh * (1.0 - y ** 2)
        elif act == "relu":
            dv = dh * (y > 0)
        else:
            dv = dh
        gr = {}
        if spec[8]:
            a = 1.0 / np.sqrt(np.asarray(p["var"], np.float64) + Lyr.BN_EPS)
            uc = u - np.asarray(p["mean"], np.float64)[None, :, None]
            gr["gamma"] = np.sum(dv * uc, axis=(0, 2)) * a
            gr["beta"] = np.sum(dv, axis=(0, 2))
            du = dv * (a * np.asarray(p["gamma"], np.float64))[None, :, None]
        else:
            du = dv
        dx, gr["w"], gr["b"] = _conv_bwd(h_in, du, spec, p)
        grads[li] = gr
        dh = dx
    return loss, y_hat, grads


def deepclean_loss(x, strain, params, layers, g):
    """Loss only (for finite differences)."""
    h = np.asarray(x, np.float64)
    for spec, p in zip(layers, params):
        u = _conv_fwd(h, spec, p)
        if spec[8]:
            u = Lyr.batchnorm_eval(u, p["gamma"], p["beta"], p["mean"], p["var"])
        h = Lyr.activation(u, spec[9])
    r = fir_valid(np.asarray(strain, np.float64) - h[:, 0, :], g)
    return float(np.sum(r ** 2) / r.size)
