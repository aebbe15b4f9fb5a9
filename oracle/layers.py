"""Layer definitions in float64 (test infrastructure; see package header).

Conv1d (DeepClean/BBHnet conv layers):
    y[b, o, t] = bias[o] + sum_{i, k} w[o, i, k] * x[b, i, s*t + k - p_l]
with x = 0 outside [0, L) and L_out = floor((L + p_l + p_r - K) / s) + 1.

ConvTranspose1d (DeepClean decoder), scatter form:
    y[b, o, s*t + k - p] += w[i, o, k] * x[b, i, t]    for all i, t, k,
kept for output indices in [0, L_out), L_out = (L - 1) s - 2 p + K + op.

BatchNorm in eval mode: z_hat = (z - mu) / sqrt(var + eps) * gamma + beta,
eps = 1e-5 (PyTorch's default; the source is silent).

The fold (used by the library, checked here): with a = gamma / sqrt(var+eps),
    w' = w * a  (along the output-channel axis),  b' = (b - mu) * a + beta.
"""
from __future__ import annotations

import numpy as np

BN_EPS = 1e-5


def conv1d(x, w, b, stride=1, pad_l=0, pad_r=0):
    """x (B, C_in, L), w (C_out, C_in, K), b (C_out,) -> (B, C_out, L_out)."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    B, cin, L = x.shape
    cout, cin_w, K = w.shape
    assert cin_w == cin
    lout = (L + pad_l + pad_r - K) // stride + 1
    xp = np.zeros((B, cin, L + pad_l + pad_r))
    xp[:, :, pad_l:pad_l + L] = x
    y = np.zeros((B, cout, lout)) + np.asarray(b, np.float64)[None, :, None]
    idx = stride * np.arange(lout)
    for k in range(K):
        # (C_out, C_in) @ (B, C_in, L_out) -> (B, C_out, L_out)
        y += np.matmul(w[:, :, k], xp[:, :, idx + k])
    return y


def conv_transpose1d(x, w, b, stride=2, pad=0, out_pad=0):
    """x (B, C_in, L), w (C_in, C_out, K), b (C_out,) -> (B, C_out, L_out)."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    B, cin, L = x.shape
    cin_w, cout, K = w.shape
    assert cin_w == cin
    lout = (L - 1) * stride - 2 * pad + K + out_pad
    full = np.zeros((B, cout, (L - 1) * stride + K + out_pad))
    t = np.arange(L)
    for k in range(K):
        # scatter: position s*t + k of the un-cropped output
        full[:, :, stride * t + k] += np.matmul(w[:, :, k].T, x)
    y = full[:, :, pad:pad + lout]
    return y + np.asarray(b, np.float64)[None, :, None]


def batchnorm_eval(z, gamma, beta, mean, var, eps=BN_EPS):
    """Eval-mode BatchNorm over the channel axis 1 of z (B, C, L)."""
    g = np.asarray(gamma, np.float64)[None, :, None]
    bt = np.asarray(beta, np.float64)[None, :, None]
    m = np.asarray(mean, np.float64)[None, :, None]
    v = np.asarray(var, np.float64)[None, :, None]
    return (z - m) / np.sqrt(v + eps) * g + bt


def fold_bn(w, b, gamma, beta, mean, var, out_axis=0, eps=BN_EPS):
    """BatchNorm folded into the preceding layer's weight and bias (FP64)."""
    a = np.asarray(gamma, np.float64) / np.sqrt(np.asarray(var, np.float64) + eps)
    shape = [1, 1, 1]
    shape[out_axis] = -1
    w2 = np.asarray(w, np.float64) * a.reshape(shape)
    b2 = (np.asarray(b, np.float64) - np.asarray(mean, np.float64)) * a + np.asarray(beta, np.float64)
    return w2, b2


def activation(z, act):
    if act == "tanh":
        return np.tanh(z)
    if act == "relu":
        return np.maximum(z, 0.0)
    assert act == "none"
    return z


def global_avg_pool(z):
    """(B, C, L) -> (B, C): mean over time."""
    return np.asarray(z, np.float64).mean(axis=-1)


def linear(h, w, b):
    """(B, C) @ w (C,) + b -> (B,) logits."""
    return np.asarray(h, np.float64) @ np.asarray(w, np.float64) + float(np.asarray(b).ravel()[0])
