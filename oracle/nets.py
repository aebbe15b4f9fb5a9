"""DeepClean-shaped and BBHnet-shaped networks in float64 (test infrastructure).

The paper names the two models (Sec. 1: DeepClean, a 1-D convolutional
autoencoder predicting witness-coupled noise in strain; BBHnet, a 1-D CNN
separating binary-black-hole signals from noise) but prints no architecture.
The layer tables come in as plain data (``layers`` argument: tuples of
(kind, c_in, c_out, k, stride, pad_left, pad_right, out_pad, bn, act)):

* DeepClean: Conv 21->8 (k7, s1, p3), Conv 8->16->32->64 (k7, s2, p3),
  ConvT 64->32->16->8 (k7, s2, p3, output padding 1), each with eval-mode
  BatchNorm and tanh; output Conv 8->1 (k7, s1, p3) with bias only.  The
  first conv has stride 1 so that 3 stride-2 downs and 3 stride-2 ups give
  back the input length.
* BBHnet: stem Conv 2->32 (k16, pad 7 left / 8 right) + BN + ReLU; four
  residual blocks with C_out = 32, 64, 128, 256, each
  relu(BN(conv2(relu(BN(conv1(x))))) + BN(shortcut(x))) with conv1 k7 s2 p3,
  conv2 k7 s1 p3, shortcut k1 s2; global average pool; linear 256 -> 1.

Parity of these tables with the paper's trained networks is unpinned (the
paper prints neither); the oracle follows the tables exactly.
"""
from __future__ import annotations

import numpy as np

from . import layers as Lyr


def apply_layer(x, spec, p, with_act=True):
    """One conv / transposed-conv layer: linear op, BatchNorm, activation."""
    kind, cin, cout, k, s, pl, pr, op, bn, act = spec
    if kind == "conv":
        z = Lyr.conv1d(x, p["w"], p["b"], stride=s, pad_l=pl, pad_r=pr)
    else:
        assert pl == pr
        z = Lyr.conv_transpose1d(x, p["w"], p["b"], stride=s, pad=pl, out_pad=op)
    if bn:
        z = Lyr.batchnorm_eval(z, p["gamma"], p["beta"], p["mean"], p["var"])
    return Lyr.activation(z, act) if with_act else z


def standardize(x, mean=None, std=None):
    """Per-channel (x - mu_c) / sigma_c of the model input (B, C, L)."""
    x = np.asarray(x, np.float64)
    if mean is not None:
        x = x - np.asarray(mean, np.float64)[None, :, None]
    if std is not None:
        x = x / np.asarray(std, np.float64)[None, :, None]
    return x


def deepclean_forward(x, params, layers, mean=None, std=None):
    """x (B, 21, L) witness windows -> (B, L) predicted strain noise."""
    h = standardize(x, mean, std)
    for spec, p in zip(layers, params):
        h = apply_layer(h, spec, p)
    return h[:, 0, :]


def bbhnet_forward(x, params, head, layers):
    """x (B, 2, L) whitened strain -> (B,) logits."""
    h = apply_layer(np.asarray(x, np.float64), layers[0], params[0])
    i = 1
    while i < len(layers):
        a = apply_layer(h, layers[i], params[i])
        a = apply_layer(a, layers[i + 1], params[i + 1])
        sc = apply_layer(h, layers[i + 2], params[i + 2])
        h = np.maximum(a + sc, 0.0)
        i += 3
    return Lyr.linear(Lyr.global_avg_pool(h), head["w"], head["b"])
