"""Round-to-nearest-even casts in float64 (test infrastructure).

The reduced-precision paths store operands as bfloat16 (8-bit exponent,
7 stored mantissa bits) or float8 e4m3 (4-bit exponent with bias 7, 3 stored
mantissa bits, largest finite 448, no infinities); every FP32 -> narrow cast
rounds to nearest, ties to even, and e4m3 saturates to +-448.
These are written from the formats' definitions: a value with binary
exponent e is rounded to a multiple of 2^(e - m) (m mantissa bits), with e
clamped to the smallest normal exponent so that subnormals keep a fixed
quantum.
"""
from __future__ import annotations

import numpy as np


def _round_to_grid(x, mant_bits, min_exp):
    x = np.asarray(x, np.float64)
    ax = np.abs(x)
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(ax > 0, ax, 1.0)))
    e = np.maximum(e, min_exp)
    q = np.exp2(e - mant_bits)
    # numpy's rint rounds half to even
    return np.sign(x) * np.rint(ax / q) * q


def to_bf16(x):
    """float64 -> nearest bfloat16 value (returned as float64)."""
    x32 = np.asarray(x, np.float32).astype(np.float64)
    return _round_to_grid(x32, 7, -126)


def to_e4m3(x):
    """float64 -> nearest float8 e4m3 value, saturating at +-448."""
    y = _round_to_grid(np.asarray(x, np.float64), 3, -6)
    return np.clip(y, -448.0, 448.0)
