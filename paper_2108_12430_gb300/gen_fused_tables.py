"""Writes csrc/fused_tables.h: the compile-time layer tables of the fused
DeepClean kernel (csrc/k_fused.cu).

The fused kernel issues every layer's MMAs and runs every layer's epilogue
from constants known at compile time (descriptor tables read at run time
slow the single MMA-issuing thread down by half).  The constants are the
tensor-core lowering of the eight DeepClean layers (Conv 21->8 k7 s1, Conv
8->16->32->64 k7 s2, ConvT 64->32->16->8 k7 s2, Conv 8->1 k7; 17-24 input
channels give the same tables) with the fused kernel's folding J per layer,
enumerated here the way the library's host lowering (lower_layer in
csrc/k_tc.cu) does it.  The library checks at model creation that its own
lowering gives exactly these tables and otherwise does not use the fused
kernel, so a stale header cannot produce wrong results.

    python -m paper_2108_12430_gb300.gen_fused_tables
"""
from __future__ import annotations

import os

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "fused_tables.h")

# (transposed, c_in, c_out, k, stride, pad, out_pad, J)
LAYERS = [
    (0, 21, 8, 7, 1, 3, 0, 8),
    (0, 8, 16, 7, 2, 3, 0, 4),
    (0, 16, 32, 7, 2, 3, 0, 2),
    (0, 32, 64, 7, 2, 3, 0, 1),
    (1, 64, 32, 7, 2, 3, 1, 1),
    (1, 32, 16, 7, 2, 3, 1, 2),
    (1, 16, 8, 7, 2, 3, 1, 4),
    (0, 8, 1, 7, 1, 3, 0, 8),
]
ROWS_M = 128
W_CHUNK = 12288


def lower(tr, cin, cout, k, s, pad, J):
    """Slices (group, phase, row shift) paired into K-steps, in the order of
    the host lowering."""
    G = (cin + 7) // 8
    Q = 2 * J if tr else J
    P = J if tr else s * J
    coutp = 1 if cout == 1 else (cout + 7) // 8 * 8
    npad = max(32, (Q * coutp + 31) // 32 * 32)
    cons = []
    for sg in range(Q):
        for kk in range(k):
            if not tr:
                q = s * sg + kk - pad
            else:
                j, psi = sg // 2, sg % 2
                if (psi + pad - kk) % 2 != 0:
                    continue
                q = j + (psi + pad - kk) // 2
            cons.append((q % P, q // P))
    dmin = min(d for _, d in cons)
    dmax = max(d for _, d in cons)
    pos = sorted(set(cons))
    steps, left = [], []
    for phi, d in pos:
        g = 0
        while g + 1 < G:
            steps.append(((g, phi, d - dmin), (g + 1, phi, d - dmin)))
            g += 2
        if g < G:
            left.append((g, phi, d - dmin))
    key = lambda a: (a[0] * 64 + a[1]) * 4096 + a[2]
    left.sort(key=key)
    for i in range(0, len(left), 2):
        steps.append((left[i], left[i + 1] if i + 1 < len(left) else left[i]))
    steps = [(b, a) if key(b) < key(a) else (a, b) for a, b in steps]
    rows = ROWS_M + (dmax - dmin)  # 16-byte rows; planes need no further alignment
    return dict(G=G, P=P, Q=Q, coutp=coutp, npad=npad, dmin=dmin, rows=rows, n_steps=len(steps), steps=steps)


def half_order(m, prev):
    """The steps of a layer reordered so that those reading only the outputs of
    the previous layer's first 32 accumulator columns come first (stable), and
    their number.  Column n = sigma * coutp + o of the previous layer holds
    output position offset sigma (this layer's phase plane) of channel o (this
    layer's channel group o / 8)."""
    if prev is None:
        return list(range(m["n_steps"])), 0
    half = lambda sl: (sl[1] * prev["coutp"] + 8 * sl[0]) // 32
    dep = [max(half(a), half(b)) for a, b in m["steps"]]
    first = [i for i in range(m["n_steps"]) if dep[i] == 0]
    return first + [i for i in range(m["n_steps"]) if dep[i] != 0], len(first)


def apack_of(m, order):
    off = lambda a: ((a[0] * m["P"] + a[1]) * m["rows"] + a[2]) * 16
    out = []
    for i in order:
        a, b = m["steps"][i]
        o0, o1 = off(a), off(b)
        out.append((o0 >> 4) | (((o1 - o0) >> 4) << 16))
    return out


def render():
    """The header's text."""
    lines = [
        "// Generated by paper_2108_12430_gb300/gen_fused_tables.py -- do not edit.",
        "// Compile-time tables of the fused DeepClean kernel (k_fused.cu): per layer the",
        "// tensor-core lowering (input buffer geometry, K-steps, per-step A-operand",
        "// start and LBO in 16-byte units relative to the input buffer) and the weight",
        "// chunking.  Steps are ordered so that the first `split` read only the",
        "// outputs of the previous layer's first 32 accumulator columns (the MMAs",
        "// can start once half the previous epilogue is done); order(i) is the host",
        "// lowering's index of step i.  The host plan checks them against its own lowering.",
        "#pragma once",
        "#include <stdint.h>",
        "",
        "namespace gw {",
        "namespace fz {",
        "",
    ]
    chunk0 = 0
    prev = None
    for li, (tr, cin, cout, k, s, pad, op, J) in enumerate(LAYERS):
        m = lower(tr, cin, cout, k, s, pad, J)
        order, split = half_order(m, prev)
        apack = apack_of(m, order)
        prev = m
        step_bytes = 32 * m["npad"]
        sps = max(1, W_CHUNK // step_bytes)
        n_chunks = (m["n_steps"] + sps - 1) // sps
        lg = lambda v: v.bit_length() - 1
        lines += [
            f"struct L{li} {{",
            f"  static constexpr int transposed = {tr}, cin = {cin}, cout = {cout}, K = {k}, stride = {s}, pad = {pad};",
            f"  static constexpr int J = {J}, Q = {m['Q']}, lgQ = {lg(m['Q'])}, coutp = {m['coutp']}, "
            f"lgcoutp = {lg(m['coutp'])}, npad = {m['npad']};",
            f"  static constexpr int G = {m['G']}, P = {m['P']}, lgP = {lg(m['P'])}, rows = {m['rows']}, "
            f"dmin = {m['dmin']};",
            f"  static constexpr int n_steps = {m['n_steps']}, step_bytes = {step_bytes}, sps = {sps}, "
            f"n_chunks = {n_chunks}, chunk0 = {chunk0}, split = {split};",
            f"  __host__ __device__ static constexpr uint32_t apack(int i) {{",
            f"    constexpr uint32_t t[{m['n_steps']}] = {{{', '.join(str(v) for v in apack)}}};",
            "    return t[i];",
            "  }",
            f"  // step i issues the host lowering's step order(i)",
            f"  __host__ __device__ static constexpr int order(int i) {{",
            f"    constexpr int t[{m['n_steps']}] = {{{', '.join(str(v) for v in order)}}};",
            "    return t[i];",
            "  }",
            "};",
            "",
        ]
        chunk0 += n_chunks
    lines += [f"constexpr int kChunks = {chunk0};", "", "}  // namespace fz", "}  // namespace gw", ""]
    return "\n".join(lines)


def main():
    with open(OUT, "w") as f:
        f.write(render())
    print(OUT)


if __name__ == "__main__":
    main()
