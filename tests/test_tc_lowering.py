"""Host-logic test of the tensor-core conv lowering (CPU only).

gw_tc_inspect returns the packed B-operand image, the K-step table and the
launch plan that the tcgen05 kernel uses.  This test replays the kernel's
data path in numpy -- input tile rows per (group, phase) plane with zero
padding, A and B operands gathered through the shared-memory descriptor
address rule (16-byte rows, 8-row core matrices, SBO = 128 B between
8-row groups, LBO between the two K-halves), accumulator chains, epilogue
position mapping -- and compares the result with the oracle's Conv1d /
ConvTranspose1d on the same bf16-rounded inputs.  Every address is checked
against its buffer, so an index slip fails here before the kernel runs.
"""
import numpy as np
import pytest

from oracle import layers as Lyr
from oracle.quant import to_bf16
from paper_2108_12430_gb300 import gwstream as G

rng = np.random.default_rng(2024)


def bf16_bits_to_f64(u16):
    return (u16.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def f64_to_bf16_bits(x):
    # inputs are already bf16-representable: truncation is exact
    return (np.asarray(x, np.float32).view(np.uint32) >> 16).astype(np.uint16)


def e4m3_table():
    """All 256 e4m3 codes decoded from the format's definition (sign, 4-bit
    exponent with bias 7, 3 mantissa bits; exponent 0 subnormal; S.1111.111 NaN)."""
    v = np.zeros(256)
    for b in range(256):
        s, e, m = b >> 7, (b >> 3) & 15, b & 7
        if e == 15 and m == 7:
            v[b] = np.nan
        elif e == 0:
            v[b] = m / 8.0 * 2.0 ** -6
        else:
            v[b] = (1 + m / 8.0) * 2.0 ** (e - 7)
        v[b] = -v[b] if s else v[b]
    return v


E4M3 = e4m3_table()
E4M3_CODE = {float(val): b for b, val in enumerate(E4M3) if np.isfinite(val) and not (val == 0 and b)}


def f64_to_e4m3_bits(x):
    # inputs are e4m3-representable: look the code up
    return np.array([E4M3_CODE[float(v)] for v in np.ravel(x)], np.uint8).reshape(np.shape(x))


def emulate(spec, x, img, table, md, fp8=False):
    transposed, cin, cout, k, stride, pl, pr, op = spec
    Gn, P, rows, MT, dmin, npad = md["groups"], md["in_P"], md["rows"], md["MT"], md["dmin"], md["npad"]
    Q, coutp, step_bytes, a_bytes = md["Q"], md["coutp"], md["step_bytes"], md["a_bytes"]
    # element size, channels per 16-byte row, K of one MMA
    esz, cg, kstep = (1, 16, 32) if fp8 else (2, 8, 16)
    lin = x.shape[1]
    lout, mout = md["lout"], md["mout"]
    assert rows * 16 * Gn * P <= a_bytes
    # a tile holds one slice of npad / nsplit columns; two accumulators of MT sub-tiles
    assert npad % md["nsplit"] == 0 and (npad // md["nsplit"]) % 32 == 0
    assert md["smem"] <= 227 * 1024 and md["ncols"] <= 512 and 2 * MT * (npad // md["nsplit"]) <= md["ncols"]
    assert Q * coutp <= npad
    xb = np.zeros((Gn * cg, lin))
    xb[:cin] = x
    if fp8:
        imgh = img.view(np.uint8)
        decode = lambda codes: E4M3[codes]
    else:
        imgh = img.view(np.uint16)
        decode = bf16_bits_to_f64
    out = np.zeros((cout, lout))
    written = np.zeros((cout, lout), int)
    r_idx = np.arange(128)[:, None]
    k_idx = np.arange(kstep)[None, :]
    for tile in range(md["tiles_per_item"]):
        m0 = tile * 128 * MT
        base = m0 + dmin
        A = np.zeros(a_bytes // esz, np.uint8 if fp8 else np.uint16)
        for plane in range(Gn * P):
            g, phi = plane // P, plane % P
            Lp = (lin - phi + P - 1) // P
            r0 = max(0, -base)
            r1 = max(r0, min(rows, Lp - base))
            for r in range(r0, r1):
                j = base + r
                assert 0 <= j < Lp
                a0 = (plane * rows + r) * cg
                vals = xb[g * cg:(g + 1) * cg, P * j + phi]
                A[a0:a0 + cg] = f64_to_e4m3_bits(vals) if fp8 else f64_to_bf16_bits(vals)
        D = np.zeros((MT, 128, npad))
        for s in range(md["n_steps"]):
            w0, w1 = int(table[2 * s]), int(table[2 * s + 1])

            def off(code):
                g, phi, dd = code & 255, (code >> 8) & 63, code >> 14
                return ((g * P + phi) * rows + dd) * 16

            o0, o1 = off(w0), off(w1)
            lbo = o1 - o0
            assert lbo >= 0
            # B operand: rows n, K-halves LBO = npad * 16 apart, 8-row groups SBO = 128 apart
            n_idx = np.arange(npad)[:, None]
            baddr = (s * step_bytes + (n_idx // 8) * 128 + (n_idx % 8) * 16 + (k_idx // cg) * (npad * 16)
                     + (k_idx % cg) * esz)
            assert baddr.max() + esz <= (s + 1) * step_bytes
            Bm = decode(imgh[baddr // esz])
            for mt in range(MT):
                start = o0 + mt * 2048
                aaddr = start + (r_idx // 8) * 128 + (r_idx % 8) * 16 + (k_idx // cg) * lbo + (k_idx % cg) * esz
                assert aaddr.min() >= 0 and aaddr.max() + esz <= a_bytes
                Am = decode(A[aaddr // esz])
                acc = Am @ Bm.T
                D[mt] = acc if s == 0 else D[mt] + acc
        # epilogue: row m, column n = sigma * coutp + o -> position Q m + sigma
        for mt in range(MT):
            for row in range(128):
                m = m0 + mt * 128 + row
                if m >= mout:
                    continue
                for n in range(npad):
                    sg, o = n // coutp, n % coutp
                    u = Q * m + sg
                    if sg < Q and o < cout and u < lout:
                        out[o, u] = D[mt, row, n]
                        written[o, u] += 1
    assert (written == 1).all()
    return out


CASES = [
    # DeepClean layers (transposed, cin, cout, k, stride, pad_l, pad_r, out_pad), input length
    ((0, 21, 8, 7, 1, 3, 3, 0), 2100, 1, 2),
    ((0, 8, 16, 7, 2, 3, 3, 0), 2102, 2, 2),
    ((0, 16, 32, 7, 2, 3, 3, 0), 1030, 2, 2),
    ((0, 32, 64, 7, 2, 3, 3, 0), 530, 2, 1),
    ((1, 64, 32, 7, 2, 3, 3, 1), 262, 1, 1),
    ((1, 32, 16, 7, 2, 3, 3, 1), 524, 1, 1),
    ((1, 16, 8, 7, 2, 3, 3, 1), 1048, 1, 1),
    ((0, 8, 1, 7, 1, 3, 3, 0), 2096, 1, 1),
    # BBHnet layers
    ((0, 2, 32, 16, 1, 7, 8, 0), 600, 1, 2),
    ((0, 32, 64, 7, 2, 3, 3, 0), 300, 2, 1),
    ((0, 64, 64, 7, 1, 3, 3, 0), 150, 1, 2),
    ((0, 128, 256, 1, 2, 0, 0, 0), 300, 2, 1),
    ((0, 256, 256, 7, 1, 3, 3, 0), 140, 1, 1),
    # the 2049-tap whitening FIR as an 8 -> 8 channel conv on the space-to-depth view
    ((0, 8, 8, 257, 1, 0, 0, 0), 600, 1, 1),
]


@pytest.mark.parametrize("batch", [1, 1 << 20])
@pytest.mark.parametrize("spec,lin,in_P,out_P", CASES)
def test_tc_lowering_matches_oracle(spec, lin, in_P, out_P, batch):
    # batch only steers the launch plan (a huge batch keeps large tiles); the
    # emulation replays item 0
    transposed, cin, cout, k, stride, pl, pr, op = spec
    w = to_bf16(rng.standard_normal((cout, cin, k)) * 0.2)
    x = to_bf16(rng.standard_normal((cin, lin)))
    # in_P = 0: the input comes in the phase count the layer asks for
    img, table, md = G.gw_tc_inspect(spec, G.GW_BF16, w, lin, 0, out_P, batch)
    assert md["in_P"] >= 1
    got = emulate(spec, x, img, table, md)
    if transposed:
        ref = Lyr.conv_transpose1d(x[None], np.transpose(w, (1, 0, 2)), np.zeros(cout), stride, pl, op)[0]
    else:
        ref = Lyr.conv1d(x[None], w, np.zeros(cout), stride, pl, pr)[0]
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


FP8_CASES = [c for c in CASES if c[0][0] == 0 and (c[0][2] >= 32 or c[0][1] == 2)]  # BBHnet-shaped convs


@pytest.mark.parametrize("spec,lin,in_P,out_P", FP8_CASES)
def test_tc_lowering_fp8_matches_oracle(spec, lin, in_P, out_P):
    # e4m3 operands: 16 channels per 16-byte row, K = 32 per MMA; weights
    # quantised per output channel with max |w| mapped to 448 (FP32 scale)
    from oracle.quant import to_e4m3
    transposed, cin, cout, k, stride, pl, pr, op = spec
    w = rng.standard_normal((cout, cin, k)) * 0.2
    x = to_e4m3(rng.standard_normal((cin, lin)) * 4)
    img, table, md = G.gw_tc_inspect(spec, G.GW_FP8, w, lin, 0, out_P, 1)
    ws = (np.abs(w).max(axis=(1, 2)) / 448.0).astype(np.float32).astype(np.float64)
    wq = to_e4m3((w / ws[:, None, None]).astype(np.float32))
    got = emulate(spec, x, img, table, md, fp8=True)
    ref = Lyr.conv1d(x[None], wq, np.zeros(cout), stride, pl, pr)[0]
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-9)


def test_tc_instruction_descriptor_fields():
    # kind::f16: D=F32 (bit 4), A=B=BF16 (bits 7, 10), K-major, N>>3 at 17, M>>4 at 24
    _, _, md = G.gw_tc_inspect((0, 32, 64, 7, 2, 3, 3, 0), G.GW_BF16, np.zeros((64, 32, 7)), 256, 0, 1)
    d = md["idesc"]
    assert (d >> 4) & 3 == 1 and (d >> 7) & 7 == 1 and (d >> 10) & 7 == 1
    assert (d >> 15) & 3 == 0 and (d >> 17) & 63 == (md["npad"] // md["nsplit"]) >> 3 and (d >> 24) & 31 == 128 >> 4


def test_tc_layer_plans_fold_positions():
    # DeepClean layers get N >= 64 columns by folding output positions
    specs = [(0, 21, 8, 7, 1, 3, 3, 0), (0, 8, 16, 7, 2, 3, 3, 0), (0, 16, 32, 7, 2, 3, 3, 0),
             (0, 32, 64, 7, 2, 3, 3, 0), (1, 64, 32, 7, 2, 3, 3, 1), (1, 32, 16, 7, 2, 3, 3, 1),
             (1, 16, 8, 7, 2, 3, 3, 1)]
    for sp in specs:
        _, _, md = G.gw_tc_inspect(sp, G.GW_BF16, np.zeros((sp[2], sp[1], sp[3])), 32768, 0, 1)
        assert md["npad"] >= 64 and md["Q"] * md["coutp"] == md["npad"], (sp, md)


def _bbhnet_plans(precision, batch):
    """Launch plans of BBHnet's 13 conv layers at `batch` items of 2048 samples."""
    from paper_2108_12430_gb300 import synth
    names = ["stem", "b1c1", "b1c2", "b1sc", "b2c1", "b2c2", "b2sc", "b3c1", "b3c2", "b3sc", "b4c1", "b4c2", "b4sc"]
    lin, out = 2048, {}
    for nm, l in zip(names, synth.bbhnet_layers()):
        _, cin, cout, k, s, pl, pr, op, _, _ = l
        li = lin_out if nm.endswith("c2") else (lin_blk if nm.endswith("sc") else lin)
        _, _, md = G.gw_tc_inspect((0, cin, cout, k, s, pl, pr, op), precision, np.zeros((cout, cin, k)), li, 0, 1,
                                   batch)
        if nm.endswith("c1"):
            lin_blk, lin_out = li, md["lout"]
        if nm == "stem" or nm.endswith("sc"):
            lin = md["lout"]
        out[nm] = md
    return out


@pytest.mark.parametrize("precision", [G.GW_BF16, G.GW_FP8])
@pytest.mark.parametrize("batch", [1, 2, 3, 16, 64, 100, 256, 1024])
def test_tc_plans_fit_and_weight_rings_are_well_formed(precision, batch):
    # every plan fits the SM (shared memory per CTA and per SM, TMEM columns);
    # a streamed weight ring filled by two producers has an even number of
    # stages (each producer owns every other stage), packed slice stages
    # belong to split layers only, and a stage holds whole K-steps
    for nm, md in _bbhnet_plans(precision, batch).items():
        assert md["smem"] <= 227 * 1024 and md["per_sm"] * (md["smem"] + 1024) <= 228 * 1024, (nm, md)
        assert md["ncols"] <= 512 and md["per_sm"] * md["ncols"] <= 512, (nm, md)
        assert 1 <= md["na"] <= 6, (nm, md)
        resident = md["sps"] == md["n_steps"] and md["nst"] == 1 and md["wprod"] == 1
        if md["wprod"] == 2:
            assert md["nst"] >= 2 and md["nst"] % 2 == 0, (nm, md)
        if md["wcompact"]:
            assert md["nsplit"] > 1 and md["MT"] == 1 and md["wstep"] * md["nsplit"] == md["step_bytes"], (nm, md)
        else:
            assert md["wstep"] == md["step_bytes"], (nm, md)
        if not resident:
            assert md["sps"] * md["wstep"] <= 64 * 1024, (nm, md)
            assert md["na"] >= 2 or md["nst"] >= 2, (nm, md)  # loads overlap MMAs in one ring or the other


def test_tc_plans_stream_the_deep_layers_in_large_stages():
    # at batch 256 the 256-channel layers stream their weights in 64 KB stages
    # (two, filled by two producers); at batch 1 they are split over 8 CTAs
    # and each streams only its packed slice
    big = _bbhnet_plans(G.GW_BF16, 256)
    for nm in ("b4c1", "b4c2"):
        md = big[nm]
        assert md["nsplit"] == 1 and md["sps"] * md["wstep"] == 64 * 1024 and md["nst"] == 2 and md["wprod"] == 2
    small = _bbhnet_plans(G.GW_BF16, 1)
    for nm in ("b4c1", "b4c2"):
        md = small[nm]
        assert md["nsplit"] == 8 and md["wcompact"] == 1 and md["wstep"] == md["step_bytes"] // 8
