"""The whole-network DeepClean kernel's compile-time step tables (no GPU).

The kernel issues a hidden layer's first `split` K-steps as soon as the first
half of the previous layer's epilogue is stored.  These tests check, from the
epilogue's own column -> (channel group, phase plane) rule written out here,
that those steps read nothing the second half writes, that the step order is a
permutation of the host lowering's, and that the committed header is what the
generator writes.
"""
import os

import numpy as np
import pytest

from paper_2108_12430_gb300 import gen_fused_tables as gft
from paper_2108_12430_gb300 import gwstream as G

HEADER = os.path.join(os.path.dirname(gft.__file__), "csrc", "fused_tables.h")


def lowered():
    out, prev = [], None
    for tr, cin, cout, k, s, pad, op, J in gft.LAYERS:
        m = gft.lower(tr, cin, cout, k, s, pad, J)
        order, split = gft.half_order(m, prev)
        out.append((m, order, split))
        prev = m
    return out


def planes_written_by_half(prev):
    """Planes (group, phase) of the next layer's input that each half of the
    previous layer's epilogue writes: half h, 8-column group j covers columns
    n0 = 32 h + 8 j, i.e. output offset n0 // coutp (the phase plane) of
    channels n0 % coutp .. + 7 (group (n0 % coutp) // 8)."""
    written = {0: set(), 1: set()}
    for half in range(2):
        for j in range(4):
            n0 = 32 * half + 8 * j
            sigma, o0 = n0 // prev["coutp"], n0 % prev["coutp"]
            written[half].add((o0 // 8, sigma))
    return written


def test_step_order_is_a_permutation():
    for m, order, split in lowered():
        assert sorted(order) == list(range(m["n_steps"]))
        assert 0 <= split <= m["n_steps"]


@pytest.mark.parametrize("li", range(1, len(gft.LAYERS)))
def test_first_steps_read_only_the_first_half(li):
    tables = lowered()
    prev = tables[li - 1][0]
    m, order, split = tables[li]
    assert prev["npad"] == 64  # the previous layer is a hidden layer drained in two halves
    written = planes_written_by_half(prev)
    assert not written[0] & written[1]
    for i, h in enumerate(order):
        planes = {(g, phi) for g, phi, _ in m["steps"][h]}
        assert planes <= written[0] | written[1]
        if i < split:
            assert planes <= written[0], (li, i, planes)
    # every step after the split reads something of the second half (the split is tight)
    for h in order[split:]:
        assert {(g, phi) for g, phi, _ in m["steps"][h]} & written[1]


def test_first_layer_keeps_the_host_order():
    m, order, split = lowered()[0]
    assert order == list(range(m["n_steps"])) and split == 0


def test_committed_header_is_current():
    with open(HEADER) as f:
        assert f.read() == gft.render()


def decode(code):
    """A K-step table word of the host lowering: (channel group, phase plane, row shift)."""
    return code & 255, (code >> 8) & 63, code >> 14


@pytest.mark.parametrize("li", range(len(gft.LAYERS) - 1))
def test_tables_match_the_libraries_own_lowering(li):
    """The library lowers each hidden layer itself (gw_tc_inspect, host only;
    the same lowering the per-layer kernel runs and the model checks the
    tables against before it uses the whole-network kernel): same geometry,
    and every kernel step's A-operand start and LBO, computed from the
    library's slice codes with the whole-network buffers' rows per plane,
    equal the header's packed value.  (The output layer is lowered there with
    another folding, so only the model-creation check covers it.)"""
    tr, cin, cout, k, s, pad, op, J = gft.LAYERS[li]
    m, order, _ = lowered()[li]
    _, table, md = G.gw_tc_inspect((tr, cin, cout, k, s, pad, pad, op), G.GW_BF16, np.zeros((cout, cin, k)),
                                   32768, 0, 1, 64)
    assert (md["Q"], md["n_steps"], md["npad"], md["in_P"], md["dmin"], md["groups"], md["coutp"]) == \
        (m["Q"], m["n_steps"], m["npad"], m["P"], m["dmin"], m["G"], m["coutp"])
    assert 128 + md["dspan"] == m["rows"]
    rows, P = m["rows"], m["P"]
    packed = gft.apack_of(m, order)
    for i, h in enumerate(order):
        o0, o1 = (((g * P + phi) * rows + dd) * 16 for g, phi, dd in (decode(int(table[2 * h])),
                                                                       decode(int(table[2 * h + 1]))))
        assert o1 >= o0
        assert packed[i] == (o0 >> 4) | (((o1 - o0) >> 4) << 16), (li, i)
