"""The whole-network DeepClean kernel's compile-time step tables (no GPU).

The kernel issues a hidden layer's first `split` K-steps as soon as the first
half of the previous layer's epilogue is stored.  These tests check, from the
epilogue's own column -> (channel group, phase plane) rule written out here,
that those steps read nothing the second half writes, that the step order is a
permutation of the host lowering's, and that the committed header is what the
generator writes.
"""
import os

import pytest

from paper_2108_12430_gb300 import gen_fused_tables as gft

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
