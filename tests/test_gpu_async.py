"""Queued host-buffer pushes (gw_stream_push_async / gw_stream_sync).

A queued push runs the same kernels in the same order as a synchronous
host-mode push, so its outputs are compared bit for bit with those of
gw_stream_push on a second stream fed the same data (whose parity with the
oracle the other GPU tests establish), and once directly with the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import nets, stream as ostream
from paper_2108_12430_gb300 import gwstream as G, synth
from tests.gpu_util import Ctx, rel_l2
from tests.test_gpu_f32 import TOL32

pytestmark = pytest.mark.gpu


@pytest.fixture
def ctx(gpu_lib):
    c = Ctx()
    yield c
    c.close()


def pinned(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()
    return t


def make_stream(ctx, m, W, S, nb, mode=G.GW_AGG_AVERAGE, delta=None):
    s = G.gw_stream_create(ctx.h, [m], 1, 21, W, S, nb, mode, W - S if delta is None else delta)
    ctx.objs.append((G.gw_stream_destroy, s))
    return s


def split(w, x, sizes, S):
    out, t = [], 0
    for n in sizes:
        out.append((n, w[:, :, t:t + n * S], x[:, t:t + n * S]))
        t += n * S
    return out


@pytest.mark.parametrize("prec", [G.GW_FP32, G.GW_BF16])
def test_async_pushes_match_sync_pushes(ctx, prec):
    m = ctx.deepclean(2, prec)
    W, S, sizes = 1024, 128, [3, 1, 5, 4, 2, 5, 1]
    rng = np.random.default_rng(21)
    T = sum(sizes) * S
    w = synth.witness_channels(21, 21, T)[None].astype(np.float32)
    x = rng.standard_normal((1, T)).astype(np.float32)
    parts = split(w, x, sizes, S)
    ref = []
    s_sync = make_stream(ctx, m, W, S, 5)
    for n, wp, xp in parts:
        o = np.zeros((1, n * S), np.float32)
        G.gw_stream_push(s_sync, n, np.ascontiguousarray(wp), np.ascontiguousarray(xp), o)
        ref.append(o)
    s = make_stream(ctx, m, W, S, 5)
    st = torch.cuda.Stream()
    bufs = [(n, pinned(wp), pinned(xp), torch.zeros(1, n * S).pin_memory()) for n, wp, xp in parts]
    # two sequences of queued pushes with a synchronisation between them
    for lo, hi in ((0, 4), (4, len(bufs))):
        for n, wb, xb, ob in bufs[lo:hi]:
            G.gw_stream_push_async(s, n, wb.data_ptr(), xb.data_ptr(), ob.data_ptr(), st.cuda_stream)
        G.gw_stream_sync(s)
    assert G.gw_stream_head(s) == T
    for (n, _, _, ob), r in zip(bufs, ref):
        assert np.array_equal(ob.numpy(), r)
    G.gw_stream_status(s)
    if prec == G.GW_FP32:
        got = np.concatenate([ob.numpy().reshape(n, S) for n, _, _, ob in bufs])
        params = synth.deepclean_params(2)
        fwd = lambda wins: nets.deepclean_forward(wins, params, synth.DEEPCLEAN_LAYERS, None, None)
        _, want = ostream.run_deepclean_stream(fwd, w[0].astype(np.float64), x[0].astype(np.float64), W, S,
                                               sum(sizes), ostream.AVERAGE, W - S)
        assert got.shape == want.shape
        assert rel_l2(got, want) <= TOL32


def test_async_rejection_rewinds_to_the_rejected_push(ctx):
    # queued push 2 of 5 holds a NaN: pushes 0 and 1 complete, 2..4 change
    # nothing and the head is rewound; pushing 2..4 again (valid) gives what a
    # stream that never saw the NaN gives
    m = ctx.deepclean(3, G.GW_BF16)
    W, S, n = 1024, 128, 5
    rng = np.random.default_rng(4)
    w = rng.standard_normal((1, 21, n * S)).astype(np.float32)
    x = rng.standard_normal((1, n * S)).astype(np.float32)
    parts = split(w, x, [1] * n, S)
    s_ref = make_stream(ctx, m, W, S, 2)
    ref = []
    for _, wp, xp in parts:
        o = np.zeros((1, S), np.float32)
        G.gw_stream_push(s_ref, 1, np.ascontiguousarray(wp), np.ascontiguousarray(xp), o)
        ref.append(o)
    s = make_stream(ctx, m, W, S, 2)
    st = torch.cuda.Stream()
    bufs = [(pinned(wp), pinned(xp), torch.zeros(1, S).pin_memory()) for _, wp, xp in parts]
    bad = pinned(parts[2][1])
    bad[0, 7, 11] = float("nan")
    for k, (wb, xb, ob) in enumerate(bufs):
        G.gw_stream_push_async(s, 1, (bad if k == 2 else wb).data_ptr(), xb.data_ptr(), ob.data_ptr(),
                               st.cuda_stream)
    # a synchronous push while pushes are pending is refused
    with pytest.raises(G.GwError) as e:
        G.gw_stream_push(s, 1, np.zeros((1, 21, S), np.float32), np.zeros((1, S), np.float32),
                         np.zeros((1, S), np.float32))
    assert e.value.code == G.GW_ESTATE
    with pytest.raises(G.GwError) as e:
        G.gw_stream_sync(s)
    assert e.value.code == G.GW_ENONFINITE and e.value.first_rejected == 2
    assert G.gw_stream_head(s) == 2 * S
    for k in (0, 1):
        assert np.array_equal(bufs[k][2].numpy(), ref[k])
    for k in range(2, n):
        wb, xb, ob = bufs[k]
        G.gw_stream_push_async(s, 1, wb.data_ptr(), xb.data_ptr(), ob.data_ptr(), st.cuda_stream)
    G.gw_stream_sync(s)
    assert G.gw_stream_head(s) == n * S
    for k in range(2, n):
        assert np.array_equal(bufs[k][2].numpy(), ref[k])


def test_async_pushes_on_two_cuda_streams_are_refused(ctx):
    m = ctx.deepclean(0, G.GW_BF16)
    W, S = 512, 64
    s = make_stream(ctx, m, W, S, 1)
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    wb, xb, ob = pinned(np.zeros((1, 21, S))), pinned(np.zeros((1, S))), torch.zeros(1, S).pin_memory()
    G.gw_stream_push_async(s, 1, wb.data_ptr(), xb.data_ptr(), ob.data_ptr(), a.cuda_stream)
    with pytest.raises(G.GwError) as e:
        G.gw_stream_push_async(s, 1, wb.data_ptr(), xb.data_ptr(), ob.data_ptr(), b.cuda_stream)
    assert e.value.code == G.GW_EINVAL
    G.gw_stream_sync(s)
    assert G.gw_stream_head(s) == S
    G.gw_stream_sync(s)  # nothing pending: returns at once
