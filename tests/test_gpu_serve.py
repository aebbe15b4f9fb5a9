"""Serving loop (continuous batching over many streams) against the FP64
end-to-end oracle of one stream (oracle/pipeline.py).

Each stream has two detectors; a snapshot runs DeepClean per detector,
subtraction + aggregation, 2x resampling, whitening and BBHnet.  Streams of
different strides are submitted interleaved, so ticks mix streams and batch
sizes vary.  Tolerances: FP32 path relative L2 <= 1e-5 on the predicted
noise (cleaned minus strain) and on the logits; BF16 path <= 2e-2 on the
predicted noise and logits within 0.05 absolute.

The logit bound is stated for BBHnet on whitened strain of about unit
variance.  A randomly initialised DeepClean predicts noise far larger than
the strain, which whitening then amplifies, so the BF16 end-to-end cases
scale its output layer (weights and bias, on both sides alike) by 1e-2 to
bring the prediction to the strain's scale, as a trained model's would be.
"""
import functools
import time

import numpy as np
import pytest

from oracle import fir as ofir, nets, pipeline, stream as ostream
from paper_2108_12430_gb300 import gwstream as G, synth
from tests.gpu_util import Ctx, rel_l2

pytestmark = pytest.mark.gpu
TOL32, TOL16, LOGIT16 = 1e-5, 2e-2, 0.05
C, FS, FS2 = 21, 4096.0, 2048.0
KF, FC = 127, 900.0
BBH_SEED = 9


@pytest.fixture
def ctx(gpu_lib):
    c = Ctx()
    yield c
    c.close()


def standardisation(d):
    r = np.random.default_rng(50 + d)
    return r.normal(0, 0.1, C).astype(np.float32), r.uniform(0.8, 1.25, C).astype(np.float32)


@functools.lru_cache(maxsize=None)
def stream_inputs(seed, S, n):
    """float32 witness [2][C][n S] and strain [2][n S] of one stream."""
    wit = np.stack([synth.witness_channels(seed + 7 * d, C, n * S) for d in range(2)])
    strn = np.stack([synth.coupled_strain(seed + 7 * d, wit[d]) for d in range(2)])
    return wit.astype(np.float32), strn.astype(np.float32)


def dc_params(d, out_scale):
    params = synth.deepclean_params(d + 1)
    if out_scale != 1.0:
        params[-1] = dict(params[-1])
        params[-1]["w"] = (params[-1]["w"] * np.float32(out_scale)).astype(np.float32)
        params[-1]["b"] = (params[-1]["b"] * np.float32(out_scale)).astype(np.float32)
    return params


@functools.lru_cache(maxsize=None)
def oracle_stream(seed, S, n, mode, delta, W, Lb, Kh, nfft, out_scale, post_k=0):
    wit, strn = stream_inputs(seed, S, n)
    fwd = []
    for d in range(2):
        params = dc_params(d, out_scale)
        mean, std = standardisation(d)
        fwd.append(lambda w, p=params, m=mean.astype(np.float64), s=std.astype(np.float64):
                   nets.deepclean_forward(w, p, synth.DEEPCLEAN_LAYERS, m, s))
    f_dec = ofir.lowpass_fir(KF, FC, FS)
    _, psd = synth.psd_grid(FS2, nfft)
    h = ofir.whitening_fir(psd, FS2, nfft, Kh)
    params, head = synth.bbhnet_params(BBH_SEED)
    cl, logits = pipeline.run_pipeline([wit[d].astype(np.float64) for d in range(2)],
                                       [strn[d].astype(np.float64) for d in range(2)], W, S, n, mode, delta, fwd,
                                       f_dec, h, params, head, synth.bbhnet_layers(), Lb=Lb,
                                       post=post_taps(post_k) if post_k else None)
    return cl, logits


def post_taps(K):
    """The 55-65 Hz post-processing band-pass, designed by the oracle and
    rounded to float32 as the library stores its taps."""
    return ofir.bandpass_fir(FS, 8192, K).astype(np.float32).astype(np.float64)


class Rig:
    """Models, FIRs and a server on one context."""

    def __init__(self, ctx, prec, *, W=2048, max_stride=512, max_streams=8, max_batch=8, mode=G.GW_AGG_AVERAGE,
                 delta=512, Lb=512, Kh=257, nfft=512, bbh_prec=None, out_scale=1.0, post_k=0, **kw):
        self.ctx, self.W, self.mode, self.delta, self.Lb, self.Kh, self.nfft = ctx, W, mode, delta, Lb, Kh, nfft
        self.prec, self.out_scale, self.post_k = prec, out_scale, post_k
        self.c = (post_k - 1) // 2 if post_k else 0
        self.dc = []
        for d in range(2):
            mean, std = standardisation(d)
            m = G.gw_model_create(ctx.h, G.GW_MODEL_DEEPCLEAN, prec, C, synth.flatten_params(dc_params(d, out_scale)),
                                  mean, std)
            ctx.objs.append((G.gw_model_destroy, m))
            self.dc.append(m)
        self.bbh = ctx.bbhnet(BBH_SEED, prec if bbh_prec is None else bbh_prec)
        self.fdec = G.gw_fir_create_lowpass(ctx.h, FC, FS, KF)
        ctx.objs.append((G.gw_fir_destroy, self.fdec))
        _, psd = synth.psd_grid(FS2, nfft)
        self.fw = G.gw_fir_create_whitening(ctx.h, psd, FS2, Kh)
        ctx.objs.append((G.gw_fir_destroy, self.fw))
        self.kw = dict(n_det=2, n_witness=C, window=W, max_stride=max_stride, max_streams=max_streams,
                       max_batch=max_batch, agg_mode=mode, agg_delay=delta, bbh_len=Lb)
        self.kw.update(kw)
        if post_k:
            self.fpost = G.gw_fir_create_bandpass(ctx.h, FS, 8192, post_k)
            ctx.objs.append((G.gw_fir_destroy, self.fpost))
            self.kw["post"] = self.fpost
        self.s = G.gw_server_create(ctx.h, self.dc, self.bbh, self.fdec, self.fw, **self.kw)
        ctx.objs.append((G.gw_server_destroy, self.s))

    def run(self, streams, order):
        """streams: list of (seed, S, n); order: stream index per submission.
        Submits everything without waiting, then waits; returns per stream
        (cleaned [2][n][S], logits [n])."""
        sids = [G.gw_server_open(self.s, S) for _, S, _ in streams]
        outs = [(np.zeros((n, 2, S), np.float32), np.zeros((n, 1), np.float32)) for _, S, n in streams]
        ins = [stream_inputs(seed, S, n) for seed, S, n in streams]
        keep, tickets = [], []
        k_next = [0] * len(streams)
        for i in order:
            seed, S, n = streams[i]
            k = k_next[i]
            k_next[i] += 1
            wit, strn = ins[i]
            w = np.ascontiguousarray(wit[:, :, k * S:(k + 1) * S])
            x = np.ascontiguousarray(strn[:, k * S:(k + 1) * S])
            keep.append((w, x))
            tickets.append(G.gw_server_submit(self.s, sids[i], w, x, outs[i][0][k], outs[i][1][k]))
        for t in tickets:
            G.gw_server_wait(self.s, t, 60_000_000)
        for sid in sids:
            G.gw_server_close(self.s, sid)
        return [(o[0].transpose(1, 0, 2), o[1][:, 0]) for o in outs]

    def oracle(self, seed, S, n):
        return oracle_stream(seed, S, n, self.mode, self.delta, self.W, self.Lb, self.Kh, self.nfft, self.out_scale,
                             self.post_k)


def interleaved(streams, seed=0):
    r = np.random.default_rng(seed)
    order = [i for i, (_, _, n) in enumerate(streams) for _ in range(n)]
    r.shuffle(order)
    return order


def strain_emitted(seed, S, n, delta, c=0):
    _, strn = stream_inputs(seed, S, n)
    out = np.zeros((2, n, S))
    for k in range(n):
        t = ostream.emit_times(k, S, delta) - c
        ok = t >= 0
        out[:, k, ok] = strn[:, t[ok]]
    return out


def check(rig, streams, got, tol, logit_check):
    for (seed, S, n), (cl, lg) in zip(streams, got):
        ref_cl, ref_lg = rig.oracle(seed, S, n)
        st = strain_emitted(seed, S, n, rig.delta, rig.c)
        err = rel_l2(cl - st, ref_cl - st)
        print(f"stream seed={seed} S={S}: noise rel-L2 {err:.2e}, logit max abs err {np.abs(lg - ref_lg).max():.2e}"
              f" (|logit| <= {np.abs(ref_lg).max():.2f})")
        assert err <= tol
        assert np.isfinite(lg).all()
        logit_check(lg, ref_lg)


STREAMS = [(100, 256, 26), (200, 128, 44), (300, 512, 14)]


def test_lowpass_design_matches_oracle(ctx):
    f = G.gw_fir_create_lowpass(ctx.h, FC, FS, KF)
    ctx.objs.append((G.gw_fir_destroy, f))
    np.testing.assert_allclose(G.gw_fir_taps(f), ofir.lowpass_fir(KF, FC, FS), rtol=0, atol=1e-13)


def test_server_matches_oracle_fp32(ctx):
    rig = Rig(ctx, G.GW_FP32)
    got = rig.run(STREAMS, interleaved(STREAMS))
    check(rig, STREAMS, got, TOL32, lambda g, r: rel_l2(g, r) <= TOL32 or pytest.fail(f"logit rel-L2 {rel_l2(g, r)}"))
    st = G.gw_server_stats_read(rig.s)
    assert st["snapshots"] == sum(n for _, _, n in STREAMS)
    assert st["ticks"] >= max(n for _, _, n in STREAMS)
    assert st["mean_batch"] > 1.0  # ticks really mixed streams
    assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"]


def test_server_matches_oracle_bf16(ctx):
    rig = Rig(ctx, G.GW_BF16, out_scale=1e-2)
    got = rig.run(STREAMS, interleaved(STREAMS, 1))

    def logits_ok(g, r):
        assert np.abs(g - r).max() <= LOGIT16

    check(rig, STREAMS, got, TOL16, logits_ok)


def test_server_bf16_unscaled_network(ctx):
    # BF16 with DeepClean exactly as created (no output scaling): the
    # predicted noise is held to the BF16 bound; the logits, of whitened data
    # that a random network's prediction dominates, only have to be finite
    rig = Rig(ctx, G.GW_BF16)
    got = rig.run(STREAMS, interleaved(STREAMS, 4))
    check(rig, STREAMS, got, TOL16, lambda g, r: None)


POST_STREAMS = [(110, 256, 16), (310, 512, 10)]


def test_server_post_processing_fp32(ctx):
    # the 55-65 Hz band-pass of the aggregated prediction before subtraction
    # (2049 taps: c = 1024 samples of delay), against the oracle pipeline with
    # the same post-processing
    rig = Rig(ctx, G.GW_FP32, post_k=2049)
    got = rig.run(POST_STREAMS, interleaved(POST_STREAMS, 5))
    check(rig, POST_STREAMS, got, TOL32,
          lambda g, r: rel_l2(g, r) <= TOL32 or pytest.fail(f"logit rel-L2 {rel_l2(g, r)}"))


def test_server_post_processing_bf16(ctx):
    rig = Rig(ctx, G.GW_BF16, out_scale=1e-2, post_k=2049)
    got = rig.run(POST_STREAMS, interleaved(POST_STREAMS, 6))
    check(rig, POST_STREAMS, got, TOL16, lambda g, r: np.abs(g - r).max() <= LOGIT16 or pytest.fail("logits"))


@pytest.mark.parametrize("prec", [G.GW_FP32, G.GW_BF16])
def test_same_result_alone_and_in_the_mix(ctx, prec):
    # A stream's results do not depend on which other streams share its ticks,
    # their number, or the batch bucket: run alone, then interleaved with two
    # streams of other strides, with a smaller max_batch so that buckets vary.
    x = [(100, 256, 26)]
    alone = Rig(ctx, prec).run(x, [0] * 26)[0]
    mix = x + [(400, 128, 40), (500, 512, 12)]
    mixed = Rig(ctx, prec, max_batch=2).run(mix, interleaved(mix, 7))[0]
    d_cl = np.abs(alone[0] - mixed[0]).max()
    d_lg = np.abs(alone[1] - mixed[1]).max()
    print("alone vs mix max abs diff: cleaned", d_cl, "logits", d_lg)
    assert d_cl == 0.0 and d_lg == 0.0


def test_graphs_and_eager_launches_agree(ctx):
    s = [(100, 256, 26), (300, 512, 14)]
    order = interleaved(s, 3)
    a = Rig(ctx, G.GW_BF16, use_graphs=1).run(s, order)
    b = Rig(ctx, G.GW_BF16, use_graphs=0).run(s, order)
    for (ca, la), (cb, lb) in zip(a, b):
        assert np.array_equal(ca, cb) and np.array_equal(la, lb)


def test_latest_mode_and_full_size_window_bf16(ctx):
    # The serving configuration's window (8 s at 4096 Hz) and whitening filter
    # (2049 taps at 2048 Hz, 1 s BBHnet input), causal LATEST aggregation.
    streams = [(600, 512, 3), (700, 256, 4)]
    rig = Rig(ctx, G.GW_BF16, W=32768, mode=G.GW_AGG_LATEST, delta=0, Lb=2048, Kh=2049, nfft=8192, out_scale=1e-2)
    got = rig.run(streams, interleaved(streams, 2))
    check(rig, streams, got, TOL16, lambda g, r: np.abs(g - r).max() <= LOGIT16 or pytest.fail("logits"))


def test_admission_by_hbm_budget(ctx):
    probe = Rig(ctx, G.GW_BF16)
    per_stream = G.gw_server_stream_bytes(probe.s, 256)
    assert per_stream > 0
    base = G.gw_ctx_bytes_in_use(ctx.h)
    small = Ctx(budget=base + int(2.5 * per_stream))
    try:
        rig = Rig(small, G.GW_BF16)
        assert G.gw_ctx_bytes_in_use(small.h) == base
        a = G.gw_server_open(rig.s, 256)
        b = G.gw_server_open(rig.s, 128)
        with pytest.raises(G.GwError) as e:
            G.gw_server_open(rig.s, 512)
        assert e.value.code == G.GW_EBUDGET
        assert G.gw_ctx_bytes_in_use(small.h) == base + 2 * per_stream
        G.gw_server_close(rig.s, a)
        c = G.gw_server_open(rig.s, 512)  # admitted once memory is free
        G.gw_server_close(rig.s, b)
        G.gw_server_close(rig.s, c)
        assert G.gw_ctx_bytes_in_use(small.h) == base
    finally:
        small.close()


def test_wait_timeout_and_batching_window(ctx):
    # With a 1.5 s batching window and room for 4 snapshots, a lone snapshot
    # waits for the window to close: a short wait times out, a long one
    # returns, and the result matches the same snapshot served at once.
    rig = Rig(ctx, G.GW_FP32, max_batch=4, max_wait_us=1_500_000)
    sid = G.gw_server_open(rig.s, 256)
    wit, strn = stream_inputs(100, 256, 26)
    w = np.ascontiguousarray(wit[:, :, :256])
    x = np.ascontiguousarray(strn[:, :256])
    out = np.zeros((2, 256), np.float32)
    score = np.zeros(1, np.float32)
    t0 = time.perf_counter()
    t = G.gw_server_submit(rig.s, sid, w, x, out, score)
    with pytest.raises(G.GwError) as e:
        G.gw_server_wait(rig.s, t, 1000)
    assert e.value.code == G.GW_ETIMEOUT
    G.gw_server_wait(rig.s, t, -1)
    assert time.perf_counter() - t0 >= 1.3
    ref = Rig(ctx, G.GW_FP32).run([(100, 256, 1)], [0])[0]
    assert np.array_equal(out, ref[0][:, 0]) and score[0] == ref[1][0]
    G.gw_server_close(rig.s, sid)


def test_replay_matches_submit_and_reports_latency(ctx):
    streams = [(100, 256, 26), (300, 512, 14)]
    order = interleaved(streams, 5)
    ref = Rig(ctx, G.GW_BF16).run(streams, order)
    rig = Rig(ctx, G.GW_BF16)
    sids = [G.gw_server_open(rig.s, S) for _, S, _ in streams]
    r = np.random.default_rng(0)
    t_us = np.cumsum(r.exponential(200.0, len(order)))
    wit, strn, clean, k_next = [], [], [], [0, 0]
    for i in order:
        seed, S, n = streams[i]
        k = k_next[i]
        k_next[i] += 1
        wv, sv = stream_inputs(seed, S, n)
        wit.append(np.ascontiguousarray(wv[:, :, k * S:(k + 1) * S]))
        strn.append(np.ascontiguousarray(sv[:, k * S:(k + 1) * S]))
        clean.append(np.zeros((2, S), np.float32))
    score = np.zeros(len(order), np.float32)
    lat = np.zeros(len(order))
    G.gw_server_replay(rig.s, [sids[i] for i in order], t_us, wit, strn, clean, score, lat)
    assert (lat > 0).all()
    k_next = [0, 0]
    for j, i in enumerate(order):
        k = k_next[i]
        k_next[i] += 1
        assert np.array_equal(clean[j], ref[i][0][:, k]) and score[j] == ref[i][1][k]
    st = G.gw_server_stats_read(rig.s, reset=True)
    assert st["snapshots"] == len(order) and st["p50_us"] <= st["p99_us"]
    # the slowest request's time is bounded by what its parts can add up to:
    # it waited for a launch, then for at most the in-flight ticks and its own
    assert 0 < st["max_tick_device_us"] and 0 <= st["max_launch_wait_us"] <= st["max_us"]
    assert 0 <= st["max_submit_late_us"] < st["busy_s"] * 1e6 and 0 < st["max_launch_call_us"]
    st0 = G.gw_server_stats_read(rig.s)
    assert st0["snapshots"] == 0 and st0["max_tick_device_us"] == st0["max_launch_wait_us"] == 0
    assert st0["max_submit_late_us"] == st0["max_launch_call_us"] == 0


def test_non_finite_snapshot_is_refused(ctx):
    rig = Rig(ctx, G.GW_FP32)
    sid = G.gw_server_open(rig.s, 256)
    wit, strn = stream_inputs(100, 256, 26)
    w = np.ascontiguousarray(wit[:, :, :256])
    w[1, 3, 17] = np.nan
    x = np.ascontiguousarray(strn[:, :256])
    out = np.zeros((2, 256), np.float32)
    with pytest.raises(G.GwError) as e:
        G.gw_server_submit(rig.s, sid, w, x, out)
    assert e.value.code == G.GW_ENONFINITE
    # nothing was queued: the stream still starts at snapshot 0
    w = np.ascontiguousarray(wit[:, :, :256])
    t = G.gw_server_submit(rig.s, sid, w, x, out)
    G.gw_server_wait(rig.s, t, 60_000_000)
    ref = Rig(ctx, G.GW_FP32).run([(100, 256, 1)], [0])[0]
    assert np.array_equal(out, ref[0][:, 0])
    G.gw_server_close(rig.s, sid)


def test_server_argument_errors(ctx):
    rig = Rig(ctx, G.GW_BF16, max_streams=2, max_batch=2)
    for bad in (200, 1024, 4):  # not dividing the window / above max_stride / not a multiple of 8
        with pytest.raises(G.GwError) as e:
            G.gw_server_open(rig.s, bad)
        assert e.value.code == G.GW_EINVAL
    a = G.gw_server_open(rig.s, 256)
    b = G.gw_server_open(rig.s, 256)
    with pytest.raises(G.GwError) as e:
        G.gw_server_open(rig.s, 256)
    assert e.value.code == G.GW_ESTATE
    with pytest.raises(G.GwError) as e:
        G.gw_server_wait(rig.s, 12345, 0)
    assert e.value.code == G.GW_EINVAL
    G.gw_server_close(rig.s, a)
    G.gw_server_close(rig.s, b)
    with pytest.raises(G.GwError) as e:
        G.gw_server_close(rig.s, a)
    assert e.value.code == G.GW_EINVAL
    with pytest.raises(G.GwError):
        G.gw_server_create(ctx.h, rig.dc, rig.bbh, rig.fdec, rig.fw, n_det=2, n_witness=C, window=2048,
                           max_stride=512, max_streams=4, max_batch=8, agg_delay=0)  # max_batch > max_streams
