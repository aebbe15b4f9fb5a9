"""Thin ctypes binding of ``libgwstream.so`` (include/gwstream.h).

Argument marshalling only: every function keeps the C name, converts Python
ints/arrays to C types, raises ``GwError`` on a negative status and returns
out-parameters.  No compute happens here.  Device buffers are passed as
integer addresses (e.g. ``torch.Tensor.data_ptr()``), CUDA streams as the
integer handle ``torch.cuda.Stream.cuda_stream`` (0 = default stream).

The library must have been built (``paper_2108_12430_gb300.build.build()``,
which ``__graft_entry__.build()`` calls); there is no fallback if it is
missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgwstream.so")

GW_OK, GW_EINVAL, GW_EBUDGET, GW_ENOMEM, GW_ECUDA, GW_ETIMEOUT, GW_ESTATE, GW_ENOTIMPL, GW_ENONFINITE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
GW_FP32, GW_BF16, GW_FP8 = 0, 1, 2
GW_MODEL_DEEPCLEAN, GW_MODEL_BBHNET = 0, 1
GW_AGG_LATEST, GW_AGG_AVERAGE = 0, 1
GW_MEM_HOST, GW_MEM_DEVICE = 0, 1

ERROR_NAMES = {GW_EINVAL: "GW_EINVAL", GW_EBUDGET: "GW_EBUDGET", GW_ENOMEM: "GW_ENOMEM", GW_ECUDA: "GW_ECUDA",
               GW_ETIMEOUT: "GW_ETIMEOUT", GW_ESTATE: "GW_ESTATE", GW_ENOTIMPL: "GW_ENOTIMPL",
               GW_ENONFINITE: "GW_ENONFINITE"}

# Every symbol include/gwstream.h declares (checked by the CPU tests).
EXPORTS = (
    "gw_last_error", "gw_version", "gw_ctx_create", "gw_ctx_destroy", "gw_ctx_bytes_in_use",
    "gw_model_param_count", "gw_model_create", "gw_model_destroy", "gw_deepclean_forward", "gw_bbhnet_score",
    "gw_fir_create_whitening", "gw_fir_destroy", "gw_fir_ntaps", "gw_fir_taps", "gw_whiten",
    "gw_stream_create", "gw_stream_destroy", "gw_stream_push", "gw_stream_push_async", "gw_stream_sync",
    "gw_stream_head", "gw_stream_status",
    "gw_profile_enable", "gw_profile_read", "gw_launch_count", "gw_alloc_count", "gw_deepclean_forward_noalloc",
    "gw_model_status", "gw_tc_inspect", "gw_fir_create_lowpass",
    "gw_server_create", "gw_server_open", "gw_server_close", "gw_server_stream_bytes", "gw_server_submit",
    "gw_server_wait", "gw_server_stats_read", "gw_server_replay", "gw_server_destroy",
    "gw_trainer_create", "gw_trainer_destroy", "gw_trainer_status", "gw_trainer_param_count", "gw_trainer_bytes", "gw_trainer_forward",
    "gw_trainer_backward", "gw_fir_create_band_loss", "gw_band_loss", "gw_band_loss_backward", "gw_fir_backward",
    "gw_adam_step", "gw_adam_step_dev", "gw_model_calibrate", "gw_model_test_wait_timeout", "gw_fir_create_bandpass",
    "gw_scored_stream_create", "gw_scored_stream_push", "gw_scored_stream_wait", "gw_scored_stream_destroy",
    "gw_partition_streams",
)


class GwError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class gw_model_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("precision", C.c_int), ("n_in", C.c_int),
                ("params", C.POINTER(C.c_float)), ("n_params", C.c_size_t),
                ("in_mean", C.POINTER(C.c_float)), ("in_std", C.POINTER(C.c_float)),
                ("act_scales", C.POINTER(C.c_float)), ("n_act_scales", C.c_int)]


class gw_stream_desc(C.Structure):
    _fields_ = [("n_det", C.c_int), ("n_witness", C.c_int), ("window", C.c_int), ("stride", C.c_int),
                ("max_batch", C.c_int), ("agg_mode", C.c_int), ("agg_delay", C.c_int), ("post", C.c_void_p)]


class gw_server_desc(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("n_det", "n_witness", "window", "max_stride", "max_streams", "max_batch",
                                        "max_pending", "agg_mode", "agg_delay", "bbh_len", "max_wait_us",
                                        "max_inflight", "use_graphs", "form_lead_us")] + [("post", C.c_void_p)]


class gw_server_stats(C.Structure):
    _fields_ = [("snapshots", C.c_int64), ("ticks", C.c_int64), ("kernels", C.c_int64), ("mean_batch", C.c_double),
                ("p50_us", C.c_double), ("p99_us", C.c_double), ("mean_us", C.c_double), ("max_us", C.c_double),
                ("busy_s", C.c_double), ("max_tick_device_us", C.c_double), ("max_launch_wait_us", C.c_double),
                ("max_submit_late_us", C.c_double), ("max_launch_call_us", C.c_double)]


class gw_trainer_desc(C.Structure):
    _fields_ = [("n_in", C.c_int), ("max_batch", C.c_int), ("length", C.c_int), ("checkpoint", C.c_int),
                ("precision", C.c_int), ("tc_data", C.c_int)]


_lib = None
P = C.c_void_p
I = C.c_int
I64 = C.c_int64
SZ = C.c_size_t


def _declare(lib):
    sig = {
        "gw_last_error": (C.c_char_p, []),
        "gw_version": (C.c_char_p, []),
        "gw_ctx_create": (I, [I, SZ, C.POINTER(P)]),
        "gw_ctx_destroy": (I, [P]),
        "gw_ctx_bytes_in_use": (SZ, [P]),
        "gw_model_param_count": (SZ, [I, I]),
        "gw_model_create": (I, [P, C.POINTER(gw_model_desc), C.POINTER(P)]),
        "gw_model_destroy": (I, [P]),
        "gw_deepclean_forward": (I, [P, P, I64, I64, I, I, P, P]),
        "gw_bbhnet_score": (I, [P, P, I, I, P, P]),
        "gw_fir_create_whitening": (I, [P, C.POINTER(C.c_double), I, C.c_double, I, I, C.POINTER(P)]),
        "gw_fir_destroy": (I, [P]),
        "gw_fir_ntaps": (I, [P]),
        "gw_fir_taps": (I, [P, C.POINTER(C.c_double)]),
        "gw_whiten": (I, [P, P, I, I, I, P, P]),
        "gw_stream_create": (I, [P, C.POINTER(gw_stream_desc), C.POINTER(P), C.POINTER(P)]),
        "gw_stream_destroy": (I, [P]),
        "gw_stream_push": (I, [P, I, P, P, P, I, P]),
        "gw_stream_push_async": (I, [P, I, P, P, P, P]),
        "gw_stream_sync": (I, [P, C.POINTER(I)]),
        "gw_stream_head": (I64, [P]),
        "gw_stream_status": (I, [P, P]),
        "gw_profile_enable": (I, [I]),
        "gw_profile_read": (I, [C.c_char_p, SZ, C.POINTER(C.c_double), C.POINTER(C.c_int64), I]),
        "gw_launch_count": (I64, []),
        "gw_alloc_count": (I64, []),
        "gw_deepclean_forward_noalloc": (I, [P, P, I64, I64, I, I, P, P]),
        "gw_model_status": (I, [P, P]),
        "gw_model_test_wait_timeout": (I, [P, C.POINTER(C.c_int), P]),
        "gw_tc_inspect": (I, [C.POINTER(C.c_int), I, C.POINTER(C.c_double), I, I, I, I, P, SZ,
                              C.POINTER(C.c_uint32), I, C.POINTER(C.c_int)]),
        "gw_fir_create_lowpass": (I, [P, C.c_double, C.c_double, I, I, C.POINTER(P)]),
        "gw_server_create": (I, [P, C.POINTER(gw_server_desc), C.POINTER(P), P, P, P, C.POINTER(P)]),
        "gw_server_open": (I, [P, I, C.POINTER(I)]),
        "gw_server_close": (I, [P, I]),
        "gw_server_stream_bytes": (I64, [P, I]),
        "gw_server_submit": (I, [P, I, P, P, P, P, C.POINTER(C.c_uint64)]),
        "gw_server_wait": (I, [P, C.c_uint64, I64]),
        "gw_server_stats_read": (I, [P, I, C.POINTER(gw_server_stats)]),
        "gw_server_replay": (I, [P, I, P, P, P, P, P, P, P]),
        "gw_server_destroy": (I, [P]),
        "gw_trainer_create": (I, [P, C.POINTER(gw_trainer_desc), P, P, C.POINTER(P)]),
        "gw_trainer_destroy": (I, [P]),
        "gw_trainer_status": (I, [P, P]),
        "gw_trainer_param_count": (I64, [P]),
        "gw_trainer_bytes": (I64, [P]),
        "gw_trainer_forward": (I, [P, P, P, I, P, P]),
        "gw_trainer_backward": (I, [P, P, P, P]),
        "gw_fir_create_bandpass": (I, [P, C.c_double, I, I, C.c_double, C.c_double, C.c_double, I, C.POINTER(P)]),
        "gw_fir_create_band_loss": (I, [P, C.POINTER(C.c_double), I, C.c_double, I, C.c_double, C.c_double,
                                        C.c_double, C.c_double, I, C.POINTER(P)]),
        "gw_band_loss": (I, [P, P, P, I, I, P, P, P]),
        "gw_band_loss_backward": (I, [P, P, I, I, P, P, P]),
        "gw_fir_backward": (I, [P, P, I, I, I, P, P]),
        "gw_adam_step": (I, [P, P, P, P, I64, I, C.c_float, C.c_float, C.c_float, C.c_float, P]),
        "gw_adam_step_dev": (I, [P, P, P, P, I64, P, C.c_float, C.c_float, C.c_float, C.c_float, P]),
        "gw_model_calibrate": (I, [P, P, I, I, C.c_float, P, P]),
        "gw_scored_stream_create": (I, [P, C.POINTER(P), P, P, P, I, I, I, I, I, I, I, I, C.POINTER(P)]),
        "gw_scored_stream_push": (I, [P, P, P, P, P, C.POINTER(C.c_uint64)]),
        "gw_scored_stream_wait": (I, [P, C.c_uint64, I64]),
        "gw_scored_stream_destroy": (I, [P]),
        "gw_partition_streams": (I, [I, C.POINTER(C.c_int), C.POINTER(C.c_int64), I, C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def lib():
    """Load the library (built in-tree); raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2108_12430_gb300.build.build() first")
        l = C.CDLL(LIB_PATH)
        _declare(l)
        _lib = l
    return _lib


def _check(rc):
    if rc < 0:
        raise GwError(rc, lib().gw_last_error().decode())
    return rc


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float)) if a is not None else None


# ---- C-ABI mirrors -----------------------------------------------------------

def gw_version():
    return lib().gw_version().decode()


def gw_ctx_create(device=0, hbm_budget_bytes=0):
    h = P()
    _check(lib().gw_ctx_create(device, hbm_budget_bytes, C.byref(h)))
    return h


def gw_ctx_destroy(ctx):
    _check(lib().gw_ctx_destroy(ctx))


def gw_ctx_bytes_in_use(ctx):
    return lib().gw_ctx_bytes_in_use(ctx)


def gw_model_param_count(kind, n_in):
    return lib().gw_model_param_count(kind, n_in)


def gw_model_create(ctx, kind, precision, n_in, params, in_mean=None, in_std=None, act_scales=None):
    params = np.ascontiguousarray(params, np.float32)
    keep = [params]
    d = gw_model_desc()
    d.kind, d.precision, d.n_in = kind, precision, n_in
    d.params, d.n_params = _fptr(params), params.size
    if in_mean is not None:
        in_mean = np.ascontiguousarray(in_mean, np.float32); keep.append(in_mean)
    if in_std is not None:
        in_std = np.ascontiguousarray(in_std, np.float32); keep.append(in_std)
    d.in_mean, d.in_std = _fptr(in_mean), _fptr(in_std)
    if act_scales is not None:
        act_scales = np.ascontiguousarray(act_scales, np.float32); keep.append(act_scales)
        d.act_scales, d.n_act_scales = _fptr(act_scales), act_scales.size
    h = P()
    _check(lib().gw_model_create(ctx, C.byref(d), C.byref(h)))
    return h


def gw_model_destroy(m):
    _check(lib().gw_model_destroy(m))


def gw_model_status(m, stream=0):
    _check(lib().gw_model_status(m, stream or None))


def gw_model_test_wait_timeout(m, stream=0):
    """Runs the bounded-wait failure test; returns the status the host observed
    for the stalled launch (raises if the follow-up normal launch fails)."""
    obs = C.c_int(0)
    _check(lib().gw_model_test_wait_timeout(m, C.byref(obs), stream or None))
    return obs.value


def gw_deepclean_forward(m, x_ptr, ld, window_stride, B, L, y_ptr, stream=0):
    _check(lib().gw_deepclean_forward(m, x_ptr, ld, window_stride, B, L, y_ptr, stream or None))


def gw_deepclean_forward_noalloc(m, x_ptr, ld, window_stride, B, L, y_ptr, stream=0):
    _check(lib().gw_deepclean_forward_noalloc(m, x_ptr, ld, window_stride, B, L, y_ptr, stream or None))


def gw_model_calibrate(m, x_ptr, B, L, headroom=1.0, stream=0):
    """Sets an FP8 BBHnet's activation scales from a calibration batch; returns them."""
    n = 14
    out = np.zeros(n, np.float32)
    _check(lib().gw_model_calibrate(m, x_ptr, B, L, headroom, out.ctypes.data, stream or None))
    return out


def gw_bbhnet_score(m, x_ptr, B, L, logits_ptr, stream=0):
    _check(lib().gw_bbhnet_score(m, x_ptr, B, L, logits_ptr, stream or None))


def gw_fir_create_whitening(ctx, psd, fs, ntaps, precision=GW_FP32):
    psd = np.ascontiguousarray(psd, np.float64)
    h = P()
    _check(lib().gw_fir_create_whitening(ctx, psd.ctypes.data_as(C.POINTER(C.c_double)), psd.size, fs, ntaps,
                                         precision, C.byref(h)))
    return h


def gw_fir_create_lowpass(ctx, fc, fs, ntaps, precision=GW_FP32):
    h = P()
    _check(lib().gw_fir_create_lowpass(ctx, fc, fs, ntaps, precision, C.byref(h)))
    return h


def gw_fir_destroy(f):
    _check(lib().gw_fir_destroy(f))


def gw_fir_ntaps(f):
    return _check(lib().gw_fir_ntaps(f))


def gw_fir_taps(f):
    out = np.zeros(gw_fir_ntaps(f), np.float64)
    _check(lib().gw_fir_taps(f, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def gw_whiten(f, x_ptr, B, Cc, L_in, y_ptr, stream=0):
    _check(lib().gw_whiten(f, x_ptr, B, Cc, L_in, y_ptr, stream or None))


def gw_stream_create(ctx, models, n_det, n_witness, window, stride, max_batch, agg_mode, agg_delay, post=None):
    d = gw_stream_desc(n_det, n_witness, window, stride, max_batch, agg_mode, agg_delay, post)
    arr = (P * 2)(*(list(models) + [None] * (2 - len(models))))
    h = P()
    _check(lib().gw_stream_create(ctx, C.byref(d), arr, C.byref(h)))
    return h


def gw_stream_destroy(s):
    _check(lib().gw_stream_destroy(s))


def gw_stream_push(s, n_snap, witness, strain, clean_out, mem=GW_MEM_HOST, stream=0):
    """Host mode: numpy float32 arrays; device mode: integer device addresses."""
    if mem == GW_MEM_HOST:
        for a in (witness, strain, clean_out):
            assert a.dtype == np.float32 and a.flags.c_contiguous
        args = (witness.ctypes.data, strain.ctypes.data, clean_out.ctypes.data)
    else:
        args = (witness, strain, clean_out)
    _check(lib().gw_stream_push(s, n_snap, args[0], args[1], args[2], mem, stream or None))


GW_STREAM_MAX_PENDING = 1024


def gw_stream_push_async(s, n_snap, witness, strain, clean_out, stream=0):
    """Queues a host-buffer push; the buffers are host addresses (ints) of
    page-locked memory, or C-contiguous float32 numpy arrays (kept alive and
    unmodified by the caller until gw_stream_sync)."""
    ptrs = []
    for a in (witness, strain, clean_out):
        if isinstance(a, np.ndarray):
            assert a.dtype == np.float32 and a.flags.c_contiguous
            a = a.ctypes.data
        ptrs.append(a)
    _check(lib().gw_stream_push_async(s, n_snap, ptrs[0], ptrs[1], ptrs[2], stream or None))


def gw_stream_sync(s):
    """Waits for the queued pushes.  A push with a non-finite sample raises
    GwError(GW_ENONFINITE) whose first_rejected is its index among them."""
    k = I(-1)
    rc = lib().gw_stream_sync(s, C.byref(k))
    if rc < 0:
        e = GwError(rc, lib().gw_last_error().decode())
        e.first_rejected = k.value
        raise e


def gw_stream_head(s):
    return lib().gw_stream_head(s)


def gw_stream_status(s, stream=0):
    return lib().gw_stream_status(s, stream or None)


def gw_server_create(ctx, deepclean, bbhnet, decimator, whitening, *, n_det, n_witness, window, max_stride,
                     max_streams, max_batch, max_pending=0, agg_mode=GW_AGG_AVERAGE, agg_delay=0, bbh_len=2048,
                     max_wait_us=0, max_inflight=2, use_graphs=1, form_lead_us=0, post=None):
    d = gw_server_desc(n_det, n_witness, window, max_stride, max_streams, max_batch,
                       max_pending or 4 * max_batch, agg_mode, agg_delay, bbh_len, max_wait_us, max_inflight,
                       use_graphs, form_lead_us, post)
    arr = (P * 2)(*(list(deepclean) + [None] * (2 - len(deepclean))))
    h = P()
    _check(lib().gw_server_create(ctx, C.byref(d), arr, bbhnet, decimator, whitening, C.byref(h)))
    return h


def gw_server_open(s, stride):
    sid = I()
    _check(lib().gw_server_open(s, stride, C.byref(sid)))
    return sid.value


def gw_server_close(s, sid):
    _check(lib().gw_server_close(s, sid))


def gw_server_stream_bytes(s, stride):
    return _check(lib().gw_server_stream_bytes(s, stride))


def gw_server_submit(s, sid, witness, strain, clean_out, score_out=None):
    """witness [n_det][C][S], strain [n_det][S], clean_out [n_det][S], score_out [1]: float32 numpy arrays that
    must stay alive until gw_server_wait returns for the ticket."""
    for a in (witness, strain, clean_out) + ((score_out,) if score_out is not None else ()):
        assert a.dtype == np.float32 and a.flags.c_contiguous
    t = C.c_uint64()
    _check(lib().gw_server_submit(s, sid, witness.ctypes.data, strain.ctypes.data, clean_out.ctypes.data,
                                  score_out.ctypes.data if score_out is not None else None, C.byref(t)))
    return t.value


def gw_scored_stream_create(ctx, deepclean, bbhnet, decimator, whitening, n_witness, window, stride, agg_mode,
                            agg_delay, bbh_len, max_pending=64):
    dcs = (P * len(deepclean))(*deepclean)
    out = P()
    _check(lib().gw_scored_stream_create(ctx, dcs, bbhnet, decimator, whitening, len(deepclean), n_witness, window,
                                         stride, agg_mode, agg_delay, bbh_len, max_pending, C.byref(out)))
    return out


def gw_scored_stream_push(s, witness, strain, clean_out, score_out):
    """witness [n_det][C][S], strain [n_det][S], clean_out [n_det][S], score_out [1]: float32 numpy arrays that
    must stay alive until gw_scored_stream_wait returns for the ticket."""
    for a in (witness, strain, clean_out, score_out):
        assert a.dtype == np.float32 and a.flags.c_contiguous
    t = C.c_uint64()
    _check(lib().gw_scored_stream_push(s, witness.ctypes.data, strain.ctypes.data, clean_out.ctypes.data,
                                       score_out.ctypes.data, C.byref(t)))
    return t.value


def gw_scored_stream_wait(s, ticket, timeout_us=-1):
    _check(lib().gw_scored_stream_wait(s, ticket, timeout_us))


def gw_scored_stream_destroy(s):
    _check(lib().gw_scored_stream_destroy(s))


def gw_partition_streams(strides, bytes_, budgets, current=None, check=True):
    """Placement of streams on devices (host only): returns (status, device per stream, load per device)."""
    strides = np.ascontiguousarray(strides, np.int32)
    bytes_ = np.ascontiguousarray(bytes_, np.int64)
    budgets = np.ascontiguousarray(budgets, np.int64)
    n, nd = strides.size, budgets.size
    out = np.zeros(n, np.int32)
    load = np.zeros(nd, np.float64)
    cur = None if current is None else np.ascontiguousarray(current, np.int32)
    ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
    rc = lib().gw_partition_streams(n, ip(strides), bytes_.ctypes.data_as(C.POINTER(C.c_int64)), nd,
                                    budgets.ctypes.data_as(C.POINTER(C.c_int64)), ip(cur) if cur is not None else None,
                                    ip(out), load.ctypes.data_as(C.POINTER(C.c_double)))
    if check and rc not in (GW_OK, GW_EBUDGET):
        _check(rc)
    return rc, out, load


def gw_server_wait(s, ticket, timeout_us=-1):
    _check(lib().gw_server_wait(s, ticket, timeout_us))


def gw_server_stats_read(s, reset=False):
    st = gw_server_stats()
    _check(lib().gw_server_stats_read(s, 1 if reset else 0, C.byref(st)))
    return {k: getattr(st, k) for k, _ in gw_server_stats._fields_}


def gw_server_replay(s, ids, t_us, witness, strain, clean, score=None, latency_us=None):
    """ids int32 [n], t_us float64 [n]; witness / strain / clean: lists of float32 arrays (one per request) or
    uint64 arrays of their host addresses; score float32 [n] and latency_us float64 [n] optional outputs."""
    n = len(ids)
    ids = np.ascontiguousarray(ids, np.int32)
    t_us = np.ascontiguousarray(t_us, np.float64)
    addr = lambda xs: (np.ascontiguousarray(xs, np.uint64) if isinstance(xs, np.ndarray) and xs.dtype == np.uint64
                       else np.array([a.ctypes.data for a in xs], np.uint64))
    wp, sp, cp = addr(witness), addr(strain), addr(clean)
    _check(lib().gw_server_replay(s, n, ids.ctypes.data, t_us.ctypes.data, wp.ctypes.data, sp.ctypes.data,
                                  cp.ctypes.data, score.ctypes.data if score is not None else None,
                                  latency_us.ctypes.data if latency_us is not None else None))


def gw_server_destroy(s):
    _check(lib().gw_server_destroy(s))


def gw_trainer_create(ctx, n_in, max_batch, length, checkpoint=0, in_mean=None, in_std=None, precision=GW_FP32,
                      tc_data=0):
    d = gw_trainer_desc(n_in, max_batch, length, checkpoint, precision, tc_data)
    m = None if in_mean is None else np.ascontiguousarray(in_mean, np.float32)
    s = None if in_std is None else np.ascontiguousarray(in_std, np.float32)
    h = P()
    _check(lib().gw_trainer_create(ctx, C.byref(d), m.ctypes.data if m is not None else None,
                                   s.ctypes.data if s is not None else None, C.byref(h)))
    return h


def gw_trainer_destroy(t):
    _check(lib().gw_trainer_destroy(t))


def gw_trainer_status(t, stream=0):
    _check(lib().gw_trainer_status(t, stream or None))


def gw_trainer_param_count(t):
    return _check(lib().gw_trainer_param_count(t))


def gw_trainer_bytes(t):
    return _check(lib().gw_trainer_bytes(t))


def gw_trainer_forward(t, params_ptr, x_ptr, B, y_ptr, stream=0):
    _check(lib().gw_trainer_forward(t, params_ptr, x_ptr, B, y_ptr, stream or None))


def gw_trainer_backward(t, dy_ptr, dparams_ptr, stream=0):
    _check(lib().gw_trainer_backward(t, dy_ptr, dparams_ptr, stream or None))


def gw_fir_create_bandpass(ctx, fs, nfft, ntaps, f1=55.0, f2=65.0, ramp=2.0, precision=GW_FP32):
    h = P()
    _check(lib().gw_fir_create_bandpass(ctx, fs, nfft, ntaps, f1, f2, ramp, precision, C.byref(h)))
    return h.value


def gw_fir_create_band_loss(ctx, psd, fs, ntaps, f1=55.0, f2=65.0, ramp=2.0, f_ref=60.0, precision=GW_FP32):
    psd = np.ascontiguousarray(psd, np.float64)
    h = P()
    _check(lib().gw_fir_create_band_loss(ctx, psd.ctypes.data_as(C.POINTER(C.c_double)), psd.size, fs, ntaps, f1, f2,
                                         ramp, f_ref, precision, C.byref(h)))
    return h


def gw_band_loss(g, strain_ptr, y_ptr, B, L, loss_ptr, r_ptr, stream=0):
    _check(lib().gw_band_loss(g, strain_ptr, y_ptr, B, L, loss_ptr, r_ptr, stream or None))


def gw_band_loss_backward(g, r_ptr, B, L, dloss_ptr, dy_ptr, stream=0):
    _check(lib().gw_band_loss_backward(g, r_ptr, B, L, dloss_ptr or None, dy_ptr, stream or None))


def gw_fir_backward(f, dy_ptr, B, Cc, L_in, dx_ptr, stream=0):
    _check(lib().gw_fir_backward(f, dy_ptr, B, Cc, L_in, dx_ptr, stream or None))


def gw_adam_step(p_ptr, g_ptr, m_ptr, v_ptr, n, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=0):
    _check(lib().gw_adam_step(p_ptr, g_ptr, m_ptr, v_ptr, n, step, lr, beta1, beta2, eps, stream or None))


def gw_adam_step_dev(p_ptr, g_ptr, m_ptr, v_ptr, n, step_ptr, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=0):
    """Adam with the step count in device memory (int32 at step_ptr, incremented on the device)."""
    _check(lib().gw_adam_step_dev(p_ptr, g_ptr, m_ptr, v_ptr, n, step_ptr, lr, beta1, beta2, eps, stream or None))


def gw_profile_enable(on=True):
    _check(lib().gw_profile_enable(1 if on else 0))


def gw_profile_read(max_entries=64):
    """{kernel name: (total_ms, launches)} since the last gw_profile_enable."""
    names = C.create_string_buffer(1 << 16)
    ms = (C.c_double * max_entries)()
    cnt = (C.c_int64 * max_entries)()
    n = _check(lib().gw_profile_read(names, len(names), ms, cnt, max_entries))
    keys = names.value.decode().split("\n")[:n]
    return {k: (ms[i], cnt[i]) for i, k in enumerate(keys)}


def gw_launch_count():
    return lib().gw_launch_count()


def gw_alloc_count():
    return lib().gw_alloc_count()


TC_META = ("n_steps", "npad", "groups", "in_P", "Q", "dspan", "dmin", "MT", "rows", "a_bytes", "sps", "nst",
           "step_bytes", "ncols", "tiles_per_item", "mout", "coutp", "idesc", "smem", "lout", "nsplit",
           "wstep", "wcompact", "wprod", "na", "per_sm")


def gw_tc_inspect(spec, precision, wfold, lin, in_P, out_P, batch=1):
    """Host-only lowering of one layer: (image bytes, table uint32, meta dict)."""
    spec_a = (C.c_int * 8)(*spec)
    wf = np.ascontiguousarray(wfold, np.float64)
    cap = 1 << 24
    img = np.zeros(cap, np.uint8)
    table = np.zeros(1 << 14, np.uint32)
    meta = (C.c_int * len(TC_META))()
    _check(lib().gw_tc_inspect(spec_a, precision, wf.ctypes.data_as(C.POINTER(C.c_double)), lin, in_P, out_P, batch,
                               img.ctypes.data, cap, table.ctypes.data_as(C.POINTER(C.c_uint32)), table.size, meta))
    md = dict(zip(TC_META, list(meta)))
    md["idesc"] &= 0xFFFFFFFF
    return img[:md["n_steps"] * md["step_bytes"]].copy(), table[:2 * md["n_steps"]].copy(), md
