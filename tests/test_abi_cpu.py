"""CPU-only checks of the C-ABI library: it builds, loads, and exports every
symbol include/gwstream.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

from paper_2108_12430_gb300 import build, gwstream

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gwstream.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gw_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_header_symbols():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(gwstream.EXPORTS), set(names) ^ set(gwstream.EXPORTS)


def test_param_counts_match_generators():
    from paper_2108_12430_gb300 import synth
    lib = gwstream.lib()
    dc = synth.flatten_params(synth.deepclean_params(0))
    assert lib.gw_model_param_count(gwstream.GW_MODEL_DEEPCLEAN, 21) == dc.size
    layers, head = synth.bbhnet_params(0)
    assert lib.gw_model_param_count(gwstream.GW_MODEL_BBHNET, 2) == synth.flatten_params(layers, head).size
    assert lib.gw_model_param_count(7, 2) == 0


def test_error_paths_without_gpu():
    lib = gwstream.lib()
    h = ctypes.c_void_p()
    assert lib.gw_ctx_create(0, 0, None) == gwstream.GW_EINVAL
    assert b"NULL" in lib.gw_last_error()
    assert lib.gw_model_destroy(None) == gwstream.GW_EINVAL
    assert lib.gw_stream_push(None, 1, None, None, None, 0, None) == gwstream.GW_EINVAL
    assert gwstream.gw_version().startswith("gwstream")


def test_server_error_paths_without_gpu():
    lib = gwstream.lib()
    h = ctypes.c_void_p()
    sid = ctypes.c_int()
    assert lib.gw_server_create(None, None, None, None, None, None, ctypes.byref(h)) == gwstream.GW_EINVAL
    assert lib.gw_server_open(None, 256, ctypes.byref(sid)) == gwstream.GW_EINVAL
    assert lib.gw_server_close(None, 0) == gwstream.GW_EINVAL
    assert lib.gw_server_submit(None, 0, None, None, None, None, None) == gwstream.GW_EINVAL
    assert lib.gw_server_wait(None, 1, 0) == gwstream.GW_EINVAL
    assert lib.gw_server_stats_read(None, 0, None) == gwstream.GW_EINVAL
    assert lib.gw_server_destroy(None) == gwstream.GW_EINVAL
    assert lib.gw_server_stream_bytes(None, 256) == gwstream.GW_EINVAL
    assert lib.gw_fir_create_lowpass(None, 900.0, 4096.0, 127, 0, ctypes.byref(h)) == gwstream.GW_EINVAL
    assert b"NULL" in lib.gw_last_error()
