"""The benchmark's compact JSON line (no GPU): what it keeps of the configs."""
import bench


def test_compact_line_keeps_numbers_short_strings_and_errors():
    err = "GW_ETIMEOUT: a tensor-core kernel gave up a bounded wait"
    out = bench.compact_configs({
        "config5_bf16": {"saturated": {"snapshots_per_s": 161467.25292735078, "ticks": 3922},
                         "workload": "w" * 60, "tick_kernels_eager": {"batch1": {}}},
        "config4_error": err,
        "config5_fp32": {"error": err, "p50_us": 1.23456789},
        "config1_bf16": {"p50_us": 23.18400051444769, "note": "short"},
    })
    # floats to four significant digits, nested dicts of scalars kept
    assert out["config5_bf16"]["saturated"] == {"snapshots_per_s": 161500.0, "ticks": 3922}
    # long descriptions and per-kernel tables are left out, error messages kept whole
    assert "workload" not in out["config5_bf16"] and "tick_kernels_eager" not in out["config5_bf16"]
    assert out["config4_error"] == err and out["config5_fp32"]["error"] == err
    assert out["config1_bf16"] == {"p50_us": 23.18, "note": "short"}
    # the serving block comes last, so that a truncated tail still shows it
    assert list(out)[-1] == "config5_bf16"
