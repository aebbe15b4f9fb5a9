"""Streaming DeepClean benchmark on one GB300 (or N independent replicas).

Workload: DeepClean-shaped streaming inference, windows of 21 x 32768 samples
(8 s at 4096 Hz), stride 256 samples per snapshot, 64 snapshots per batch,
full overlap-add aggregation (each cleaned sample averaged over the 128
windows that cover it).  One step = one push of 64 new snapshots through the
whole streaming path: device ring update, DeepClean on the 64 windows, and
the fused subtract + overlap-add that emits 64 x 256 cleaned samples.

Metric: snapshots/s (whole job), with p50/p99 step latency, for the BF16
tensor-core path and the plain FP32 path (value = the BF16 path when built).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gw|reference]

Under torchrun each rank runs an independent replica on its own GPU (the path
has no cross-stream exchange); the timed region is bracketed by barriers and
the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

W, S, B, C = 32768, 256, 64, 21
METRIC = "streaming snapshots/s and p50/p99 latency, BF16 vs FP32 path at stated error, 1 GB300"
WORKLOAD = "DeepClean streaming: 21x32768 windows (8 s @ 4096 Hz), stride 256, batch 64, overlap-add"
L2_BYTES = 129 * 1024 * 1024
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the whole-network DeepClean kernel on this workload, from the ncu capture
# summarised in profiles/deepclean_fused_stream_batch64.md (None when the
# kernel has changed since that capture)
FUSED_TRAFFIC_BYTES_PER_LAUNCH = 5_337_344


def dc_flops_per_window(L=W):
    """Algorithmic FLOPs of one DeepClean window (2 per MAC, valid outputs only)."""
    from paper_2108_12430_gb300 import synth
    f, lin = 0, L
    for kind, cin, cout, k, s, pl, pr, op, bn, act in synth.DEEPCLEAN_LAYERS:
        if kind == "conv":
            lout = (lin + pl + pr - k) // s + 1
            f += 2 * cout * cin * k * lout
        else:
            lout = (lin - 1) * s - pl - pr + k + op
            f += 2 * cout * cin * k * lin
        lin = lout
    return f


def dc_algorithmic_bytes_per_push(L=W, batch=B, stride=S, c_in=C):
    """Algorithmic bytes of one push's DeepClean: the unique witness input
    once (BF16, channels padded to groups of 8; the batch's windows overlap),
    the FP32 predictions written once, and the aggregation's read-modify-write
    of the overlap-add accumulator and the strain read over the batch's span
    (the parameters, 0.08 MB, are not counted)."""
    cpad = (c_in + 7) // 8 * 8
    span = L + (batch - 1) * stride
    return cpad * span * 2 + batch * L * 4 + span * 4 * 3


def dc_layer_flops(L=W):
    from paper_2108_12430_gb300 import synth
    out, lin = [], L
    for kind, cin, cout, k, s, pl, pr, op, bn, act in synth.DEEPCLEAN_LAYERS:
        if kind == "conv":
            lout = (lin + pl + pr - k) // s + 1
            out.append(2 * cout * cin * k * lout)
        else:
            lout = (lin - 1) * s - pl - pr + k + op
            out.append(2 * cout * cin * k * lin)
        lin = lout
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx = float(p[1])
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def rank_env():
    """(world size, rank, local rank) from the launcher's environment; (1, 0, 0) alone."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def slowest(dist, world, value, device):
    """The largest value over all ranks (the slowest rank's timed interval)."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units every replica processed over the slowest one's time."""
    return units_per_rank * world / seconds


def make_stream_inputs(n_samples, seed=1234):
    from paper_2108_12430_gb300 import synth
    wit = synth.witness_channels(seed, C, n_samples)
    strain = synth.coupled_strain(seed, wit)
    return wit.astype(np.float32), strain.astype(np.float32)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_path(G, torch, precision, steps, warmup, wit_d, str_d, flush, dev_index):
    """Time `steps` device-resident pushes; returns per-step ms and profile."""
    from paper_2108_12430_gb300 import synth
    ctx = G.gw_ctx_create(dev_index, 0)
    params = synth.flatten_params(synth.deepclean_params(1234))
    m = G.gw_model_create(ctx, G.GW_MODEL_DEEPCLEAN, precision, C, params)
    s = G.gw_stream_create(ctx, [m], 1, C, W, S, B, G.GW_AGG_AVERAGE, W - S)
    out = torch.zeros(B * S, device="cuda")
    st = torch.cuda.current_stream()
    h = st.cuda_stream
    n_step = B * S

    def push(i):
        o = i * n_step
        G.gw_stream_push(s, B, wit_d[:, o:o + n_step].contiguous().data_ptr(),
                         str_d[o:o + n_step].contiguous().data_ptr(), out.data_ptr(), G.GW_MEM_DEVICE, h)

    # pre-slice inputs so the timed region holds only the library's work
    slices = [(wit_d[:, i * n_step:(i + 1) * n_step].contiguous(), str_d[i * n_step:(i + 1) * n_step].contiguous())
              for i in range(warmup + steps)]

    def push_pre(i):
        w_, s_ = slices[i]
        G.gw_stream_push(s, B, w_.data_ptr(), s_.data_ptr(), out.data_ptr(), G.GW_MEM_DEVICE, h)

    for i in range(warmup):
        push_pre(i)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    l0 = G.gw_launch_count()
    for i in range(steps):
        flush.zero_()  # evict L2 between timed steps (outside the events)
        evs[i][0].record(st)
        push_pre(warmup + i)
        evs[i][1].record(st)
    torch.cuda.synchronize()
    launches = G.gw_launch_count() - l0
    ms = [a.elapsed_time(b) for a, b in evs]
    res = {"ms": ms, "launches_per_step": launches / steps}
    return ctx, m, s, res, push_pre


def profile_pass(G, torch, push_fn, first, steps, flush):
    G.gw_profile_enable(True)
    for i in range(steps):
        flush.zero_()
        push_fn(first + i)
    torch.cuda.synchronize()
    prof = G.gw_profile_read()
    G.gw_profile_enable(False)
    return prof


def accuracy(G, torch, precision, dev_index):
    """rel-L2 of two full 21 x 32768 windows against the FP64 oracle (CPU leg)."""
    from paper_2108_12430_gb300 import synth
    ctx = G.gw_ctx_create(dev_index, 0)
    params = synth.deepclean_params(1234)
    m = G.gw_model_create(ctx, G.GW_MODEL_DEEPCLEAN, precision, C, synth.flatten_params(params))
    x = synth.witness_channels(77, C, W + S)
    y = torch.zeros(2, W, device="cuda")
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    G.gw_deepclean_forward(m, xd.data_ptr(), W + S, S, 2, W, y.data_ptr())
    torch.cuda.synchronize()
    wins = np.stack([x[:, :W], x[:, S:S + W]]).astype(np.float32).astype(np.float64)
    ref = cpu_leg_deepclean(wins, params)
    got = y.cpu().numpy().astype(np.float64)
    err = max(float(np.linalg.norm(got[i] - ref[i]) / np.linalg.norm(ref[i])) for i in range(2))
    G.gw_model_destroy(m)
    G.gw_ctx_destroy(ctx)
    return err


def e2e_pass(G, torch, s, wit_h, str_h, first, steps):
    """Host-buffer pushes through the public API: H2D + compute + D2H per step."""
    n_step = B * S
    out = torch.empty(B * S, dtype=torch.float32).pin_memory()
    lat = []
    lib = G.lib()
    h = torch.cuda.current_stream().cuda_stream
    for i in range(steps):
        w_, s_ = wit_h[first + i], str_h[first + i]
        t0 = time.perf_counter()
        rc = lib.gw_stream_push(s, B, w_.data_ptr(), s_.data_ptr(), out.data_ptr(), G.GW_MEM_HOST, h)
        lat.append((time.perf_counter() - t0) * 1e3)
        if rc < 0:
            raise G.GwError(rc, lib.gw_last_error().decode())
    return lat


def e2e_pipelined(G, torch, s, wit_h, str_h, first, steps):
    """Queued host-buffer pushes through the public API: each step's H2D copy,
    compute and D2H copy of its cleaned samples (into its own pinned buffer)
    are queued with gw_stream_push_async; one gw_stream_sync ends the timed
    region.  Returns the wall time in ms."""
    outs = [torch.empty(B * S, dtype=torch.float32).pin_memory() for _ in range(steps)]
    lib = G.lib()
    h = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        rc = lib.gw_stream_push_async(s, B, wit_h[first + i].data_ptr(), str_h[first + i].data_ptr(),
                                      outs[i].data_ptr(), h)
        if rc < 0:
            raise G.GwError(rc, lib.gw_last_error().decode())
    G.gw_stream_sync(s)
    return (time.perf_counter() - t0) * 1e3


def gpu_arm(args):
    import torch
    import torch.distributed as dist

    from paper_2108_12430_gb300 import build as Bld
    Bld.build()
    from paper_2108_12430_gb300 import gwstream as G

    world, rank, local = rank_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev_index = torch.cuda.current_device()
    K, Wm = args.steps, args.warmup
    npipe = max(K, 8)  # pipelined host-buffer steps
    n_total = (Wm + K + 8 + npipe) * B * S
    wit, strain = make_stream_inputs(n_total, seed=1234 + rank)
    wit_d = torch.from_numpy(wit).cuda()
    str_d = torch.from_numpy(strain).cuda()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    pk, pk_src = peaks()

    paths = {}
    precisions = [("bf16", G.GW_BF16), ("fp32", G.GW_FP32)]
    if args.only:
        precisions = [p for p in precisions if p[0] == args.only]
    headline = None
    clocks = None
    for name, prec in precisions:
        try:
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            with ClockSampler(dev_index) as cs:
                ctx, m, s, res, push_fn = run_path(G, torch, prec, K, Wm, wit_d, str_d, flush, dev_index)
            if world > 1:
                dist.barrier()
        except G.GwError as e:
            if e.code == G.GW_ENOTIMPL:
                paths[name] = {"unavailable": str(e)}
                continue
            raise
        ms = np.array(res["ms"])
        tot = slowest(dist, world, float(ms.sum()), "cuda")
        if args.lite:
            # profiling runs: only the device-resident timed pushes above
            G.gw_stream_destroy(s)
            G.gw_model_destroy(m)
            G.gw_ctx_destroy(ctx)
            paths[name] = {"ms_per_step": float(np.mean(res["ms"]))}
            continue
        prof = profile_pass(G, torch, push_fn, Wm, min(K, 8), flush)
        # host-buffer e2e: pinned host copies of the next steps' inputs (the
        # pushes continue the same stream)
        n_step = B * S
        first = Wm + K
        ne2e = min(K, 8)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        wit_h = {first + i: pin(wit[:, (first + i) * n_step:(first + i + 1) * n_step])
                 for i in range(ne2e)}
        str_h = {first + i: pin(strain[(first + i) * n_step:(first + i + 1) * n_step]) for i in range(ne2e)}
        f2 = first + ne2e
        wit_h.update({f2 + i: pin(wit[:, (f2 + i) * n_step:(f2 + i + 1) * n_step]) for i in range(npipe)})
        str_h.update({f2 + i: pin(strain[(f2 + i) * n_step:(f2 + i + 1) * n_step]) for i in range(npipe)})
        if world > 1:
            dist.barrier()
        lat = e2e_pass(G, torch, s, wit_h, str_h, first, ne2e)
        e2e_tot = slowest(dist, world, float(sum(lat)), "cuda")
        if world > 1:
            dist.barrier()
        pipe_ms = slowest(dist, world, e2e_pipelined(G, torch, s, wit_h, str_h, f2, npipe), "cuda")
        err = accuracy(G, torch, prec, dev_index) if rank == 0 else None
        G.gw_stream_destroy(s)
        G.gw_model_destroy(m)
        G.gw_ctx_destroy(ctx)
        # DeepClean's kernels: the whole-network kernel (BF16) or the eight
        # per-layer convolutions (FP32)
        dc_ms = sum(v[0] for k, v in prof.items() if k.startswith("conv") or k == "deepclean_fused")
        prof_steps = min(K, 8)
        dc_flops = dc_flops_per_window() * B * prof_steps
        paths[name] = {
            "value": job_rate(B * K, world, tot / 1e3),
            "ms_per_step": tot / K,
            "p50_ms": float(np.percentile(ms, 50)),
            "p99_ms": float(np.percentile(ms, 99)),
            "rel_l2_vs_fp64_oracle": err,
            "e2e_value": job_rate(B * npipe, world, pipe_ms / 1e3),
            "e2e_ms_per_step": pipe_ms / npipe,
            "e2e_sync_value": job_rate(B * ne2e, world, e2e_tot / 1e3),
            "e2e_p50_ms": float(np.percentile(lat, 50)),
            "e2e_p99_ms": float(np.percentile(lat, 99)),
            "gpu_launches_per_step": res["launches_per_step"],
            "deepclean_tflops": dc_flops / (dc_ms / 1e3) / 1e12 if dc_ms else None,
            "kernels": {k: {"ms_per_step": v[0] / prof_steps, "launches_per_step": v[1] / prof_steps}
                        for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])},
            "clocks": cs.summary(),
        }
        if headline is None:
            headline = name
            clocks = paths[name]["clocks"]

    if rank != 0 or args.lite:
        if args.lite and rank == 0:
            print(json.dumps({"lite": True, "paths": paths}))
        if world > 1:
            dist.destroy_process_group()
        return
    hp = paths[headline]
    kernels = hp["kernels"]
    flops_step = dc_flops_per_window() * B
    if headline == "bf16":
        # one launch of the whole-network kernel per push: a dense
        # contraction far above the ridge point (31.5 GFLOP on ~11 MB of
        # algorithmic traffic), so the binding roofline is the tensor core
        kname = "deepclean_fused"
        k_ms = kernels[kname]["ms_per_step"] / kernels[kname]["launches_per_step"]
        achieved = flops_step / (k_ms / 1e3) / 1e12
        peak = pk["bf16_tflops"]
        ai = flops_step / dc_algorithmic_bytes_per_push()
        ridge = pk["bf16_tflops"] * 1e12 / (pk["hbm_gbs"] * 1e9)
        roofline = {"bound": "tensor", "kernel": kname + " (1 launch per step)", "achieved": achieved,
                    "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": FUSED_TRAFFIC_BYTES_PER_LAUNCH,
                    "peak_source": f"dense bf16 burst, {pk_src} (the kernel is timed alone: one launch per push)",
                    "launch_ms": k_ms, "flop_per_launch": flops_step,
                    "per_unit": f"{dc_flops_per_window()} flop per 21x32768 window x {B} windows per launch",
                    "algorithmic_bytes_per_launch": dc_algorithmic_bytes_per_push(),
                    "arithmetic_intensity_flop_per_byte": ai, "ridge_flop_per_byte": ridge,
                    "traffic_unit": "DRAM bytes per launch (ncu capture, cold cache)"}
        if FUSED_TRAFFIC_BYTES_PER_LAUNCH:
            roofline["traffic_over_algorithmic"] = FUSED_TRAFFIC_BYTES_PER_LAUNCH / dc_algorithmic_bytes_per_push()
    else:
        conv_ms_step = sum(v["ms_per_step"] for k, v in kernels.items() if k.startswith("conv"))
        achieved = flops_step / (conv_ms_step / 1e3) / 1e12
        peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roofline = {"bound": "alu", "kernel": "conv_f32 (8 launches per step)", "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                    "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x max SM clock"}
    configs = {}
    # the other configurations: a library error in one is recorded as its
    # result and the rest still run, so that the line is always printed
    for name, run in (("configs_1_3", lambda: extra_configs(G, torch, dev_index, flush)),
                      ("bulk", lambda: bulk_config(G, torch, dev_index, flush)),
                      ("study", lambda: study_config(dev_index)),
                      ("config4", lambda: train_config(G, torch, dev_index, flush)),
                      ("config5", lambda: serve_configs(G, dev_index))):
        try:
            configs.update(run())
        except G.GwError as e:
            configs[f"{name}_error"] = str(e)
    cpu = cpu_baseline(budget_s=args.cpu_seconds)
    cpu["one_core"] = cpu_baseline_one_core()
    line = {
        "metric": METRIC,
        "value": hp["value"],
        "unit": "snapshots/s",
        "n_gpus": world,
        "steps": K,
        "warmup": Wm,
        "ms_per_step": hp["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16" if headline == "bf16" else "f32",
        "data": "synthetic (seeded witness noise + coloured aLIGO-like strain with 60 Hz coupling)",
        "config": {"workload": WORKLOAD, "window": W, "stride": S, "batch": B, "channels": C,
                   "aggregation": "AVERAGE, delay W-S", "path": headline,
                   "l2": "flushed between timed steps (256 MiB write outside the events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "p50_ms": hp["p50_ms"],
        "p99_ms": hp["p99_ms"],
        "rel_l2_vs_fp64_oracle": hp["rel_l2_vs_fp64_oracle"],
        "e2e": {"value": hp["e2e_value"], "unit": "snapshots/s", "ms_per_step": hp["e2e_ms_per_step"],
                "h2d_bytes_per_step": (C + 1) * B * S * 4, "d2h_bytes_per_step": B * S * 4 + 4,
                "mode": "pipelined host-buffer pushes: gw_stream_push_async per step (pinned inputs, "
                        "H2D + check + compute + D2H of the cleaned samples and the reject flag), "
                        "one gw_stream_sync at the end of the timed region",
                "sync": {"value": hp["e2e_sync_value"], "p50_ms": hp["e2e_p50_ms"], "p99_ms": hp["e2e_p99_ms"],
                         "mode": "gw_stream_push in host mode, returning per step"}},
        "gpu_launches": int(round(hp["gpu_launches_per_step"] * K)),
        "roofline": roofline,
        "paths": {k: {kk: vv for kk, vv in v.items() if kk != "clocks"} for k, v in paths.items()},
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    # the full records (per-kernel breakdowns, descriptions) go to stderr, so
    # that the one JSON line stays short; the line carries the numbers, with
    # the serving configuration last
    detail = {"paths_kernels": {k: v.get("kernels") for k, v in paths.items()}, "configs": configs}
    print(json.dumps(detail), file=sys.stderr)
    for v in line["paths"].values():
        v.pop("kernels", None)
    line["configs"] = compact_configs(configs)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def compact_configs(configs):
    """The configs' numbers for the JSON line: scalars (floats to 4 significant
    digits) and one level of nested dicts of scalars; descriptions, series and
    per-kernel tables are left to the stderr record.  config5_bf16 comes last."""
    def keep(v, key=""):
        # short strings, and error messages whole
        return isinstance(v, (int, float, bool)) or v is None or (isinstance(v, str) and
                                                                   (len(v) <= 40 or key.endswith("error")))

    def rnd(v):
        return float(f"{v:.4g}") if isinstance(v, float) else v

    out = {}
    order = [k for k in configs if k != "config5_bf16"] + [k for k in configs if k == "config5_bf16"]
    for k in order:
        v = configs[k]
        if not isinstance(v, dict):
            out[k] = rnd(v) if keep(v, k) else None
            continue
        c = {}
        for kk, vv in v.items():
            if "kernel" in kk and kk != "kernels_per_tick":
                continue
            if isinstance(vv, dict):
                sub = {a: rnd(b) for a, b in vv.items() if keep(b, a) and "kernel" not in a}
                if sub:
                    c[kk] = sub
            elif keep(vv, kk):
                c[kk] = rnd(vv)
        out[k] = c
    return out


def bbhnet_flops_per_window(L=2048):
    """Algorithmic FLOPs of one BBHnet window (stem, 4 blocks, head)."""
    from paper_2108_12430_gb300 import synth
    f, lin = 0, L
    lay = synth.bbhnet_layers()
    # stem then blocks: conv1 and shortcut read the block input, conv2 conv1's output
    kind, cin, cout, k, s, pl, pr, op, bn, act = lay[0]
    lin = (lin + pl + pr - k) // s + 1
    f += 2 * cout * cin * k * lin
    for i in range(1, len(lay), 3):
        c1, c2, sc = lay[i], lay[i + 1], lay[i + 2]
        l2 = (lin + c1[5] + c1[6] - c1[3]) // c1[4] + 1
        f += 2 * c1[2] * c1[1] * c1[3] * l2 + 2 * c2[2] * c2[1] * c2[3] * l2 + 2 * sc[2] * sc[1] * sc[3] * l2
        lin = l2
    return f + 2 * 256


def time_call(torch, fn, steps, warmup, flush=None):
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    evs = []
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        fn()
        b.record(st)
        evs.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def extra_configs(G, torch, dev_index, flush, steps=10, warmup=3):
    """Config 1 (one 1 s DeepClean window) latency and config 3 (whitening +
    BBHnet on 256 x 2 x 4096 raw strain) throughput, BF16, FP8 (BBHnet) and
    FP32, each with its error against the FP64 oracle (CPU leg) on sampled
    items."""
    from paper_2108_12430_gb300 import synth
    out = {}
    ctx = G.gw_ctx_create(dev_index, 0)
    try:
        # config 1
        x1 = synth.witness_channels(0, C, 4096)
        t0 = time.perf_counter()
        ref1 = cpu_leg_deepclean(x1[None].astype(np.float32).astype(np.float64), synth.deepclean_params(0))[0]
        out["config1_oracle"] = {"kind": "oracle", "us_per_forward": (time.perf_counter() - t0) * 1e6,
                                 "cores": cpu_threads(), "sample": "the one window whose output the error fields use"}
        x1d = torch.from_numpy(x1.astype(np.float32)).cuda()
        y1 = torch.zeros(1, 4096, device="cuda")
        for name, prec in (("bf16", G.GW_BF16), ("fp32", G.GW_FP32)):
            m = G.gw_model_create(ctx, G.GW_MODEL_DEEPCLEAN, prec, C, synth.flatten_params(synth.deepclean_params(0)))
            ms = time_call(torch, lambda: G.gw_deepclean_forward(m, x1d.data_ptr(), 4096, 0, 1, 4096, y1.data_ptr()),
                           steps, warmup)
            err = float(np.linalg.norm(y1.cpu().numpy()[0] - ref1) / np.linalg.norm(ref1))
            # the same forward captured once into a CUDA graph and replayed
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                G.gw_deepclean_forward(m, x1d.data_ptr(), 4096, 0, 1, 4096, y1.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
            ms_g = time_call(torch, graph.replay, steps, warmup)
            err_g = float(np.linalg.norm(y1.cpu().numpy()[0] - ref1) / np.linalg.norm(ref1))
            del graph
            out[f"config1_{name}"] = {"workload": "DeepClean forward 1x21x4096", "p50_us": float(np.median(ms) * 1e3),
                                      "p99_us": float(np.percentile(ms, 99) * 1e3), "rel_l2_vs_fp64_oracle": err,
                                      "graph_replay_p50_us": float(np.median(ms_g) * 1e3),
                                      "graph_replay_p99_us": float(np.percentile(ms_g, 99) * 1e3),
                                      "graph_replay_rel_l2_vs_fp64_oracle": err_g}
            G.gw_model_destroy(m)
        # config 3: whitening (2049 taps) + BBHnet, batch 256
        Bc, Lr = 256, 4096
        fs, nfft = 2048.0, 8192
        fgrid, psd = synth.psd_grid(fs, nfft)
        xr, label, snr = synth.injected_strain(31, Bc, Lr)
        xrd = torch.from_numpy(xr.astype(np.float32)).cuda()
        wd = torch.zeros(Bc, 2, Lr - 2048, device="cuda")
        logit = torch.zeros(Bc, device="cuda")
        idx = [0, 77, 255]
        layers, head = synth.bbhnet_params(3)
        t0 = time.perf_counter()
        xw_ref, ref3 = cpu_leg_whiten_bbhnet(xr[idx].astype(np.float32).astype(np.float64), psd, fs, nfft, layers,
                                             head)
        out["config3_oracle"] = {"kind": "oracle", "windows_per_s": len(idx) / (time.perf_counter() - t0),
                                 "cores": cpu_threads(),
                                 "sample": f"{len(idx)} windows (whitening design + FIR + BBHnet) whose outputs the "
                                           "error fields use"}
        for name, prec in (("bf16", G.GW_BF16), ("fp8", G.GW_FP8), ("fp32", G.GW_FP32)):
            fh = G.gw_fir_create_whitening(ctx, psd, fs, 2049, G.GW_BF16 if prec == G.GW_FP8 else prec)
            mb = G.gw_model_create(ctx, G.GW_MODEL_BBHNET, prec, 2, synth.flatten_params(layers, head))
            if prec == G.GW_FP8:
                # static activation scales from a separate calibration batch,
                # whitened by the library
                xc, _, _ = synth.injected_strain(32, 64, Lr)
                xcd = torch.from_numpy(xc.astype(np.float32)).cuda()
                wc = torch.zeros(64, 2, Lr - 2048, device="cuda")
                G.gw_whiten(fh, xcd.data_ptr(), 64, 2, Lr, wc.data_ptr())
                G.gw_model_calibrate(mb, wc.data_ptr(), 64, Lr - 2048)

            def step():
                G.gw_whiten(fh, xrd.data_ptr(), Bc, 2, Lr, wd.data_ptr())
                G.gw_bbhnet_score(mb, wd.data_ptr(), Bc, Lr - 2048, logit.data_ptr())

            ms = time_call(torch, step, steps, warmup, flush)
            G.gw_profile_enable(True)
            for _ in range(3):
                step()
            torch.cuda.synchronize()
            prof = G.gw_profile_read()
            G.gw_profile_enable(False)
            got = logit.cpu().numpy()[idx]
            wgot = wd.cpu().numpy()[idx]
            werr = float(np.linalg.norm(wgot - xw_ref) / np.linalg.norm(xw_ref))
            flops = bbhnet_flops_per_window() * Bc + 2 * 2049 * Bc * 2 * 2048
            out[f"config3_{name}"] = {
                "workload": "whiten 2049 taps + BBHnet, batch 256 x 2 x 4096",
                "ms_per_batch": float(np.mean(ms)), "windows_per_s": Bc / (np.mean(ms) / 1e3),
                "tflops": flops / (np.mean(ms) / 1e3) / 1e12,
                "whiten_rel_l2": werr, "max_abs_logit_err": float(np.abs(got - ref3).max()),
                "kernels_ms": {k: v[0] / 3 for k, v in prof.items()}}
            G.gw_model_destroy(mb)
            G.gw_fir_destroy(fh)
    finally:
        G.gw_ctx_destroy(ctx)
    return out


def bulk_config(G, torch, dev_index, flush, steps=10, warmup=3):
    """Offline bulk mode (Methods, offline deployment: snapshots at r = 0.25 Hz
    over a recording): 8 s windows at stride S = f_s / r = 16384, 64 windows
    per push (256 s of data), every sample averaged over the two windows that
    cover it; BF16, device-resident input; reported as seconds of data cleaned
    per second."""
    from paper_2108_12430_gb300 import synth
    Sb, Bb = 16384, 64
    out = {}
    ctx = G.gw_ctx_create(dev_index, 0)
    try:
        m = G.gw_model_create(ctx, G.GW_MODEL_DEEPCLEAN, G.GW_BF16, C, synth.flatten_params(synth.deepclean_params(0)))
        s = G.gw_stream_create(ctx, [m], 1, C, W, Sb, Bb, G.GW_AGG_AVERAGE, W - Sb)
        n = Bb * Sb
        wit = torch.from_numpy(synth.witness_channels(77, C, n).astype(np.float32)).cuda()
        stn = torch.zeros(n, device="cuda")
        cln = torch.zeros(n, device="cuda")
        step = lambda: G.gw_stream_push(s, Bb, wit.data_ptr(), stn.data_ptr(), cln.data_ptr(), G.GW_MEM_DEVICE)
        ms = time_call(torch, step, steps, warmup, flush)
        per = float(np.mean(ms))
        out["bulk_bf16"] = {"workload": f"offline bulk: DeepClean {C}x{W} windows at stride {Sb} (r = 0.25 Hz), "
                                        f"{Bb} windows per push, overlap-add", "ms_per_push": per,
                            "data_seconds_per_push": n / 4096.0,
                            "data_seconds_per_s": n / 4096.0 / (per / 1e3)}
        G.gw_stream_destroy(s)
        G.gw_model_destroy(m)
    finally:
        G.gw_ctx_destroy(ctx)
    return out


def study_config(dev_index):
    """The aggregation-latency study (Methods, "Aggregation latency"): train
    DeepClean on synthetic 60 Hz coupling with the library's training step,
    clean a held-out segment offline and online (8 s windows, stride 256,
    causal scheme with aggregation latency 0 / 0.5 / 0.75 s) and compare ASD
    ratios; the paper reports ~23% / ~4% / ~1% of [50, 70] Hz bins off the
    offline ratio by more than 10%."""
    from paper_2108_12430_gb300 import study
    import time as _t
    out = {}
    for name, taps in (("study_aggregation_latency", 0), ("study_aggregation_latency_post2049", 2049)):
        t0 = _t.time()
        r = study.aggregation_latency_study(device=dev_index, post_taps=taps)
        r.pop("losses", None)
        r["wall_s"] = _t.time() - t0
        out[name] = r
    return out


def train_config(G, torch, dev_index, flush, steps=10, warmup=3):
    """Config 4: one DeepClean training step on 32 windows of 21 x 8192 -
    forward with tape, band-limited PSD-weighted loss (2049-tap weight FIR,
    55-65 Hz), its backward, the hand-written network backward and an Adam
    update of the FP32 master parameters - timed with CUDA events, with and
    without per-block activation checkpointing, and with the weight gradients
    on the tensor cores (BF16 operands, FP32 accumulation)."""
    from paper_2108_12430_gb300 import synth
    Bt, Lt = 32, 8192
    out = {}
    ctx = G.gw_ctx_create(dev_index, 0)
    try:
        _, psd = synth.psd_grid(4096.0, 8192)
        g = G.gw_fir_create_band_loss(ctx, psd, 4096.0, 2049)
        x = torch.from_numpy(np.stack([synth.witness_channels(900 + b, C, Lt) for b in range(Bt)])
                             .astype(np.float32)).cuda()
        s = torch.from_numpy((np.random.default_rng(9).standard_normal((Bt, Lt)) * 0.3).astype(np.float32)).cuda()
        st = torch.cuda.current_stream().cuda_stream
        for ck, prec, tcd, name in ((0, G.GW_FP32, 0, "config4_fp32"), (1, G.GW_FP32, 0, "config4_fp32_checkpoint"),
                                    (0, G.GW_BF16, 0, "config4_bf16_wgrad"), (0, G.GW_BF16, 1, "config4_bf16")):
            t = G.gw_trainer_create(ctx, C, Bt, Lt, ck, precision=prec, tc_data=tcd)
            p = torch.from_numpy(synth.flatten_params(synth.deepclean_params(1234))).cuda()
            m, v, dp = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
            y, dy = torch.empty(Bt, Lt, device="cuda"), torch.empty(Bt, Lt, device="cuda")
            r = torch.empty(Bt, Lt - 2048, device="cuda")
            loss = torch.empty(1, device="cuda")
            it = [0]

            def step():
                it[0] += 1
                G.gw_trainer_forward(t, p.data_ptr(), x.data_ptr(), Bt, y.data_ptr(), st)
                G.gw_band_loss(g, s.data_ptr(), y.data_ptr(), Bt, Lt, loss.data_ptr(), r.data_ptr(), st)
                G.gw_band_loss_backward(g, r.data_ptr(), Bt, Lt, 0, dy.data_ptr(), st)
                G.gw_trainer_backward(t, dy.data_ptr(), dp.data_ptr(), st)
                G.gw_adam_step(p.data_ptr(), dp.data_ptr(), m.data_ptr(), v.data_ptr(), p.numel(), it[0], 1e-4,
                               stream=st)

            l0 = G.gw_launch_count()
            ms = time_call(torch, step, steps, warmup, flush)
            launches = (G.gw_launch_count() - l0) / (steps + warmup)
            G.gw_profile_enable(True)
            for _ in range(3):
                step()
            torch.cuda.synchronize()
            prof = G.gw_profile_read()
            G.gw_profile_enable(False)
            fwd = dc_flops_per_window(Lt) * Bt
            flops = 3 * fwd + (fwd // 2 if ck else 0) + 2 * 2 * 2049 * Bt * (Lt - 2048)
            G.gw_trainer_status(t, st)
            # the same step captured once as a CUDA graph and replayed (Adam
            # reads its step count from device memory)
            step_t = torch.zeros(1, dtype=torch.int32, device="cuda")

            def step_dev(s_):
                G.gw_trainer_forward(t, p.data_ptr(), x.data_ptr(), Bt, y.data_ptr(), s_)
                G.gw_band_loss(g, s.data_ptr(), y.data_ptr(), Bt, Lt, loss.data_ptr(), r.data_ptr(), s_)
                G.gw_band_loss_backward(g, r.data_ptr(), Bt, Lt, 0, dy.data_ptr(), s_)
                G.gw_trainer_backward(t, dy.data_ptr(), dp.data_ptr(), s_)
                G.gw_adam_step_dev(p.data_ptr(), dp.data_ptr(), m.data_ptr(), v.data_ptr(), p.numel(),
                                   step_t.data_ptr(), 1e-4, stream=s_)

            step_dev(st)
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                step_dev(torch.cuda.current_stream().cuda_stream)
            gms = time_call(torch, graph.replay, steps, warmup, flush)
            G.gw_trainer_status(t, st)
            out[name] = {
                "workload": "DeepClean training step, 32 x 21 x 8192, band loss 2049 taps, Adam",
                "weight_gradients": "tensor cores, BF16 operands" if prec == G.GW_BF16 else "FP32 SIMT",
                "forward_and_data_gradients": "tensor cores, BF16 operands" if tcd else "FP32 SIMT",
                "ms_per_step": float(np.mean(ms)), "p50_ms": float(np.median(ms)),
                "windows_per_s": Bt / (np.mean(ms) / 1e3), "tflops": flops / (np.mean(ms) / 1e3) / 1e12,
                "graph_replay_ms_per_step": float(np.mean(gms)),
                "graph_replay_windows_per_s": Bt / (np.mean(gms) / 1e3),
                "flops_per_step": flops, "loss": float(loss.item()), "kernels_per_step": launches,
                "state_bytes": G.gw_trainer_bytes(t),
                "kernels_ms": {k: round(vv[0] / 3, 4) for k, vv in sorted(prof.items(), key=lambda kv: -kv[1][0])}}
            G.gw_trainer_destroy(t)
        G.gw_fir_destroy(g)
    finally:
        G.gw_ctx_destroy(ctx)
    return out


SERVE_STREAMS, SERVE_STRIDES, SERVE_BUDGET = 64, (128, 256, 512), 20 * 2 ** 30
# while a tick runs, the next one is formed only once the running tick is
# expected to end within this lead (snapshots arriving meanwhile join it)
SERVE_FORM_LEAD_US = 60


def serve_configs(G, dev_index, seconds=1.5, precisions=None):
    """Config 5: end-to-end serving of 64 concurrent two-detector streams with
    strides 128 / 256 / 512 (DeepClean 21 x 32768 per detector -> subtract ->
    resample to 2048 Hz -> whiten (2049 taps) -> BBHnet 2 x 2048), per-stream
    state on the device admitted under a 20 GB budget, one CUDA-graph launch
    per tick.  Requests are replayed by the library's native load generator
    through the public submit / wait calls, host buffers in and out, at three
    loads: saturation (every stream always has snapshots queued), Poisson
    arrivals at half the saturated rate, and Poisson arrivals at each stream's
    real-time rate (4096 / stride snapshots/s).  Latency = submit (or
    scheduled arrival) -> results written to the caller's buffers.  A stream
    has at most one snapshot in a tick, so one stream alone cannot go faster
    than the tick rate; the loaded points give every stream the same rate."""
    from paper_2108_12430_gb300 import synth
    out = {}
    fs2, nfft = 2048.0, 8192
    _, psd = synth.psd_grid(fs2, nfft)
    rng = np.random.default_rng(55)
    pool_n, out_n = 16, 1024
    pools = {}
    for S in SERVE_STRIDES:
        wit = synth.witness_channels(77 + S, C, pool_n * S).reshape(C, pool_n, S).transpose(1, 0, 2)
        wit = np.ascontiguousarray(np.stack([wit, wit[::-1]], 1), np.float32)          # [pool][2][C][S]
        strn = np.ascontiguousarray(rng.standard_normal((pool_n, 2, S)) * 0.1, np.float32)
        pools[S] = (wit, strn, np.zeros((out_n, 2, S), np.float32))
    stride_of = np.array([SERVE_STRIDES[i % 3] for i in range(SERVE_STREAMS)])

    def addresses(ids, seq):
        wa, sa, ca = (np.zeros(len(ids), np.uint64) for _ in range(3))
        for S in SERVE_STRIDES:
            sel = stride_of[ids] == S
            w, x, c = pools[S]
            j = seq[sel]
            wa[sel] = w.ctypes.data + (j % pool_n).astype(np.uint64) * np.uint64(2 * C * S * 4)
            sa[sel] = x.ctypes.data + (j % pool_n).astype(np.uint64) * np.uint64(2 * S * 4)
            ca[sel] = c.ctypes.data + (j % out_n).astype(np.uint64) * np.uint64(2 * S * 4)
        return wa, sa, ca

    for name, prec in (("bf16", G.GW_BF16), ("fp32", G.GW_FP32)):
        if precisions and name not in precisions:
            continue
        ctx = G.gw_ctx_create(dev_index, SERVE_BUDGET)
        objs = []
        try:
            dcs = [G.gw_model_create(ctx, G.GW_MODEL_DEEPCLEAN, prec, C,
                                     synth.flatten_params(synth.deepclean_params(1234 + d))) for d in range(2)]
            layers, head = synth.bbhnet_params(3)
            bbh = G.gw_model_create(ctx, G.GW_MODEL_BBHNET, prec, 2, synth.flatten_params(layers, head))
            fdec = G.gw_fir_create_lowpass(ctx, 900.0, 4096.0, 127)
            fw = G.gw_fir_create_whitening(ctx, psd, fs2, 2049)
            objs = [(G.gw_model_destroy, m) for m in dcs + [bbh]] + [(G.gw_fir_destroy, fdec), (G.gw_fir_destroy, fw)]
            srv = G.gw_server_create(ctx, dcs, bbh, fdec, fw, n_det=2, n_witness=C, window=W, max_stride=512,
                                     max_streams=SERVE_STREAMS, max_batch=SERVE_STREAMS, max_pending=4 * SERVE_STREAMS,
                                     agg_mode=G.GW_AGG_AVERAGE, agg_delay=W - 512, bbh_len=2048, max_inflight=2,
                                     form_lead_us=SERVE_FORM_LEAD_US)
            objs.append((G.gw_server_destroy, srv))
            fixed = G.gw_ctx_bytes_in_use(ctx)
            per_stream = G.gw_server_stream_bytes(srv, 256)
            sids = np.array([G.gw_server_open(srv, int(stride_of[i])) for i in range(SERVE_STREAMS)], np.int32)
            seq_next = np.zeros(SERVE_STREAMS, np.int64)

            def replay(ids, t_us):
                seq = np.zeros(len(ids), np.int64)
                for i in range(SERVE_STREAMS):
                    sel = ids == i
                    seq[sel] = seq_next[i] + np.arange(sel.sum())
                    seq_next[i] += sel.sum()
                wa, sa, ca = addresses(ids, seq)
                score = np.zeros(len(ids), np.float32)
                lat = np.zeros(len(ids))
                G.gw_server_stats_read(srv, reset=True)
                t0 = time.perf_counter()
                G.gw_server_replay(srv, sids[ids], t_us, wa, sa, ca, score, lat)
                wall = time.perf_counter() - t0
                st = G.gw_server_stats_read(srv, reset=True)
                assert np.isfinite(score).all()
                return {"snapshots": len(ids), "snapshots_per_s": len(ids) / wall, "wall_s": wall,
                        "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                        "max_us": float(lat.max()), "mean_batch": st["mean_batch"],
                        "kernels_per_tick": st["kernels"] / max(st["ticks"], 1), "ticks": st["ticks"],
                        # where the slowest request's time went: a tick on the device, the wait
                        # for a launch, or the load generator queueing late
                        "max_tick_device_us": st["max_tick_device_us"],
                        "max_launch_wait_us": st["max_launch_wait_us"],
                        "max_submit_late_us": st["max_submit_late_us"],
                        "max_launch_call_us": st["max_launch_call_us"]}

            def saturated(n):
                # every request is due at once: throughput only (its latency
                # is the request's place in the flood)
                n = max(SERVE_STREAMS, n // SERVE_STREAMS * SERVE_STREAMS)
                r = replay(np.tile(np.arange(SERVE_STREAMS), n // SERVE_STREAMS), np.zeros(n))
                return {k: v for k, v in r.items() if not k.endswith("_us")}

            def poisson(total_rate, n, realtime_mix=False):
                # each stream a Poisson source: equal rates, or rates in the
                # ratio of the streams' real-time rates 4096 / stride
                w = 4096.0 / stride_of if realtime_mix else np.ones(SERVE_STREAMS)
                ids = rng.choice(SERVE_STREAMS, size=n, p=w / w.sum())
                return replay(ids, np.cumsum(rng.exponential(1e6 / total_rate, n)))

            saturated(SERVE_STREAMS * 8)  # warm-up
            cal = saturated(SERVE_STREAMS * 32)
            sat = saturated(int(cal["snapshots_per_s"] * seconds))
            half = poisson(0.5 * sat["snapshots_per_s"], int(0.5 * sat["snapshots_per_s"] * seconds))
            high = poisson(0.9 * sat["snapshots_per_s"], int(0.9 * sat["snapshots_per_s"] * seconds))
            rt_rate = float((4096.0 / stride_of).sum())
            rt = poisson(rt_rate, int(rt_rate * seconds), realtime_mix=True)
            for sid in sids:
                G.gw_server_close(srv, int(sid))
            G.gw_server_destroy(srv)
            objs.pop()
            try:
                ticks = tick_profile(G, ctx, dcs, bbh, fdec, fw, pools)
            except G.GwError as e:  # a diagnostic breakdown: its failure is reported, the line still printed
                ticks = {"error": str(e)}
            out[f"config5_{name}"] = {
                "workload": "serving 64 streams x 2 detectors, strides 128/256/512, DeepClean 21x32768 -> subtract "
                            "-> 2x resample -> whiten 2049 taps -> BBHnet 2x2048, AVERAGE delay W-512",
                "streams": SERVE_STREAMS, "budget_bytes": SERVE_BUDGET, "stream_state_bytes": per_stream,
                "fixed_bytes": fixed, "streams_admissible_under_budget": int((SERVE_BUDGET - fixed) // per_stream),
                "saturated": sat, "poisson_half_load": half, "poisson_90pct_load": high,
                "poisson_realtime": dict(rt, rate_per_s=rt_rate), "tick_kernels_eager": ticks,
                "launch": "one CUDA graph per tick (batch bucket), inputs read from pinned mapped host slots",
                "form_lead_us": SERVE_FORM_LEAD_US}
        except G.GwError as e:  # the error is the configuration's result; the other lines still print
            out[f"config5_{name}"] = {"error": str(e)}
        finally:
            for fn, o in reversed(objs):
                try:
                    fn(o)
                except G.GwError:
                    pass  # a server left in an error state still frees what it can
            G.gw_ctx_destroy(ctx)
    return out


def tick_profile(G, ctx, dcs, bbh, fdec, fw, pools, n_ticks=20):
    """Per-kernel device time of one tick at batch 1 and at batch 64, from a
    server launching eagerly (no graph) with the library's event profiler."""
    srv = G.gw_server_create(ctx, dcs, bbh, fdec, fw, n_det=2, n_witness=C, window=W, max_stride=512,
                             max_streams=SERVE_STREAMS, max_batch=SERVE_STREAMS, max_pending=4 * SERVE_STREAMS,
                             agg_mode=G.GW_AGG_AVERAGE, agg_delay=W - 512, bbh_len=2048, max_inflight=1,
                             use_graphs=0, max_wait_us=50_000)  # a tick launches once `batch` snapshots are queued
    res = {}
    try:
        sids = [G.gw_server_open(srv, 256) for _ in range(SERVE_STREAMS)]
        wit, strn, outs = pools[256]
        score = np.zeros(1, np.float32)
        for batch in (1, SERVE_STREAMS):
            # the batching window closes when max_batch snapshots are queued or
            # after 50 ms, so a tick holds exactly `batch` snapshots
            for rep in range(2):  # warm-up, then profiled
                G.gw_profile_enable(rep == 1)
                for t in range(n_ticks):
                    tk = [G.gw_server_submit(srv, sids[i], wit[t % len(wit)], strn[t % len(strn)],
                                             outs[(t * batch + i) % len(outs)], score) for i in range(batch)]
                    for x in tk:
                        G.gw_server_wait(srv, x, 60_000_000)
            prof = G.gw_profile_read()
            G.gw_profile_enable(False)
            tot = sum(v[0] for v in prof.values()) / n_ticks
            res[f"batch{batch}"] = {"sum_kernel_ms_per_tick": tot,
                                    "kernels": {k: round(v[0] / n_ticks * 1e3, 2) for k, v in
                                                sorted(prof.items(), key=lambda kv: -kv[1][0])},
                                    "unit": "us per tick (both detector branches summed)",
                                    "note": "event intervals per kernel; the two detectors' branches run on two "
                                            "streams at once, so a kernel's interval includes time queued behind "
                                            "the other branch (the second detector's ring update waits for SMs "
                                            "held by the first one's network kernel)"}
        for sid in sids:
            G.gw_server_close(srv, sid)
    finally:
        G.gw_server_destroy(srv)
    return res


# ---------------------------------------------------------------------------
# CPU leg: the FP64 oracle on the host.  It is timed for cpu_baseline and the
# reference arm, and its outputs on the bench's own seeded inputs are the
# references of the error fields; nothing else in this file touches the
# oracle, and no GPU result depends on it.
# ---------------------------------------------------------------------------

def cpu_leg_deepclean(wins, params, mean=None, std=None):
    from oracle import nets
    from paper_2108_12430_gb300 import synth
    return nets.deepclean_forward(wins, params, synth.DEEPCLEAN_LAYERS, mean, std)


def cpu_leg_whiten_bbhnet(x, psd, fs, nfft, layers, head):
    """Whitened windows (2049 taps, valid mode) and their BBHnet logits."""
    from oracle import fir as ofir, nets
    from paper_2108_12430_gb300 import synth
    xw = ofir.fir_valid(x, ofir.whitening_fir(psd, fs, nfft, 2049))
    return xw, nets.bbhnet_forward(xw, layers, head, synth.bbhnet_layers())


def oracle_snapshot_seconds(n_windows, seed=4321):
    """Time the FP64 oracle on n_windows consecutive snapshots of the workload."""
    from oracle import nets, stream as ostream
    from paper_2108_12430_gb300 import synth
    params = synth.deepclean_params(1234)
    wit = synth.witness_channels(seed, C, W + (n_windows - 1) * S)
    strain = synth.coupled_strain(seed, wit)
    t0 = time.perf_counter()
    wins = np.stack([wit[:, j * S:j * S + W] for j in range(n_windows)])
    preds = nets.deepclean_forward(wins, params, synth.DEEPCLEAN_LAYERS)
    agg = ostream.aggregate(preds, W, S, ostream.AVERAGE, 0)
    ostream.clean(strain, agg, S, 0)
    return time.perf_counter() - t0


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def cpu_baseline(budget_s=12.0, n_max=1024, seed=4321):
    """The FP64 oracle on the host's cores: consecutive 21 x 32768 snapshot
    windows of one stream (stride 256) spread over one worker process per
    core (each held to one BLAS thread), then the overlap-add aggregation
    (latency W - S) and the subtraction, timed end to end after a warm-up
    round; the sample size is set so that it takes about budget_s."""
    from oracle import pool, stream as ostream
    from paper_2108_12430_gb300 import synth
    workers = pool.host_cores()
    params = synth.deepclean_params(1234)
    wit = synth.witness_channels(seed, C, W + (n_max - 1) * S)
    strain = synth.coupled_strain(seed, wit)
    with pool.DeepCleanPool(wit, W, S, params, synth.DEEPCLEAN_LAYERS, workers=workers, chunk=1) as P:
        t0 = time.perf_counter()
        P.forward(range(workers))  # one window per worker: the rate of one round
        per_round = time.perf_counter() - t0
        n = int(min(n_max, max(workers, int(budget_s / max(per_round, 1e-3)) * workers)))
        t0 = time.perf_counter()
        preds = P.forward(range(n))
        agg = ostream.aggregate_by_window(preds, W, S, ostream.AVERAGE, W - S)
        ostream.clean(strain, agg, S, W - S)
        t = time.perf_counter() - t0
    return {"value": n / t, "unit": "snapshots/s", "cores": workers, "kind": "oracle",
            "sample": f"{n} consecutive 21x32768 windows (stride 256) through the FP64 numpy oracle DeepClean "
                      f"({workers} worker processes, one BLAS thread each) + overlap-add aggregation "
                      f"(delay W-S) + subtraction, {t:.1f} s"}


def cpu_baseline_one_core(n_windows=8):
    """The same oracle in a child process (fork + exec) whose numerical
    libraries are held to one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = f"import bench; bench.oracle_snapshot_seconds(1); print(bench.oracle_snapshot_seconds({n_windows}, seed=4322))"
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=300)
        if r.returncode != 0:
            return {"unavailable": (r.stderr.strip().splitlines() or ["child failed"])[-1][:200]}
        t = float(r.stdout.strip().splitlines()[-1])
    except (subprocess.TimeoutExpired, ValueError, IndexError) as e:
        return {"unavailable": f"{type(e).__name__}: {e}"[:200]}
    return {"value": n_windows / t, "unit": "snapshots/s", "cores": 1, "kind": "oracle",
            "sample": f"{n_windows} consecutive 21x32768 windows (stride 256) through the FP64 numpy oracle "
                      f"DeepClean + aggregation in one thread, {t:.1f} s"}


def reference_arm(args):
    """The method's reference implementation here is the FP64 oracle (the
    paper's method has no runnable code): each step is one round of
    snapshot windows, one per host core, through the oracle's DeepClean,
    then their overlap-add aggregation and subtraction."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import pool, stream as ostream
    from paper_2108_12430_gb300 import synth
    workers = pool.host_cores()
    n_steps = args.warmup + args.steps
    n_win = workers * n_steps
    wit = synth.witness_channels(4321, C, W + (n_win - 1) * S)
    strain = synth.coupled_strain(4321, wit)
    params = synth.deepclean_params(1234)
    ts = []
    with pool.DeepCleanPool(wit, W, S, params, synth.DEEPCLEAN_LAYERS, workers=workers, chunk=1) as P:
        for i in range(n_steps):
            ks = range(i * workers, (i + 1) * workers)
            t0 = time.perf_counter()
            preds = P.forward(ks)
            agg = ostream.aggregate_by_window(preds, W, S, ostream.AVERAGE, 0)
            ostream.clean(strain, agg, S, 0)
            if i >= args.warmup:
                ts.append(time.perf_counter() - t0)
    tot = sum(ts)
    v = args.steps * workers / tot
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "snapshots/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "window": W, "stride": S, "batch": B,
                                        "reference_sample": f"{workers} windows (one per host core) per step"},
        "p50_ms": float(np.percentile(ts, 50) * 1e3), "p99_ms": float(np.percentile(ts, 99) * 1e3),
        "cpu_baseline": {"value": v, "unit": "snapshots/s", "cores": workers, "kind": "oracle",
                         "sample": f"{workers} windows of 21x32768 per step through the FP64 numpy oracle, "
                                   "one worker process per core"},
        "e2e": {"value": v, "unit": "snapshots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gw", "reference"], default="gw")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--only", choices=["bf16", "fp32"], default=None,
                    help="time one path only (profiling)")
    ap.add_argument("--serve-only", action="store_true",
                    help="only the serving configuration (config 5); prints its JSON")
    ap.add_argument("--train-only", action="store_true",
                    help="only the training configuration (config 4); prints its JSON")
    ap.add_argument("--lite", action="store_true",
                    help="timed device pushes only: no e2e, accuracy, CPU baseline or JSON contract line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.train_only:
        from paper_2108_12430_gb300 import build as Bld
        Bld.build()
        from paper_2108_12430_gb300 import gwstream as G
        import torch
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
        print(json.dumps(train_config(G, torch, torch.cuda.current_device(), flush)))
    elif args.serve_only:
        from paper_2108_12430_gb300 import build as Bld
        Bld.build()
        from paper_2108_12430_gb300 import gwstream as G
        import torch
        print(json.dumps(serve_configs(G, torch.cuda.current_device(), precisions=args.only and [args.only])))
    elif args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
