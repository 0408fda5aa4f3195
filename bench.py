#!/usr/bin/env python
"""Throughput of the spherical-harmonic transform dwarf on GB300.

One step = one spectral-transform timestep of the TCo1279 workload (octahedral
grid O1280, 137 levels): 137 (vorticity, divergence) pairs -> winds (u, v) and
274 scalars -> (field, d/dphi) on the grid (inverse), then the winds -> (vor,
div) and the scalars -> spectra (direct).  548 spectral fields go through
inverse + direct each step; the metric is those fields per second.  Inputs are
seeded synthetic spectra ((n+1)^-1.5 complex Gaussians), resident in HBM
before the timed region and larger than L2 (no flush needed).

Output: one JSON line (rank 0).  Extra keys: roofline of the dominant kernel
(CUDA events on the launching stream, inside the timed region), the FP64 CPU
oracle on a bounded sample (cpu_baseline), end-to-end through the C ABI from
pinned host buffers (e2e), error vs the FP64 oracle, clocks during the timed
region, kernel launches.

--impl reference times the FP64 CPU oracle (the reference of this project) on
the host cores, on a bounded sample of the same workload per step.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fields/sec inverse+direct at TCo1279 137 lev, 1 GB300; % roofline; err vs FP64"
UNIT = "fields/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons for one GPU."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                pw.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_median": statistics.median(pw) if pw else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value, world):
    """Max of a float over ranks (identity on one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(fields_per_rank, steps, world, max_ms):
    """Whole-job fields/s: the fields of every rank over the slowest rank's time."""
    return world * fields_per_rank * steps / (max_ms / 1e3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ------------------------------------------------------------------- workload
def legendre_flops(plan_T, L, nleg, nmax):
    """4 * sum_m (# n in [m, nmax]) * L_m * nleg: 2 flops per multiply-add on
    the real and the imaginary column of each Legendre field."""
    tot = 0
    for m in range(plan_T + 1):
        tot += (nmax - m + 1) * L[m]
    return 4.0 * tot * nleg


def northern_counts(T, N):
    """L_m: northern octahedral rings whose truncation mmax_i = min(T, 2i+7) reaches m."""
    mmax = np.minimum(T, 2 * np.arange(1, N + 1) + 7)
    return [int((mmax >= m).sum()) for m in range(T + 1)]


class Workload:
    def __init__(self, T, levels, prec, timing=True, seed_base=None):
        import torch

        from paper_1908_06097_gb300 import inputs, st

        self.T, self.levels, self.prec = T, levels, prec
        self.timing = timing
        # Legendre tile widths autotuned at plan creation (outside the timed region);
        # "fp64otf": the FP64 path with on-the-fly Legendre functions (no stored table)
        flags = st.FLAG_AUTOTUNE | (st.FLAG_STAGE_TIMING if timing else 0)
        if prec == "fp64otf":
            prec, flags = "fp64", flags | st.FLAG_OTF
        elif prec == "fp64df":  # FP64 plans with double-float Legendre contractions
            prec, flags = "fp64", flags | st.FLAG_DF64
        self.uv = st.Plan(T, levels, prec=prec, flags=flags)
        self.sc = st.Plan(T, 2 * levels, prec=prec, flags=flags)
        sb = inputs.SEED_BASE + 2 if seed_base is None else seed_base
        self.h_vor = inputs.spectral_fields(T, levels, sb)
        self.h_div = inputs.spectral_fields(T, levels, sb + 100)
        self.h_s = inputs.spectral_fields(T, 2 * levels, sb + 200)
        self.vor = torch.from_numpy(self.h_vor).cuda()
        self.div = torch.from_numpy(self.h_div).cuda()
        self.s = torch.from_numpy(self.h_s).cuda()
        self.u, self.v = self.uv.grid_empty(), self.uv.grid_empty()
        self.g, self.dp = self.sc.grid_empty(), self.sc.grid_empty()
        self.vor2, self.div2 = self.uv.spec_empty(), self.uv.spec_empty()
        self.s2 = self.sc.spec_empty()
        self.fields = 4 * levels
        self.launches = 0

    def step(self, stream=None, io=None):
        """One timestep; io = (vor, div, s, vor2, div2, s2) device arrays in
        place of the workload's own."""
        vor, div, s, vor2, div2, s2 = io or (self.vor, self.div, self.s, self.vor2, self.div2, self.s2)
        self.uv.inv_uv(vor, div, self.u, self.v, stream)
        n = self.uv.last_launches()
        self.sc.inv_deriv(s, self.g, None, self.dp, stream)
        n += self.sc.last_launches()
        self.uv.dir_uv(self.u, self.v, vor2, div2, stream)
        n += self.uv.last_launches()
        self.sc.dir(self.g, s2, stream)
        n += self.sc.last_launches()
        self.launches = n
        return n

    def stage_times(self):
        ms, ln = [0.0] * 6, [0] * 6
        for p in (self.uv, self.sc):
            a, b = p.stage_times()
            ms = [x + y for x, y in zip(ms, a)]
            ln = [x + y for x, y in zip(ln, b)]
        return ms, ln

    def stage_reset(self):
        if self.timing:
            self.stage_times()

    def stage_work(self):
        """Algorithmic work per stage for one step: (flops, bytes)."""
        T, lv, N = self.T, self.levels, self.T + 1
        L = northern_counts(T, N)
        eb = 8 if self.prec in ("fp64", "fp64otf", "fp64df") else 4
        npts = self.uv.npts
        nfour = sum(min(T, (4 * i + 16) // 2 - 1) + 1 for i in range(1, N + 1)) * 2
        ncoef = self.uv.ncoef
        leg_inv = legendre_flops(T, L, 2 * lv, T + 1) + legendre_flops(T, L, 4 * lv, T + 1)
        leg_dir = legendre_flops(T, L, 2 * lv, T + 1) + legendre_flops(T, L, 2 * lv, T)
        # FFT stages move the grid (float64) and the Fourier coefficients (complex, eb)
        c2r_bytes = (6 * lv) * (npts * 8 + nfour * 2 * eb)
        r2c_bytes = (4 * lv) * (npts * 8 + nfour * 2 * eb)
        pre_bytes = (4 * lv) * ncoef * 16 + (6 * lv) * ncoef * 2 * eb
        post_bytes = (4 * lv) * ncoef * 16 + (4 * lv) * ncoef * 2 * eb
        return {0: (0, pre_bytes), 1: (leg_inv, 0), 2: (0, c2r_bytes), 3: (0, r2c_bytes), 4: (leg_dir, 0),
                5: (0, post_bytes)}

    def close(self):
        self.uv.close()
        self.sc.close()


STAGE_NAMES = ["pre", "leg_inv", "c2r", "r2c", "leg_dir", "post"]

# DRAM bytes (read + write) per grid point and grid field of the c2r stage,
# from an ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of both
# BF16X6 c2r launches of one TCo1279 / 137-level step: 61.13 GB for 822 grid
# fields.  Valid for the kernel of that capture only.
NCU_DRAM_BYTES_PER_POINT = {"bf16x6": {"c2r": 11.27}}
# grid fields per step of each ring-FFT stage, per level: c2r writes u, v, s1,
# s2, d/dphi s1, d/dphi s2; r2c reads u, v, s1, s2
GRID_FIELDS_PER_LEVEL = {"c2r": 6, "r2c": 4}


def time_steps(wl, steps, warmup, world, stream):
    import torch

    for _ in range(warmup):
        wl.step(stream)
    torch.cuda.synchronize()
    wl.stage_reset()
    barrier(world)
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    launches = 0
    evs[0].record(stream)
    for k in range(steps):
        launches += wl.step(stream)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    per = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
    total = evs[0].elapsed_time(evs[steps])
    return total, per, launches


def oracle_sample(T, h_s):
    """FP64 CPU oracle on one scalar field: inverse with d/dphi, then direct."""
    import oracle

    oracle.build()
    t0 = time.perf_counter()
    g, _, dp = oracle.inverse(T, 0, T + 1, h_s[:1], deriv=True)
    s2 = oracle.direct(T, 0, T + 1, g)
    dt = time.perf_counter() - t0
    return dt, g, dp, s2, oracle.num_threads()


def relmax(x, ref):
    return float(np.abs(x - ref).max() / max(np.abs(ref).max(), 1e-300))


def run_ours(args):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1908_06097_gb300 import st

    st.load()
    pk, pk_src = peaks()
    T, lv, prec = args.T, args.levels, args.prec
    wl = Workload(T, lv, prec)
    stream = torch.cuda.current_stream()
    clk = ClockSampler(local)
    # warm-up + timed region (clocks sampled during it)
    for _ in range(args.warmup):
        wl.step(stream)
    torch.cuda.synchronize()
    clk.start()
    total_ms, per_ms, launches = time_steps(wl, args.steps, 0, world, stream)
    clocks = clk.stop()
    stage_ms, stage_n = wl.stage_times()
    total_max = reduce_max(total_ms, world)
    value = job_throughput(wl.fields, args.steps, world, total_max)
    # roofline of the dominant stage
    work = wl.stage_work()
    dom = int(np.argmax(stage_ms))
    fl, by = work[dom]
    per_launch_ms = stage_ms[dom] / max(stage_n[dom], 1)
    launches_per_step = stage_n[dom] / args.steps
    if fl > 0:
        achieved = fl / launches_per_step / (per_launch_ms / 1e3) / 1e12
        if prec in ("bf16x3", "bf16x6"):
            bound, peak, unit = "tensor", pk.get("bf16_tflops_sustained", 1700.0), "TFLOP/s"
        elif prec == "fp32":
            bound, peak, unit = "alu", 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12, "TFLOP/s"
        elif prec == "fp64df":
            # FP32 issue rate / 12.75 FP32 operations per double-float multiply-add
            # (12, and a 3-operation renormalisation every 4)
            bound, peak, unit = "alu", 152 * 128 * 2 / 12.75 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12, "TFLOP/s"
        else:
            bound, peak, unit = "alu", 152 * 2 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12, "TFLOP/s"
    else:
        achieved = by / launches_per_step / (per_launch_ms / 1e3) / 1e9
        bound, peak, unit = "hbm", pk.get("hbm_gbs", 6800.0), "GB/s"
    traffic = None
    per_pt = NCU_DRAM_BYTES_PER_POINT.get(prec, {}).get(STAGE_NAMES[dom])
    if per_pt and launches_per_step > 0:
        fields_per_launch = GRID_FIELDS_PER_LEVEL[STAGE_NAMES[dom]] * lv / launches_per_step
        traffic = round(per_pt * wl.uv.npts * fields_per_launch)
    roofline = {"bound": bound, "kernel": STAGE_NAMES[dom], "achieved": round(achieved, 3), "peak": round(peak, 3),
                "unit": unit, "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": pk_src if bound != "alu" else "derived from unit counts and max SM clock",
                "launch_ms": round(per_launch_ms, 4)}
    stages = {STAGE_NAMES[i]: {"ms_per_step": round(stage_ms[i] / args.steps, 3),
                               "launches_per_step": stage_n[i] / args.steps} for i in range(6)}
    for i in range(6):
        fl, by = work[i]
        t = stage_ms[i] / args.steps / 1e3
        if t > 0:
            if fl:
                stages[STAGE_NAMES[i]]["tflops"] = round(fl / t / 1e12, 3)
            else:
                stages[STAGE_NAMES[i]]["gbs"] = round(by / t / 1e9, 1)
    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(total_max / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp64": "f64", "fp64otf": "f64", "fp64df": "f64 (Legendre in f32 pairs)", "fp32": "f32", "bf16x3": "bf16x3",
                     "bf16x6": "bf16x6"}[prec],
           "data": "synthetic",
           "config": {"workload": f"TCo{T} O{T + 1} {lv} levels: vor/div->u,v + 2 scalars with d/dphi, "
                                  "inverse+direct", "T": T, "grid": f"O{T + 1}", "levels": lv,
                      "fields_per_step": wl.fields, "precision": prec, "parallelism": f"replica x{world}",
                      "l2": "inputs larger than L2 (no flush)",
                      "leg_tile_widths": {"winds": wl.uv.tuning(), "scalars": wl.sc.tuning()}},
           "roofline": roofline, "stages": stages, "gpu_launches": launches, "clocks": clocks}
    # error vs the FP64 oracle and the CPU baseline (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.no_oracle:
        dt, g_ref, dp_ref, s_ref, cores = oracle_sample(T, wl.h_s)
        torch.cuda.synchronize()
        err = {"grid": relmax(wl.g[0].cpu().numpy(), g_ref[0]), "dphi": relmax(wl.dp[0].cpu().numpy(), dp_ref[0]),
               "round_trip_spec": relmax(wl.s2[0].cpu().numpy(), s_ref[0]),
               "sample": "scalar field 0 (inverse with d/dphi, then direct of the GPU grid) vs the FP64 oracle"}
        out["err_vs_fp64"] = err
        out["cpu_baseline"] = {"value": round(1.0 / dt, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"1 scalar field of the TCo{T} workload (inverse with d/dphi + direct), "
                                         f"{dt:.1f} s on {cores} host threads"}
    # end to end through the C ABI from pinned host buffers
    if not args.no_e2e:
        out["e2e"] = run_e2e(wl, args, world, stream)
    wl.close()
    del wl
    torch.cuda.empty_cache()
    others = {}
    for op in [c for c in args.compare.split(",") if c and c != prec]:
        wlo = Workload(T, lv, op, timing=False)
        to, _, _ = time_steps(wlo, 1, 1, world, stream)
        fo = wlo.fields / (to / 1e3)
        others[op] = {"fields_per_s": round(fo, 3), "ms_per_step": round(to, 1),
                      "speedup_of_this_path": round(value / world / fo, 2)}
        if rank == 0 and world == 1 and not args.no_oracle:
            torch.cuda.synchronize()
            others[op]["err_vs_fp64"] = {"grid": relmax(wlo.g[0].cpu().numpy(), g_ref[0]),
                                         "dphi": relmax(wlo.dp[0].cpu().numpy(), dp_ref[0]),
                                         "round_trip_spec": relmax(wlo.s2[0].cpu().numpy(), s_ref[0])}
        wlo.close()
        del wlo
        torch.cuda.empty_cache()
    if others:
        out["other_paths"] = others
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def run_e2e(wl, args, world, stream):
    """End to end from pinned host memory: every step copies its spectral
    inputs host -> device, transforms them through the C ABI and copies the
    resulting spectra device -> host.  The device inputs and outputs are
    double-buffered and all copies run, in order, on one copy stream of their
    own: the input copy of step k + 2, then the output copy of step k, both
    while step k + 1 computes.  The two directions never run at once: on this
    GPU's host link one direction alone moves about 200 GB/s, both at once
    about 85 GB/s together.  The timed region runs from the first input copy
    to the end of the last output copy."""
    import torch

    hv = torch.from_numpy(wl.h_vor).pin_memory()
    hd = torch.from_numpy(wl.h_div).pin_memory()
    hs = torch.from_numpy(wl.h_s).pin_memory()
    ov = torch.empty_like(hv).pin_memory()
    od = torch.empty_like(hd).pin_memory()
    os_ = torch.empty_like(hs).pin_memory()
    steps = max(args.steps, 6)
    sets = [(wl.vor, wl.div, wl.s, wl.vor2, wl.div2, wl.s2),
            (torch.empty_like(wl.vor), torch.empty_like(wl.div), torch.empty_like(wl.s),
             torch.empty_like(wl.vor2), torch.empty_like(wl.div2), torch.empty_like(wl.s2))]
    s_copy = torch.cuda.Stream()
    in_ready = [torch.cuda.Event(), torch.cuda.Event()]
    out_done = [torch.cuda.Event(), torch.cuda.Event()]
    comp_done = [torch.cuda.Event(), torch.cuda.Event()]
    hin, hout = (hv, hd, hs), (ov, od, os_)

    def h2d(k):  # inputs of step k into set k % 2, once step k - 2 has read that set
        b = k % 2
        with torch.cuda.stream(s_copy):
            if k >= 2:
                s_copy.wait_event(comp_done[b])
            for a in range(3):
                sets[b][a].copy_(hin[a], non_blocking=True)
            in_ready[b].record(s_copy)

    def compute(k):  # set k % 2, once its inputs are in and its outputs of step k - 2 are out
        b = k % 2
        stream.wait_event(in_ready[b])
        if k >= 2:
            stream.wait_event(out_done[b])
        wl.step(stream, sets[b])
        comp_done[b].record(stream)

    def d2h(k):
        b = k % 2
        with torch.cuda.stream(s_copy):
            s_copy.wait_event(comp_done[b])
            for a in range(3):
                hout[a].copy_(sets[b][3 + a], non_blocking=True)
            out_done[b].record(s_copy)

    def run(n):
        h2d(0)
        h2d(1)
        for k in range(n):
            compute(k)
            if k + 2 < n:
                h2d(k + 2)
            d2h(k)

    run(2)  # warm-up
    torch.cuda.synchronize()
    # copies out of freshly pinned host buffers run several times slower than
    # later ones (measured: 160-450 ms against 34 ms for the 7.2 GB of inputs),
    # so each buffer is copied a few more times before the timed region.  (Some
    # later input copies also take 250-340 ms, with or without a transform
    # running beside them: the e2e figure varies with the host side.)
    for _ in range(3):
        h2d(0)
        h2d(1)
        d2h(0)
        d2h(1)
    torch.cuda.synchronize()
    barrier(world)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    s_copy.wait_event(t0)
    run(steps)
    stream.wait_stream(s_copy)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = reduce_max(t0.elapsed_time(t1), world)
    h2d_bytes = (hv.numel() + hd.numel() + hs.numel()) * 8
    d2h_bytes = (ov.numel() + od.numel() + os_.numel()) * 8
    return {"value": round(world * wl.fields * steps / (ms / 1e3), 3), "unit": UNIT, "h2d_bytes_per_step": h2d_bytes,
            "d2h_bytes_per_step": d2h_bytes, "steps": steps,
            "overlap": "double-buffered device I/O; one copy stream: the input copy of step k+2 and the output "
                       "copy of step k run while step k+1 computes, never both directions at once"}


def run_group(args):
    """The mixed-group workload: 64 independent transforms, truncations drawn
    from {79, 159, 319, 639} and 1..137 levels each (seed 1908060975), run as
    one group (one kernel launch per stage) captured in a CUDA graph; inverse
    then direct of every member per step.  Tile widths autotuned.  Beside it:
    the same 64 transforms as separate plan calls (also one CUDA graph), and
    the group in the --compare precisions."""
    import torch

    from paper_1908_06097_gb300 import inputs, st

    torch.cuda.set_device(0)
    st.load()
    rng = np.random.default_rng(inputs.SEED_BASE + 5)
    Ts = rng.choice([79, 159, 319, 639], size=64)
    lv = rng.integers(1, 138, size=64)
    fields = int(lv.sum())
    specs = [torch.from_numpy(inputs.spectral_fields(int(T), int(L), inputs.SEED_BASE + 5 + i)).cuda()
             for i, (T, L) in enumerate(zip(Ts, lv))]
    stream = torch.cuda.Stream()

    def capture(fn):
        stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(stream):  # first-call set-up outside the capture
            fn()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            fn()
        return graph

    def timed(graph, steps, warmup):
        for _ in range(warmup):
            graph.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(steps):
                graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def setup(prec):
        plans = [st.Plan(int(T), int(L), prec=prec, flags=st.FLAG_AUTOTUNE) for T, L in zip(Ts, lv)]
        g = st.Group(plans)
        grids = [p.grid_empty() for p in plans]
        outs = [p.spec_empty() for p in plans]
        return plans, g, grids, outs

    def teardown(plans, g):
        g.close()
        for p in plans:
            p.close()
        torch.cuda.empty_cache()

    plans, g, grids, outs = setup(args.prec)
    launches = []

    def grouped():
        g.inv(specs, grids, stream)
        n = g.last_launches()
        g.dir(grids, outs, stream)
        launches[:] = [n + g.last_launches()]

    def separate():
        for p, a, gr, o in zip(plans, specs, grids, outs):
            p.inv(a, gr, stream)
            p.dir(gr, o, stream)

    ms = timed(capture(grouped), args.steps, args.warmup)
    n_group = launches[0]
    ms_sep = timed(capture(separate), args.steps, args.warmup)
    n_sep = 0
    for p, a, gr, o in zip(plans, specs, grids, outs):
        p.inv(a, gr, stream)
        n_sep += p.last_launches()
        p.dir(gr, o, stream)
        n_sep += p.last_launches()
    torch.cuda.synchronize()
    tiles = plans[0].tuning()
    teardown(plans, g)
    out = {"metric": "fields/sec inverse+direct, 64-transform mixed group (one launch per stage, CUDA graph)",
           "value": round(fields / (ms / 1e3), 3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp64": "f64", "fp32": "f32", "bf16x3": "bf16x3", "bf16x6": "bf16x6"}[args.prec],
           "data": "synthetic",
           "config": {"workload": "64 transforms, T in {79,159,319,639}, 1-137 levels (seed 1908060975)",
                      "fields_per_step": fields, "truncations": {str(t): int((Ts == t).sum()) for t in (79, 159, 319, 639)},
                      "launches_per_step": n_group, "leg_tile_widths": tiles,
                      "l2": "working set above L2 (no flush)"},
           "gpu_launches": n_group * args.steps,
           "separate_plans": {"fields_per_s": round(fields / (ms_sep / 1e3), 3), "ms_per_step": round(ms_sep, 3),
                              "launches_per_step": n_sep,
                              "what": "the same 64 transforms as plan calls, one after another in one CUDA graph"}}
    others = {}
    for op in [c for c in args.compare.split(",") if c and c != args.prec and c not in ("fp64otf", "fp64df")]:
        plans, g, grids, outs = setup(op)
        mso = timed(capture(grouped), 1, 1)
        others[op] = {"fields_per_s": round(fields / (mso / 1e3), 3), "ms_per_step": round(mso, 1),
                      "launches_per_step": launches[0], "speedup_of_this_path": round(mso / ms, 2)}
        teardown(plans, g)
    if others:
        out["other_paths"] = others
    print(json.dumps(out), flush=True)


def run_errors(args):
    """The TCo639 precision comparison: 411 fields (137 levels x 3) through each
    precision; max and RMS relative error per field against the FP64 oracle on
    fields 0, 137, 274, 410, for the inverse and for the direct of the oracle's
    grid."""
    import torch

    import oracle
    from paper_1908_06097_gb300 import inputs, st

    torch.cuda.set_device(0)
    st.load()
    oracle.build()
    T, nf, pick = 639, 411, [0, 137, 274, 410]
    a = inputs.spectral_fields(T, nf, inputs.SEED_BASE + 1)
    g_ref = oracle.inverse(T, 0, T + 1, a[pick])
    s_ref = oracle.direct(T, 0, T + 1, g_ref)
    g_in = np.zeros((nf, g_ref.shape[1]))
    g_in[pick] = g_ref

    def errs(x, ref):
        mx = [float(np.abs(x[i] - ref[i]).max() / np.abs(ref[i]).max()) for i in range(len(ref))]
        rms = [float(np.linalg.norm(x[i] - ref[i]) / np.linalg.norm(ref[i])) for i in range(len(ref))]
        return {"max_rel": max(mx), "rms_rel": max(rms)}

    res = {}
    for prec in ("fp64", "fp64df", "fp32", "bf16x3", "bf16x6"):
        p = st.Plan(T, nf, prec="fp64", flags=st.FLAG_DF64) if prec == "fp64df" else st.Plan(T, nf, prec=prec)
        gd = p.grid_empty()
        p.inv(torch.from_numpy(a).cuda(), gd)
        sd = p.spec_empty()
        p.dir(torch.from_numpy(g_in).cuda(), sd)
        torch.cuda.synchronize()
        res[prec] = {"inverse": errs(gd.cpu().numpy()[pick], g_ref), "direct": errs(sd.cpu().numpy()[pick], s_ref)}
        p.close()
        torch.cuda.empty_cache()
    print(json.dumps({"workload": "TCo639 O640, 411 fields (137 levels x 3); errors vs the FP64 oracle on fields "
                                  "0, 137, 274, 410", "errors": res}), flush=True)


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_1908_06097_gb300 import inputs

    T = args.T
    h_s = inputs.spectral_fields(T, 1, inputs.SEED_BASE + 2 + 200)
    for _ in range(args.warmup):
        oracle_sample(T, h_s)
    ts = []
    cores = 1
    for _ in range(args.steps):
        dt, _, _, _, cores = oracle_sample(T, h_s)
        ts.append(dt)
    value = args.steps / sum(ts)
    sample = (f"1 scalar field of the TCo{T} workload per step (inverse with d/dphi + direct), FP64 CPU oracle "
              f"on {cores} host threads")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(ts) / len(ts), 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"TCo{T} O{T + 1} {args.levels} levels: vor/div->u,v + 2 scalars with d/dphi, "
                                  "inverse+direct", "T": T, "grid": f"O{T + 1}", "levels": args.levels},
           "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x6", choices=["fp64", "fp64otf", "fp64df", "fp32", "bf16x3", "bf16x6"])
    ap.add_argument("--T", type=int, default=1279)
    ap.add_argument("--levels", type=int, default=137)
    ap.add_argument("--no-oracle", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="tco1279", choices=["tco1279", "group", "errors"],
                    help="tco1279: the headline line; group: the 64-transform mixed group; errors: TCo639 error table")
    ap.add_argument("--compare", default="fp64,fp64otf,fp64df",
                    help="comma-separated other precisions timed for one step after the main run ('' for none)")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "group":
        run_group(args)
    elif args.workload == "errors":
        run_errors(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
