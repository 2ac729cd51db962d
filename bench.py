#!/usr/bin/env python3
"""Throughput benchmark of the CheFSI hot path (H*X point-orbital updates per second).

One step = one complete CheFSI solve of a synthetic cluster on a fixed Hamiltonian, the
first-SCF-step regime of the paper (Sec. 3.4): k Lanczos steps for the spectral bounds,
then `iters` CheFSI iterations (Chebyshev filter of degree m, projection, Rayleigh-Ritz,
rotation), starting from the same resident random block each step. The work unit is the
point-orbital update: one grid node of one column under one application of H, so a step
holds k*Nd + iters*(m+1)*Nd*Ns of them.

Default workload: 96^3 grid, h = 0.3 bohr, 40 atoms, Ns = 128, m = 20, 20 iterations,
FP64 (the medium cluster). Inputs are larger than L2 (the 128-column FP64 block is
0.91 GB), so no L2 flush is needed between steps.

Under torchrun (N > 1) each rank solves its own replica on its own GPU (replicas only:
the path has no data exchange), times are max-reduced over ranks and `value` sums the
ranks' work.

Three more objects follow on one GPU (N = 1), after the timed region: `mixed160`, the large
cluster (160^3, 400 atoms, Ns = 1024, degree 24) solved in the mixed-precision form and in
the FP64 form on the same GPU from the same start (times, speed-up, Ritz-value differences
of the converged states, the FP32 filter step's HBM fraction), `batching` (the batched
filter of 64 uneven clusters against per-cluster launches) and `serving`, the request loop
under Poisson arrivals (p50/p99 latency and throughput at the configured and at
sub-saturation rates, beside serial FP64 solves). Together they take about 25 minutes;
--no-mixed160, --no-batching and --serving-requests 0 skip them.

--impl reference times the FP64 CPU oracle instead (on the host cores, rank 0 only),
each step one CheFSI iteration of the same workload on a column slice, set up once.
"""
from __future__ import annotations

import argparse
import hashlib
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

from paper_1603_04334_gb300 import synth  # noqa: E402

METRIC = "H*X point-orbitals/s"
UNIT = "point-orbitals/s"
ORACLE_COLS = 16      # column slice of the block the oracle timing runs on
SM_COUNT = 152
# kernel sources whose DRAM traffic the committed ncu summary was taken on, per dtype
STENCIL_SOURCES = {"f64": ("stencil_df.cu", "df.cuh", "fx.cuh"),
                   "f32": ("stencil_tma.cu",)}


def reduce_max(value_ms: float, world: int, device=None) -> float:
    """Max over ranks of a per-rank time (the slowest replica sets the job time)."""
    if world <= 1:
        return value_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([value_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(work_per_rank_step: int, steps: int, world: int, ms: float) -> float:
    """Whole-job throughput: every rank's units over the max-over-ranks time."""
    return work_per_rank_step * steps * world / (ms / 1e3)


def work_per_step(w, dtype: str = "f64") -> int:
    """Point-orbital updates of one solve: k Lanczos applications of H to one vector, and
    m + 1 applications to the block per CheFSI iteration (m filter steps, H Y_f in the
    Rayleigh-Ritz step); the mixed form adds its FP64 refinement iteration."""
    its = w.iters + (1 if dtype == "f32" else 0)
    return w.lanczos_k * w.nd + its * (w.degree + 1) * w.nd * w.ns


def workload_config(w, dtype: str) -> dict:
    form = ("FP32 filter, FP64 Rayleigh-Ritz, + 1 FP64 refinement iteration" if dtype == "f32"
            else "FP64")
    return {"workload": f"{w.name}: {w.n}^3 grid h={w.h} bohr, {w.natoms} atoms, Ns={w.ns}, "
                        f"Chebyshev degree {w.degree}, {w.iters} CheFSI iterations, {form}",
            "n": w.n, "h": w.h, "natoms": w.natoms, "ns": w.ns, "degree": w.degree,
            "iters": w.iters, "lanczos_k": w.lanczos_k, "dtype": dtype,
            "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas"}


# ----------------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------------
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------
# roofline helpers
# ----------------------------------------------------------------------------------
def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def fp64_alu_peak_tflops(sm_max_mhz: float = 2070.0) -> float:
    # 152 SMs x 2 FP64 FMA lanes per SM per clock (1.25 TFLOP/s nominal at 2.07 GHz;
    # measured 0.595e12 DFMA/s at 1.99 GHz) x 2 flop per FMA.
    return SM_COUNT * 2 * 2 * sm_max_mhz * 1e6 / 1e12


def stencil_traffic(dtype: str):
    """DRAM bytes per stencil launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "stencil_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    h = hashlib.sha256()
    srcs = STENCIL_SOURCES.get(dtype, ())
    for fn in srcs:
        with open(os.path.join(ROOT, "paper_1603_04334_gb300", "csrc", fn), "rb") as g:
            h.update(g.read())
    ent = d.get(dtype)
    if not ent or ent.get("source_sha256") != h.hexdigest():
        return None
    return ent


def stencil_algorithmic(w, dtype: str, prof: dict, steps: int) -> dict:
    """Algorithmic bytes and flops of all stencil launches of the timed steps.

    Per point-orbital a filter step reads Y_j and Y_{j-1} and writes Y_{j+1} (3 elements);
    the first step of a filter and an H X read one block and write one (2 elements); each
    launch also reads the potential once per node (8 B: alpha (V_eff - shift) in FP64 in the
    FP64 kernel, 4 B in the FP32 kernel). Flops per point-orbital: 6 radii x (5 adds + 1 FMA) + centre
    (1 FMA + 1 multiply) + recurrence (1 FMA) = 47 (45 without the recurrence term).
    FP64 form per iteration: 2-stream first step, m - 1 3-stream steps, 2-stream H Y_f, all
    FP64. Mixed form per FP32 iteration: FP32 steps (4-byte elements) and the FP64 H Y_f of
    the FP32 block (4 B in, 8 B out); then one FP64 refinement iteration. Lanczos: k
    single-column FP64 H x."""
    nd, ns, m = w.nd, w.ns, w.degree

    def iteration(ein: int, eh_in: int, eh_out: int, vbytes_step: int):
        # ein: element bytes of the filter steps; eh_*: bytes of the H Y_f launch
        b = nd * ns * (2 * ein + (m - 1) * 3 * ein + eh_in + eh_out) + nd * (m * vbytes_step + 8)
        f = nd * ns * (45 + (m - 1) * 47 + 45)
        return b, f

    if dtype == "f64":
        b1, f1 = iteration(8, 8, 8, 8)
        it_b, it_f = w.iters * b1, w.iters * f1
    else:
        b1, f1 = iteration(4, 4, 8, 4)
        b2, f2 = iteration(8, 8, 8, 8)
        it_b, it_f = w.iters * b1 + b2, w.iters * f1 + f2
    lz_bytes = w.lanczos_k * nd * (2 * 8 + 8)
    lz_flops = w.lanczos_k * nd * 45
    n_launch, ms = prof["stencil"]
    return {"bytes": steps * (it_b + lz_bytes), "flops": steps * (it_f + lz_flops),
            "launches": n_launch, "ms": ms}


# ----------------------------------------------------------------------------------
# our implementation
# ----------------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1603_04334_gb300 import sparc

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = synth.preset(args.workload)
    dtype = args.dtype or w.filter_dtype
    tdt = torch.float64 if dtype == "f64" else torch.float32
    cl = synth.make_cluster(w, args.seed)
    stream = torch.cuda.current_stream(dev)
    ctx = sparc.Context(cl.n, cl.h, cl.R, cl.Z, cl.gamma, veff=None, sigma=cl.sigma,
                        rcut=cl.rcut, rc_erf=cl.rc_erf, stream=stream)
    X0h = synth.initial_block(args.seed + 1, w.nd, w.ns)
    X0 = torch.from_numpy(X0h).to(dev, dtype=tdt)
    X = torch.empty_like(X0)
    W = torch.empty_like(X0)
    mixed = dtype == "f32"
    X64 = torch.empty(X0.shape, dtype=torch.float64, device=dev) if mixed else None
    W64 = torch.empty_like(X64) if mixed else None

    def solve(Xsrc):
        X.copy_(Xsrc, non_blocking=True)
        b = ctx.first_bounds(w.lanczos_k, args.seed)
        ritz = resid = None
        for it in range(w.iters):
            last = it == w.iters - 1 and not mixed
            ritz, resid, b = ctx.chefsi_step(X, W, w.degree, b, want_resid=last)
        if mixed:  # refinement sweep: one FP64 iteration from the FP32 result
            X64.copy_(X)
            ritz, resid, b = ctx.chefsi_step(X64, W64, w.degree, b, want_resid=True)
        return ritz, resid

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        solve(X0)
    torch.cuda.synchronize()

    # ---- device-timed region: inputs resident in HBM -------------------------------
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    smi_index = int(vis[local_rank]) if local_rank < len(vis) and vis[local_rank].isdigit() \
        else local_rank
    clocks = ClockSampler(smi_index)
    ctx.profile_reset()
    ctx.profile_enable(True)
    n0 = sparc.launch_count()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        ritz, resid = solve(X0)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    launches = sparc.launch_count() - n0
    ms = ev0.elapsed_time(ev1)
    ctx.profile_enable(False)
    prof = ctx.profile_read()
    ms = reduce_max(ms, world, dev)
    work = work_per_step(w, dtype) * args.steps * world
    value = job_value(work_per_step(w, dtype), args.steps, world, ms)

    # ---- end-to-end: the start block from pinned host memory to the device and the
    # solved orbitals (and Ritz values, residuals, bounds) back to the host, every step ---
    e2e = None
    Xpin = Xout = Xres = None
    if not args.no_e2e:
        Xpin = torch.from_numpy(X0h).to(dtype=tdt).pin_memory()
        Xres = X64 if mixed else X                  # the solve's result block
        Xout = torch.empty(Xres.shape, dtype=Xres.dtype).pin_memory()

        def e2e_step():
            r = solve(Xpin)
            Xout.copy_(Xres, non_blocking=True)
            torch.cuda.current_stream(dev).synchronize()
            return r

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e_ms = reduce_max((t1 - t0) * 1e3, world, dev)
        n_rr = w.iters + (1 if mixed else 0)        # Rayleigh-Ritz steps per solve
        e2e = {"value": work / (e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(Xpin.numel() * Xpin.element_size()),
               # result block + per iteration Ritz values, residuals and flags + bounds
               "d2h_bytes_per_step": int(Xout.numel() * Xout.element_size()
                                         + n_rr * (2 * w.ns * 8 + 4) + 2 * 8 + 4),
               "ms_per_step": e_ms / args.steps}

    alg = stencil_algorithmic(w, dtype, prof, args.steps)
    peaks = measured_peaks()
    sm_max = ck.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    gbs = alg["bytes"] / (alg["ms"] / 1e3) / 1e9 if alg["ms"] else None
    peak = peaks.get("hbm_gbs", 6800.0)
    roof = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": gbs / peak if gbs else None,
            "peak_source": "of measured (hbm_gbs, copy)" if peaks.get("hbm_gbs")
            else "of fallback (6.8 TB/s)",
            "traffic": None,
            "avg_launch_ms": alg["ms"] / max(alg["launches"], 1),
            "launches": alg["launches"]}
    tr = stencil_traffic(dtype)
    if tr:
        # DRAM bytes of one captured launch (ncu) next to that launch's algorithmic bytes
        roof["traffic"] = tr["dram_bytes"]
        roof["traffic_launch"] = tr["launch"]
        roof["traffic_algorithmic_bytes"] = tr["algorithmic_bytes"]
        if "issue_active" in tr:
            # what bounds the kernel when DRAM does not: instruction issue in the same capture
            roof["issue"] = {"issue_active": tr["issue_active"],
                             "thread_inst_per_ptorb": tr["thread_inst_per_ptorb"]}
    if dtype == "f64":
        # The FP64 step runs its neighbour sums on the integer and FP32 pipes (exact integer
        # sums) and spends four FP64 operations per point; its FP64-equivalent flop rate is
        # compared with the FP64 pipe's issue limit as context.
        fl = alg["flops"] / (alg["ms"] / 1e3) / 1e12 if alg["ms"] > 0 else None
        roof["kernel"] = ("k_stencil_df (fused stencil + V_eff + recurrence; exact integer "
                          "neighbour sums, four FP64 operations per point)")
        roof["fp64_equiv_tflops"] = fl
        roof["fp64_pipe_peak_tflops"] = fp64_alu_peak_tflops(sm_max)
    else:
        roof["kernel"] = ("stencil phase: k_stencil_f32_tma filter steps (TMA-fed FP32) + "
                          "k_stencil_df for H Y_f, the FP64 refinement and Lanczos")

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
           "config": workload_config(w, dtype), "roofline": roof, "clocks": ck,
           "e2e": e2e, "gpu_launches": int(launches),
           "phases_ms": {k: round(v[1], 3) for k, v in prof.items()},
           "ritz_lowest": [float(x) for x in ritz[:4]],
           "max_resid": float(np.max(resid)) if resid is not None else None}
    out["after_rotation"] = after_rotation(ctx, X64 if mixed else X, ritz, w, stream,
                                           fp64_alu_peak_tflops(sm_max))
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_sample(w, args.seed, budget_s=args.cpu_budget)
    ctx.close()
    del X, W, X0, X64, W64, Xpin, Xout, Xres
    torch.cuda.empty_cache()
    if world == 1 and not args.no_mixed160:
        out["mixed160"] = mixed_vs_fp64(args.seed)
        torch.cuda.empty_cache()
    if world == 1 and not args.no_batching:
        from paper_1603_04334_gb300 import batching
        # 64 uneven clusters in one batched filter against per-cluster launches: the
        # configured mix (edges 32-96) and a mix of small clusters (edges 32-48) that each
        # under-fill the GPU
        out["batching"] = {"config_mix": batching.compare(64, args.seed),
                           "small_mix": batching.compare(64, args.seed, edges=(32, 40, 48))}
        torch.cuda.empty_cache()
    if world == 1 and args.serving_requests > 0:
        out["serving"] = serving_study(args.seed, args.serving_requests)
    return out


def mixed_vs_fp64(seed: int, resid_cut: float = 1e-4) -> dict:
    """The large cluster (160^3 grid, h = 0.25 bohr, 400 atoms, Ns = 1024, degree 24, 20
    iterations) solved in both forms on this GPU from the same start block: the mixed form
    (Lanczos bounds, 20 FP32-filter iterations, one FP64 refinement iteration) and the FP64
    form (Lanczos bounds, 20 FP64 iterations). Each solve is timed once with CUDA events on
    the context stream, after one warm-up iteration of each form (workspaces, kernel
    loading); the start block is drawn on the device (torch's seeded generator) before the
    timing starts. Ritz values of the states the FP64 run has converged (residual <=
    resid_cut) are compared with the mixed run's."""
    import torch
    from paper_1603_04334_gb300 import sparc

    w = synth.preset("cluster160")
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    cl = synth.make_cluster(w, seed)
    ctx = sparc.Context(cl.n, cl.h, cl.R, cl.Z, cl.gamma, veff=None, sigma=cl.sigma,
                        rcut=cl.rcut, rc_erf=cl.rc_erf, stream=stream)
    X32 = torch.empty((w.ns, w.nd), dtype=torch.float32, device=dev)
    W32 = torch.empty_like(X32)
    X64 = torch.empty((w.ns, w.nd), dtype=torch.float64, device=dev)
    W64 = torch.empty_like(X64)

    def start():
        g = torch.Generator(device=dev)
        g.manual_seed(seed + 1)
        X64.uniform_(-0.5, 0.5, generator=g)

    b0 = ctx.first_bounds(w.lanczos_k, seed)
    # warm-up: one iteration of each form
    start()
    X32.copy_(X64)
    ctx.chefsi_step(X32, W32, w.degree, b0, want_resid=False)
    start()
    ctx.chefsi_step(X64, W64, w.degree, b0, want_resid=True)
    torch.cuda.synchronize()

    def timed(run):
        ck = ClockSampler(torch.cuda.current_device())
        ctx.profile_reset()
        ctx.profile_enable(True)
        torch.cuda.synchronize()
        ck.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = run()
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = ck.stop()
        ctx.profile_enable(False)
        ph = {k: round(v[1], 1) for k, v in ctx.profile_read().items()}
        return r, e0.elapsed_time(e1) / 1e3, ph, clocks

    def mixed():
        b = ctx.first_bounds(w.lanczos_k, seed)
        for _ in range(w.iters):
            _, _, b = ctx.chefsi_step(X32, W32, w.degree, b, want_resid=False)
        X64.copy_(X32)
        return ctx.chefsi_step(X64, W64, w.degree, b, want_resid=True)

    def fp64():
        b = ctx.first_bounds(w.lanczos_k, seed)
        r = None
        for it in range(w.iters):
            r = ctx.chefsi_step(X64, W64, w.degree, b, want_resid=it == w.iters - 1)
            b = r[2]
        return r

    start()
    X32.copy_(X64)
    (rm, resm, _), t_m, ph_m, ck_m = timed(mixed)
    f32 = f32_filter_roofline(ctx, w, X32, W32, b0)
    start()
    (r64, res64, _), t_64, ph_64, ck_64 = timed(fp64)
    ctx.close()
    del X32, W32, X64, W64
    conv = res64 <= resid_cut
    d = np.abs(rm - r64)
    work_m = work_per_step(w, "f32")
    work_64 = work_per_step(w, "f64")
    return {"workload": workload_config(w, "f32")["workload"],
            "mixed_s": t_m, "fp64_s": t_64, "speedup": t_64 / t_m,
            "mixed_ptorb_per_s": work_m / t_m, "fp64_ptorb_per_s": work_64 / t_64,
            "resid_cut": resid_cut, "converged_fp64": int(conv.sum()),
            "converged_both": int((conv & (resm <= resid_cut)).sum()),
            "max_abs_dritz_converged": float(d[conv].max()) if conv.any() else None,
            "within_1e-5": bool(conv.any() and d[conv].max() <= 1e-5),
            "max_abs_dritz_all": float(d.max()),
            "dritz_converged_quantiles": ([float(q) for q in np.quantile(d[conv], [0.5, 0.9, 1.0])]
                                          if conv.any() else None),
            "ritz_lowest": [float(x) for x in r64[:3]],
            "mixed_phases_ms": ph_m, "fp64_phases_ms": ph_64,
            "f32_filter": f32,
            "clocks": {"mixed": ck_m, "fp64": ck_64},
            "timing": "one timed solve of each form (CUDA events), after one warm-up iteration "
                      "of each; start block drawn on the device before the timing"}


def f32_filter_roofline(ctx, w, X32, W32, bounds, reps: int = 3) -> dict:
    """The FP32 filter step alone: `reps` degree-m filters of the FP32 block (the mixed
    solve's result, any valid interval), the CUDA-event time of their stencil launches
    (k_stencil_f32_tma) from the library's phase counters, and the HBM fraction of the
    steps' algorithmic bytes: 12 B per point-orbital (Y_j, Y_{j-1} read, Y_{j+1} written;
    8 B for the first step) + 4 B of potential per node, against the measured copy."""
    import torch
    a, b, a0 = bounds
    torch.cuda.synchronize()
    ctx.profile_reset()
    ctx.profile_enable(True)
    for _ in range(reps):
        ctx.cheb_filter(X32, W32, w.degree, a, b, a0)
    torch.cuda.synchronize()
    ctx.profile_enable(False)
    n_launch, ms = ctx.profile_read()["stencil"]
    m = w.degree
    per_filter = w.nd * w.ns * (2 * 4 + (m - 1) * 3 * 4) + w.nd * m * 4
    gbs = reps * per_filter / (ms / 1e3) / 1e9
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    return {"launches": n_launch, "ms_per_step": ms / max(n_launch, 1),
            "achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak,
            "kernel": "k_stencil_f32_tma", "bytes_per_filter": per_filter,
            "sample": f"{reps} degree-{m} FP32 filters of the {w.ns}-column block"}


def serving_study(seed: int, requests: int, rates=(400.0, 20.0), below=(0.5,),
                  slots: int = 8, workers: int = 4, budget_gb: float = 150.0,
                  serial_sample: int = 24) -> dict:
    """The serving loop under Poisson arrivals: `requests` requests per rate, drawn from
    seed (edge in {48..128}, h = 0.3, 4-200 atoms, Ns 32-512, degree 20, <= 15 iterations to
    max residual 1e-4, mixed form), 150 GB budget. The continuous-batching server (at most
    `slots` active requests whose filters share launches, requests joining between rounds)
    runs the configured rates (20 and 400 req/s) first; they saturate it and measure its
    capacity; then rates below saturation (the given fractions of that capacity). Beside
    them: the worker server (`workers` threads, one stream each, a whole solve per request)
    at 400 req/s, and `serial_sample` requests spread evenly over the list solved one at a
    time in FP64 (one worker): their service times and the serial throughput."""
    from paper_1603_04334_gb300 import serve

    specs = serve.draw_requests(requests, seed)
    budget = int(budget_gb * 2 ** 30)

    def point(rate, batched, nslots):
        t0 = time.perf_counter()
        m = serve.run_arrivals(specs, rate, budget, nslots, seed + 1, batched=batched)
        lat = m["latency_s"]
        res = m["results"]
        return {"rate_req_per_s": rate, "requests": len(specs),
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(lat.mean()), "max_s": float(lat.max()),
                "throughput_req_per_s": len(specs) / m["span_s"],
                "max_running": m["stats"]["max_running"],
                "peak_reserved_gb": m["stats"]["peak_reserved"] / 2 ** 30,
                "converged": int(sum(r["converged"] for r in res)),
                "failed": int(sum(r["status"] != 0 for r in res)),
                "wall_s": time.perf_counter() - t0}

    pts = [point(r, True, slots) for r in rates]
    cap = max(p["throughput_req_per_s"] for p in pts)
    pts += [point(f * cap, True, slots) for f in below]
    wk = point(max(rates), False, workers)
    base = []
    srv = serve.Server(budget, 1)
    pick = specs[::max(1, len(specs) // serial_sample)][:serial_sample]
    try:
        for s in pick:
            f64 = serve.Spec(s.n, s.h, s.R, s.Z, s.gamma, s.ns, s.degree, s.max_iters, s.tol,
                             s.seed, "f64")
            r = srv.wait(srv.submit(f64))
            base.append(r["t_done"] - r["t_admit"])
    finally:
        srv.close()
    base = np.array(base)
    return {"workload": "edge in {48,...,128}, h=0.3, atoms 4-200, Ns 32-512, degree 20, "
                        "<= 15 CheFSI iterations to max residual 1e-4, mixed form",
            "server": f"continuous batching: at most {slots} active requests, their FP32 "
                      f"filters in shared launches, joining between CheFSI iterations",
            "budget_gb": budget_gb, "capacity_req_per_s": cap,
            "points": pts,
            "worker_server": dict(wk, server=f"{workers} worker threads, one stream each, "
                                             f"whole solves"),
            "serial_fp64": {"requests": len(base),
                            "throughput_req_per_s": len(base) / float(base.sum()),
                            "service_p50_s": float(np.percentile(base, 50)),
                            "service_p99_s": float(np.percentile(base, 99)),
                            "sample": f"{len(base)} requests spread evenly over the same "
                                      f"list (every {max(1, len(specs) // serial_sample)}th), "
                                      f"one at a time in FP64 on one worker"}}


def after_rotation(ctx, X, ritz, w, stream, fp64_peak_tflops: float, reps: int = 10) -> dict:
    """Times the steps after the rotation on the solved block, apart from the solve:
    occupations and Fermi level (N_e = Ns, kT = 1e-3 Ha), density, non-local force, and the
    electrostatic potential of that density (CG to a relative residual of 1e-10). Each is
    the median of `reps` CUDA-event timings on the context stream after 3 warm-up calls."""
    import torch

    nelec, kT = float(w.ns), 1e-3
    mu, g = ctx.occupations(ritz, nelec, kT)
    rho = torch.empty(w.nd, dtype=torch.float64, device=X.device)

    def timed(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    t_occ = timed(lambda: ctx.occupations(ritz, nelec, kT))
    t_rho = timed(lambda: ctx.density(X, g, rho))
    t_f = timed(lambda: ctx.nonlocal_force(X, g))
    # electrostatic potential of the density with the atoms' pseudocharges (CG to 1e-10)
    ctx.density(X, g, rho)
    phi = torch.empty_like(rho)
    pois = {}

    def solve_phi():
        _, pois["iters"], pois["relres"] = ctx.poisson(rho, phi, tol=1e-10)

    t_p = timed(solve_phi)
    es = X.element_size()
    nsup = ctx.info()["nsupport"]
    rho_bytes = w.nd * w.ns * es + 8 * w.nd
    rho_fp64 = 2 * w.nd * w.ns            # one multiply and one fused multiply-add per term
    f_fp64 = 52 * nsup * w.ns             # 36 for the gradient, 16 for the projections
    peak_inst = fp64_peak_tflops * 1e12 / 2  # FP64 instructions/s (an FMA counts 2 flops)
    return {"nelec": nelec, "kT": kT, "lambda_f": mu,
            "occupations_ms": t_occ,
            "density_ms": t_rho,
            "density_GBps": rho_bytes / (t_rho / 1e3) / 1e9,
            "density_fp64_inst_frac": rho_fp64 / (t_rho / 1e3) / peak_inst,
            "force_ms": t_f,
            "force_fp64_inst_frac": f_fp64 / (t_f / 1e3) / peak_inst,
            "support_entries": nsup,
            "poisson_ms": t_p, "poisson_cg_iters": pois["iters"],
            "poisson_relres": pois["relres"]}


# ----------------------------------------------------------------------------------
# the oracle (CPU baseline and the reference arm)
# ----------------------------------------------------------------------------------
def host_cores() -> int:
    """Host cores this process may run on (nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OracleRun:
    """The FP64 CPU oracle, as it stands, set up once on a column slice of a workload:
    the Hamiltonian (V_eff, projector tables), the Lanczos bounds and the first filter
    interval are built here, outside any timing; step() runs one CheFSI iteration (the
    degree-m filter and the Rayleigh-Ritz step) on the slice."""

    def __init__(self, w, seed: int, cols: int):
        import oracle
        self.oracle = oracle
        self.w = w
        cl = synth.make_cluster(w, seed)
        self.H = oracle.Hamiltonian.from_cluster(cl)
        self.X0 = synth.initial_block(seed + 1, w.nd, w.ns)[:cols].copy()
        lo, hi, _ = self.H.lanczos_bounds(w.lanczos_k, seed)
        self.b0 = oracle.chefsi_first_bounds(lo, hi)
        self.reset()

    @property
    def cols(self) -> int:
        return self.X0.shape[0]

    def reset(self):
        self.X, self.b = self.X0.copy(), list(self.b0)

    def step(self):
        self.X, _, _, self.b = self.oracle.chefsi_step(self.H, self.X, self.w.degree, self.b)

    def work_per_step(self) -> int:
        return (self.w.degree + 1) * self.w.nd * self.cols

    def timed(self, budget_s: float, max_steps: int = 64, threads: int = 0):
        """Iterations until budget_s has passed (at least one): (iterations, seconds)."""
        from oracle import oracle as O
        O.threads(threads)
        self.reset()
        t0 = time.perf_counter()
        n = 0
        while True:
            self.step()
            n += 1
            if time.perf_counter() - t0 >= budget_s or n >= max_steps:
                break
        return n, time.perf_counter() - t0


def oracle_sample(w, seed: int, budget_s: float = 12.0, single_budget_s: float = 6.0) -> dict:
    """Times the FP64 CPU oracle, as it stands, on a bounded sample of the workload: CheFSI
    iterations (filter of degree m + Rayleigh-Ritz) on a slice of the start block as wide as
    the host has cores (at least 16 columns, at most Ns), with OpenMP over the slice's
    columns on all cores; then one thread on a 4-column slice. Set-up (Hamiltonian, bounds)
    is outside the timing."""
    from oracle import oracle as O
    nproc = host_cores()
    cols = min(w.ns, max(ORACLE_COLS, nproc))
    run = OracleRun(w, seed, cols)
    n_all, t_all = run.timed(budget_s, threads=nproc)
    one = OracleRun(w, seed, min(w.ns, 4))
    n_one, t_one = one.timed(single_budget_s, threads=1)
    O.threads(nproc)
    per = run.work_per_step()
    return {"value": n_all * per / t_all, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "nproc": nproc,
            "sample": f"{n_all} CheFSI iteration(s) (degree {w.degree} filter + Rayleigh-Ritz) "
                      f"on a {cols}-column slice of {w.name}, {t_all:.1f} s, OpenMP over the "
                      f"slice's columns on all {nproc} host cores; set-up outside the timing",
            "single_thread": {"value": n_one * one.work_per_step() / t_one, "unit": UNIT,
                              "cores": 1,
                              "sample": f"{n_one} iteration(s) on a {one.cols}-column slice, one "
                                        f"thread, {t_one:.1f} s"}}


def run_reference(args, rank, world):
    """The reference arm: the oracle as it stands on the host cores. The Hamiltonian, the
    bounds and the slice are set up once outside the timing; W untimed and K timed steps,
    each one CheFSI iteration (degree-m filter + Rayleigh-Ritz) on the slice."""
    if rank != 0:
        return None
    from oracle import oracle as O
    w = synth.preset(args.workload)
    dtype = "f64"
    nproc = host_cores()
    cols = min(w.ns, max(ORACLE_COLS, nproc))
    run = OracleRun(w, args.seed, cols)
    O.threads(nproc)
    for _ in range(args.warmup):
        run.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run.step()
    t = time.perf_counter() - t0
    value = args.steps * run.work_per_step() / t
    cb = {"value": value, "unit": UNIT, "cores": nproc, "kind": "oracle", "nproc": nproc,
          "sample": f"{args.steps} CheFSI iteration(s) (degree {w.degree} filter + "
                    f"Rayleigh-Ritz) on a {cols}-column slice of {w.name}, OpenMP over the "
                    f"slice's columns on all {nproc} host cores; set-up outside the timing"}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic", "config": workload_config(w, dtype), "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="cluster96", choices=sorted(synth.PRESETS))
    ap.add_argument("--dtype", choices=["f64", "f32"], default=None)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-mixed160", action="store_true",
                    help="skip the 160^3 mixed-vs-FP64 comparison")
    ap.add_argument("--no-batching", action="store_true",
                    help="skip the batched-filter comparison (64 clusters)")
    ap.add_argument("--serving-requests", type=int, default=200,
                    help="requests per arrival rate of the serving study (0: skip it)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours" and not os.environ.get("SPARC_BENCH_ALLOW_SHORT"):
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
