"""Benchmark of the V_loc|psi> action on GB300.

Headline: bands/s of the FP32 forward apply on the 96^3 grid, cut-off sphere
R = 24 (57777 plane waves), 1024 bands per step, inputs resident in HBM
(473 MB in + 473 MB out per step, larger than L2).  The same JSON line also
carries the FP64 path, the adjoint, the 96x96x120 grid, the end-to-end
host-buffer number, the per-kernel roofline, the CPU oracle baseline and a
cuFFT comparison (torch.fft, comparison only).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own 1024 bands (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "V_loc|ψ⟩ bands/s at 96^3 (FP32 vs FP64), fraction of HBM roofline"
GRID, R, NBANDS, SEED = (96, 96, 96), 24, 1024, 2
GRID2 = (96, 96, 120)
WORKLOAD = "96^3 grid, sphere h^2+k^2+l^2<=24^2 (57777 PWs), 1024 bands/GPU, FP32 forward apply"
FALLBACK_HBM_GBS = 6800.0
# the two arms share this config dict (the workload); arm details go elsewhere
CONFIG = {"workload": WORKLOAD, "grid": list(GRID), "npw": 57777, "bands_per_gpu": NBANDS,
          "l2": "inputs larger than L2 (473 MB in + 473 MB out per step)", "parallelism": "bands split over GPUs"}
KERNEL_SOURCES = ["paper_1601_07378_gb300/csrc/fft_core.cuh", "paper_1601_07378_gb300/csrc/fft_ct.cuh",
                  "paper_1601_07378_gb300/csrc/kernels_impl.cuh", "paper_1601_07378_gb300/csrc/kernels_ct.cuh"]


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ counts
def path_counts(info, n):
    """Algorithmic bytes per band per kernel and 5 n log2 n flops per band."""
    n1, n2, n3 = n
    S, NP, npw = info["nsticks"], info["nplanes"], info["npw"]
    e = 8 if info["precision"] == 1 else 16
    cyl, slab = S * n3, NP * n2 * n3
    per_band = {
        "k1_scatter_zpass": (npw + cyl) * e,
        "k2_ypass_inv": (cyl + slab) * e,
        "k3_xpass_v": 2 * slab * e,
        "k2_ypass_fwd": (slab + cyl) * e,
        "k4_zpass_gather": (cyl + npw) * e,
    }
    f = lambda m: 5.0 * m * math.log2(m)
    flops = 2 * (S * f(n3) + NP * n3 * f(n2) + n2 * n3 * f(n1)) + 2 * n1 * n2 * n3
    B5 = 2 * npw * e + 4 * cyl * e + 4 * slab * e
    B3 = 2 * npw * e + 4 * slab * e
    return per_band, flops, B5, B3


def kernel_src_sha() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(kernel: str, prec: str):
    """DRAM bytes per band of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    ent = d.get(f"{kernel}:{prec}")
    if not ent or ent.get("source_sha") != kernel_src_sha():
        return None
    return ent["dram_bytes"] / ent["bands_per_launch"]


def peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return FALLBACK_HBM_GBS, "fallback"


def measure_alu_peaks(sampler_index: int, target_ms: float = 40.0) -> dict:
    """Arithmetic ceilings measured on this GPU with the library's probe
    kernels (vloc_alu_peak: DFMA, DADD, FFMA, paired FFMA2, paired FADD2),
    each sized to about `target_ms` and taken as the best of 3 launches,
    with the SM clocks sampled over the probes."""
    from paper_1601_07378_gb300 import vloc
    sampler = ClockSampler(sampler_index)
    sampler.start()
    sampler.wait_ready()
    out = {}
    for kind in ("dfma", "dadd", "ffma", "ffma2", "fadd2"):
        r = vloc.alu_peak(kind, 512)
        iters = max(512, int(512 * target_ms / max(r["ms"], 1e-3)))
        best = max(vloc.alu_peak(kind, iters)["gflops"] for _ in range(3))
        out[kind + "_gflops"] = round(best, 1)
    out["clocks"] = sampler.stop()
    out["how"] = ("vloc_alu_peak: 8 blocks x 256 threads per SM, 16 independent dependent chains per thread, "
                  "CUDA events, best of 3 launches of about 40 ms; FMA = 2 flops, add = 1, paired kinds twice that")
    return out


# ------------------------------------------------------------------ clocks
REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_ready(self, timeout=5.0):
        """Block until nvidia-smi has printed its first sample, so that the
        samples that follow cover the timed region."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)
        self.lines.clear()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        return summarize_clocks(self.lines)


def summarize_clocks(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen in
    nvidia-smi CSV lines (index, clocks.sm, clocks.max.sm, power.draw,
    reasons.active, then the four reasons of REASONS)."""
    sm, smax, active = [], [], set()
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for name, v in zip(REASONS, f[5:9]):
            if v.lower().startswith("active"):
                active.add(name)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    sm.sort()
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(active), "samples": len(sm)}


# ------------------------------------------------------------------ timing
def time_steps(fn, steps, warmup, stream, dist_on):
    import torch
    import torch.distributed as dist
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if dist_on:
        dist.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        fn()
    stop.record(stream)
    torch.cuda.synchronize()
    if dist_on:
        dist.barrier()
    from paper_1601_07378_gb300.dist import max_over_ranks
    return max_over_ranks(start.elapsed_time(stop), device="cuda")


def host_link_rates(h_in, h_out, d_in, d_out):
    """Plain pinned-memory copy rates (GB/s) right after the host-buffer leg:
    the host link is shared with other work on the machine, so its rate at
    the time gives the end-to-end number its context."""
    import torch
    rates = {}
    for name, dst, src in (("h2d", d_in, h_in), ("d2h", h_out, d_out)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        rates[name] = round(3 * src.numel() * src.element_size() / (time.perf_counter() - t0) / 1e9, 1)
    return rates


def cpu_oracle_rate(n, g, c, V, nbands_sample):
    from oracle import oracle as O
    import numpy as np
    cores = host_cores()
    sub = np.ascontiguousarray(c[:nbands_sample].astype(np.complex128))
    t0 = time.perf_counter()
    ref = O.apply(n, g, sub, V.astype(np.float64), nthreads=cores)
    dt = time.perf_counter() - t0
    return nbands_sample / dt, cores, dt, ref


# ------------------------------------------------------------------ arms
def run_reference(args, rank):
    """The reference arm: the FP64 CPU oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    import numpy as np
    from oracle import oracle as O
    from paper_1601_07378_gb300 import synth
    O.build()
    cores = host_cores()
    g = synth.sphere_glist(*GRID, R)
    per = max(1, cores)
    c = synth.coefficients(g, per, seed=SEED, dtype=np.complex64)
    V = synth.potential(*GRID, "smooth", SEED + 1000)[0].astype(np.float32)
    for _ in range(args.warmup):
        cpu_oracle_rate(GRID, g, c, V, per)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cpu_oracle_rate(GRID, g, c, V, per)
    dt = time.perf_counter() - t0
    value = args.steps * per / dt
    sample = f"{per} bands of the 96^3 R=24 workload per step (FP64 oracle on FP32-rounded inputs)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "bands/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(CONFIG, bands_per_gpu=NBANDS),
        "arm": {"sample_bands_per_step": per, "host_cores": cores},
        "cpu_baseline": {"value": value, "unit": "bands/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "bands/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    dist_on = world > 1
    torch.cuda.set_device(local_rank)
    if dist_on:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_1601_07378_gb300.build import build
    if local_rank == 0:
        build()
    if dist_on:
        dist.barrier()
    from paper_1601_07378_gb300 import synth, vloc

    stream = torch.cuda.current_stream()
    g = synth.sphere_glist(*GRID, R)
    if args.only == "density":
        # profiler driver: the charge density of --bands bands at 96^3, FP32
        c_d = torch.from_numpy(synth.coefficients(g, NBANDS, seed=SEED)).to("cuda", torch.complex64)
        rho_d = torch.empty(GRID, dtype=torch.float32, device="cuda")
        plan = vloc.VlocPlan(GRID, g, torch.complex64, chunk=args.chunk, generic=args.generic)
        ms = time_steps(lambda: plan.density(c_d, rho=rho_d), args.steps, args.warmup, stream, dist_on)
        plan.profile(True)
        for _ in range(args.steps):
            plan.density(c_d, rho=rho_d)
        prof = plan.get_profile()
        plan.profile(False)
        if rank == 0:
            print(json.dumps({"only": "density", "bands": NBANDS, "steps": args.steps, "grid": list(GRID),
                              "chunk": plan.info()["chunk_bands"], "ms_per_step": ms / args.steps,
                              "bands_per_s": world * NBANDS * args.steps / ms * 1e3,
                              "kernels": {k: [n // args.steps, round(t / args.steps, 4)] for k, (n, t) in prof.items()}}))
        return
    if args.only == "headline":
        # profiler driver: the headline steps alone, nothing else
        cdt, rdt = (torch.complex64, torch.float32) if args.prec == "f32" else (torch.complex128, torch.float64)
        c_d = torch.from_numpy(synth.coefficients(g, NBANDS, seed=SEED)).to("cuda", cdt)
        V_d = torch.from_numpy(synth.potential(*GRID, "smooth", SEED + 1000)[0]).to("cuda", rdt)
        out_d = torch.empty_like(c_d)
        grid = tuple(int(x) for x in args.grid.split(","))
        if grid != GRID:
            g = synth.sphere_glist(*grid, min(grid) // 4)
            c_d = torch.from_numpy(synth.coefficients(g, NBANDS, seed=SEED)).to("cuda", cdt)
            V_d = torch.from_numpy(synth.potential(*grid, "smooth", SEED + 1000)[0]).to("cuda", rdt)
            out_d = torch.empty_like(c_d)
        plan = vloc.VlocPlan(grid, g, cdt, chunk=args.chunk, generic=args.generic,
                             double_float=args.df and args.prec == "f64")
        ms = time_steps(lambda: plan.apply(c_d, V_d, out=out_d), args.steps, args.warmup, stream, dist_on)
        plan.profile(True)
        for _ in range(args.steps):
            plan.apply(c_d, V_d, out=out_d)
        prof = plan.get_profile()
        plan.profile(False)
        if rank == 0:
            print(json.dumps({"only": "headline", "prec": args.prec, "double_float": plan.info()["double_float"],
                              "bands": NBANDS, "steps": args.steps,
                              "grid": list(grid),
                              "chunk": plan.info()["chunk_bands"], "generic": args.generic,
                              "ms_per_step": ms / args.steps, "bands_per_s": world * NBANDS * args.steps / ms * 1e3,
                              "kernel_ms_per_step": sum(t for _, t in prof.values()) / args.steps,
                              "kernels": {k: [n // args.steps, round(t / args.steps, 4)] for k, (n, t) in prof.items()}}))
        return
    c64 = synth.coefficients(g, NBANDS, seed=SEED + rank, dtype=np.complex64)
    V96 = synth.potential(*GRID, "smooth", SEED + 1000)[0]
    V120 = synth.potential(*GRID2, "smooth", SEED + 1000)[0]
    c_d = torch.from_numpy(c64).cuda()
    out_d = torch.empty_like(c_d)
    V_d = torch.from_numpy(V96.astype(np.float32)).cuda()
    plan = vloc.VlocPlan(GRID, g, torch.complex64)
    info = plan.info()
    per_band, flops, B5, B3 = path_counts(info, GRID)

    # ---- headline: FP32 forward, 1024 bands per step
    sampler = ClockSampler(local_rank)
    sampler.start()
    sampler.wait_ready()
    l0 = plan.launch_count()
    ms = time_steps(lambda: plan.apply(c_d, V_d, out=out_d), args.steps, args.warmup, stream, dist_on)
    launches = (plan.launch_count() - l0) // (args.steps + args.warmup) * args.steps
    clocks = sampler.stop()
    ms_step = ms / args.steps
    value = world * NBANDS / (ms_step / 1e3)

    # ---- per-kernel device time (profiled pass over the same steps)
    plan.profile(True)
    for _ in range(args.steps):
        plan.apply(c_d, V_d, out=out_d)
    prof = plan.get_profile()
    plan.profile(False)
    tot = sum(t for _, t in prof.values())
    dom = max(prof, key=lambda k: prof[k][1])
    nl, tms = prof[dom]
    bands_per_launch = NBANDS * args.steps / nl
    bytes_launch = per_band[dom] * bands_per_launch + (GRID[0] * GRID[1] * GRID[2] * 4 if dom == "k3_xpass_v" else 0)
    achieved = bytes_launch / (tms / nl / 1e3) / 1e9
    peak, peak_kind = peaks()
    tr = load_traffic(dom, "f32")
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": tr * bands_per_launch if tr is not None else None,
                "alg_bytes_per_launch": bytes_launch, "bands_per_launch": bands_per_launch,
                "kernel_share": {k: round(v[1] / tot, 4) for k, v in prof.items()}}
    path = {"B5_bytes_per_band": B5, "B3_bytes_per_band": B3,
            "frac_of_B5_roofline": value / world / (peak * 1e9 / B5),
            "frac_of_B3_roofline": value / world / (peak * 1e9 / B3),
            "flops_per_band": flops, "gflops": value / world * flops / 1e9}

    # ---- adjoint FP32
    ms_adj = time_steps(lambda: plan.apply(c_d, V_d, out=out_d, adjoint=True), args.steps, 2, stream, dist_on)
    adj = world * NBANDS / (ms_adj / args.steps / 1e3)

    # ---- end to end through the host-buffer entry point (pinned host memory)
    c_h = torch.from_numpy(c64).pin_memory()
    V_h = torch.from_numpy(V96.astype(np.float32)).pin_memory()
    o_h = torch.empty_like(c_h).pin_memory()
    ke = max(10, args.steps)  # the host link is shared: average over at least 10 steps
    from paper_1601_07378_gb300.dist import max_over_ranks

    def e2e_run(blocking):
        # every step copies its inputs in and its result out; the
        # asynchronous calls overlap one step's last copies with the next
        # step's first, one synchronisation at the end
        for _ in range(2):
            plan.apply_host(c_h, V_h, o_h, blocking=blocking)
        torch.cuda.synchronize()
        if dist_on:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            plan.apply_host(c_h, V_h, o_h, blocking=blocking)
        torch.cuda.synchronize()
        return max_over_ranks(time.perf_counter() - t0, device="cuda")
    # the host link is shared with the machine's other work (single runs have
    # measured 30 % slow now and then): three runs of each form, alternated,
    # the median run reported and every run listed
    runs = {False: [], True: []}
    e2e_run(False)  # untimed
    for blocking in (False, True, False, True, False, True):
        runs[blocking].append(e2e_run(blocking))
    rate = lambda ts: world * NBANDS * ke / sorted(ts)[len(ts) // 2]
    e2e = {"value": rate(runs[False]), "unit": "bands/s", "steps": ke,
           "h2d_bytes_per_step": c_h.numel() * 8 + V_h.numel() * 4, "d2h_bytes_per_step": o_h.numel() * 8,
           "blocking_calls_value": rate(runs[True]),
           "runs_bands_per_s": {"async": [round(world * NBANDS * ke / t) for t in runs[False]],
                                "blocking": [round(world * NBANDS * ke / t) for t in runs[True]]},
           "what": "vloc_apply_host_async per step (host copies in and out inside every step), one "
                   "synchronisation per run; blocking_calls_value: vloc_apply_host, synchronised per step; "
                   "the median of three alternated runs of each after an untimed one (every run listed)",
           "link_GBps": host_link_rates(c_h, o_h, c_d, out_d)}

    # ---- the same forward step replayed as one captured CUDA graph
    plang = vloc.VlocPlan(GRID, g, torch.complex64, graph=True)
    ms_g = time_steps(lambda: plang.apply(c_d, V_d, out=out_d), args.steps, args.warmup, stream, dist_on)
    graph = {"value": world * NBANDS / (ms_g / args.steps / 1e3), "unit": "bands/s",
             "ms_per_step": ms_g / args.steps, "what": "headline step as one graph launch"}
    del plang

    # ---- 96x96x120 grid (same sphere and coefficients)
    plan2 = vloc.VlocPlan(GRID2, g, torch.complex64)
    V2_d = torch.from_numpy(V120.astype(np.float32)).cuda()
    ms2 = time_steps(lambda: plan2.apply(c_d, V2_d, out=out_d), args.steps, 2, stream, dist_on)
    c2_value = world * NBANDS / (ms2 / args.steps / 1e3)
    del plan2, V2_d

    # ---- measured arithmetic ceilings (FP64 and FP32 pipes) for the FP64 legs
    alu = measure_alu_peaks(local_rank)

    # ---- FP64 path
    plan64 = vloc.VlocPlan(GRID, g, torch.complex128)
    c128_d = c_d.to(torch.complex128)
    o128_d = torch.empty_like(c128_d)
    V64_d = V_d.to(torch.float64)
    k64 = max(2, args.steps // 5)
    ms64 = time_steps(lambda: plan64.apply(c128_d, V64_d, out=o128_d), k64, 1, stream, dist_on)
    f64_value = world * NBANDS / (ms64 / k64 / 1e3)
    ms64a = time_steps(lambda: plan64.apply(c128_d, V64_d, out=o128_d, adjoint=True), k64, 1, stream, dist_on)
    f64_adj = world * NBANDS / (ms64a / k64 / 1e3)
    plan64.profile(True)
    plan64.apply(c128_d, V64_d, out=o128_d)
    prof64 = plan64.get_profile()
    plan64.profile(False)
    dom64 = max(prof64, key=lambda k: prof64[k][1])
    f64 = {"value": f64_value, "unit": "bands/s", "ms_per_step": ms64 / k64, "steps": k64,
           "adjoint": {"value": f64_adj, "unit": "bands/s"},
           "speedup_fp32_over_fp64": value / f64_value,
           "roofline": {"bound": "alu", "unit": "GFLOP/s", "achieved": f64_value / world * flops / 1e9,
                        "peak": alu["dfma_gflops"], "frac": f64_value / world * flops / 1e9 / alu["dfma_gflops"],
                        "peak_source": "measured (vloc_alu_peak DFMA, this run)",
                        "frac_of_dadd_rate": f64_value / world * flops / 1e9 / alu["dadd_gflops"],
                        "dominant_kernel": dom64,
                        "kernel_share": {k: round(v[1] / sum(t for _, t in prof64.values()), 4) for k, v in prof64.items()}},
           "hbm_frac_of_B5": f64_value / world / (peak * 1e9 / (2 * B5))}
    # ---- FP64 data in double-float arithmetic (hi + lo FP32 pairs on the FP32 pipes)
    plandf = vloc.VlocPlan(GRID, g, torch.complex128, double_float=True)
    msdf = time_steps(lambda: plandf.apply(c128_d, V64_d, out=o128_d), k64, 1, stream, dist_on)
    df_value = world * NBANDS / (msdf / k64 / 1e3)
    plandf.profile(True)
    plandf.apply(c128_d, V64_d, out=o128_d)
    profdf = plandf.get_profile()
    plandf.profile(False)
    f64_df = {"value": df_value, "unit": "bands/s", "ms_per_step": msdf / k64, "steps": k64,
              "double_float": plandf.info()["double_float"], "speedup_over_native_fp64": df_value / f64_value,
              "speedup_fp32_over_this": value / df_value,
              "hbm_frac_of_B5": df_value / world / (peak * 1e9 / (2 * B5)),
              "fp32_pipe_peaks": {"ffma2_gflops": alu["ffma2_gflops"], "fadd2_gflops": alu["fadd2_gflops"],
                                  "peak_source": "measured (vloc_alu_peak, this run)"},
              "kernel_share": {k: round(v[1] / sum(t for _, t in profdf.values()), 4) for k, v in profdf.items()},
              "what": "FP64 in and out, transforms in double-float (about 48 bits), FP64 gate 1e-12 vs the oracle"}
    del plan64, plandf, c128_d, o128_d, V64_d

    # ---- Gamma-point real mode (Sec. 4.3): 1024 real bands on the half
    # sphere (28889 PWs), two per complex transform, FP32
    gamma = None
    if not args.no_extra:
        gh = synth.half_sphere(g)
        pg = vloc.VlocPlan(GRID, gh, torch.complex64, gamma=True)
        cg = torch.from_numpy(synth.coefficients(gh, NBANDS, seed=SEED + 5, dtype=np.complex64)).cuda()
        og = torch.empty_like(cg)
        kg = max(3, args.steps // 2)
        msg = time_steps(lambda: pg.apply(cg, V_d, out=og), kg, 2, stream, dist_on)
        pg.profile(True)
        pg.apply(cg, V_d, out=og)
        profg = pg.get_profile()
        pg.profile(False)
        gamma = {"value": world * NBANDS / (msg / kg / 1e3), "unit": "bands/s", "ms_per_step": msg / kg,
                 "npw_half": len(gh), "what": "1024 real bands, 96^3, half sphere, two bands per complex transform",
                 "kernel_share": {k: round(v[1] / sum(t for _, t in profg.values()), 4) for k, v in profg.items()}}
        del pg, cg, og

    # ---- the halves on their own and the charge density (96^3, FP32)
    halves = None
    if not args.no_extra:
        def leg(fn, k, nbands, bytes_per_band):
            ms_l = time_steps(fn, k, 2, stream, dist_on)
            rate = world * nbands / (ms_l / k / 1e3)
            return {"value": rate, "unit": "bands/s", "ms_per_step": ms_l / k, "bands": nbands,
                    "alg_GBps": rate / world * bytes_per_band / 1e9,
                    "frac_of_hbm": rate / world * bytes_per_band / (peak * 1e9)}
        Nn = GRID[0] * GRID[1] * GRID[2]
        cyl_b, slab_b = info["nsticks"] * GRID[2] * 8, info["nplanes"] * GRID[1] * GRID[2] * 8
        nh = 256
        grid_d = torch.empty((nh, *GRID), dtype=torch.complex64, device="cuda")
        rho_d = torch.empty(GRID, dtype=torch.float32, device="cuda")
        kh = max(3, args.steps // 2)
        halves = {
            "to_real": leg(lambda: plan.to_real(c_d[:nh], grid_d), kh, nh,
                           info["npw"] * 8 + 2 * cyl_b + 2 * slab_b + Nn * 8),
            "to_recip": leg(lambda: plan.to_recip(grid_d, out_d[:nh]), kh, nh,
                            Nn * 8 + 2 * slab_b + 2 * cyl_b + info["npw"] * 8),
            "density": leg(lambda: plan.density(c_d, rho=rho_d), kh, NBANDS,
                           info["npw"] * 8 + 2 * cyl_b + 2 * slab_b),
            "what": "96^3, R = 24, FP32: psi = F+ S c to full grids (256 bands), r -> G of full grids "
                    "(256 bands), rho = sum |psi_n|^2 (1024 bands); alg bytes per band, every "
                    "inter-kernel round trip counted as in B5: to_real/to_recip npw + 2 cyl + 2 slab + N, "
                    "density npw + 2 cyl + 2 slab (complex64)",
        }
        del grid_d, rho_d

    # ---- second workload: lowest states of H = |G|^2/2 + V_loc by
    # Chebyshev-filtered subspace iteration, H applied through the chain; the
    # paper's test shape (80^3 grid, 35033-PW sphere, Gamma point, 1001
    # states; FP32, cell 38.3 bohr)
    eig = None
    if not args.no_extra:
        try:
            from paper_1601_07378_gb300 import eigensolver as E
            ne = (80, 80, 80)
            ge = synth.half_sphere(synth.sphere_glist(*ne, 20.3))
            Ve = synth.potential(*ne, "smooth", SEED + 7)[0]
            Ve = (-4.0 * (Ve - Ve.min())).astype(np.float32)
            pe = vloc.VlocPlan(ne, ge, torch.complex64, gamma=True)
            He = E.Hamiltonian(pe, torch.from_numpy(Ve).cuda(), cell=(38.3, 38.3, 38.3))
            E.chfsi(He, 1001, tol=1e-4, maxiter=1, degree=12, seed=SEED)  # warm-up (library handles, first launches)
            He.applies = 0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res_e = E.chfsi(He, 1001, tol=1e-4, maxiter=40, degree=12, seed=SEED)
            torch.cuda.synchronize()
            dt_e = time.perf_counter() - t0
            eig = {"seconds": dt_e, "iterations": res_e.iterations, "band_applies": res_e.h_applies,
                   "band_applies_per_s": res_e.h_applies / dt_e, "final_rel_residual": res_e.history[-1],
                   "nev": 1001, "npw_half": len(ge),
                   "what": "ChFSI (degree 12, block 1251) on H = |G|^2/2 + V_loc, 80^3, R = 20.3, Gamma point, FP32"}
            del pe, He, res_e
        except Exception as exc:  # a failed auxiliary leg must not hide the headline
            eig = {"error": repr(exc)}

    # ---- uneven multi-instance batch, one graph launch per step: 8 grids
    # 48^3 .. 144^3, R = n/4, 64 (i+1) bands each (FP32)
    batched = None
    if not args.no_extra:
        insts = []
        for i, m in enumerate(synth.BATCH_GRIDS):
            nn = (m, m, m)
            gi = synth.sphere_glist(*nn, m / 4)
            nbi = 64 * (i + 1)
            pi = vloc.VlocPlan(nn, gi, torch.complex64, graph=True, chunk=nbi)
            ci = torch.from_numpy(synth.coefficients(gi, nbi, seed=3 + i, dtype=np.complex64)).cuda()
            Vi = torch.from_numpy(synth.potential(*nn, "smooth", 1003 + i)[0].astype(np.float32)).cuda()
            insts.append((pi, ci, Vi, torch.empty_like(ci)))
        bplans, bcs, bVs, bouts = zip(*insts)
        kb = max(3, args.steps // 4)
        msb = time_steps(lambda: vloc.apply_batched(bplans, bcs, bVs, bouts), kb, 2, stream, dist_on)
        nb_tot = sum(c.shape[0] for c in bcs)
        # the same instances as serial direct launches (plans without graphs)
        splans = [vloc.VlocPlan(p.grid, p.glist, torch.complex64, chunk=c.shape[0]) for p, c in zip(bplans, bcs)]

        def serial():
            for sp, ci, Vi, oi in zip(splans, bcs, bVs, bouts):
                sp.apply(ci, Vi, out=oi)
        mss = time_steps(serial, kb, 2, stream, dist_on)
        # algorithmic bytes of the step: sum over instances of B5 x bands
        alg = sum(path_counts(p.info(), p.grid)[2] * c.shape[0] for p, c in zip(bplans, bcs))
        batched = {"value": world * nb_tot / (msb / kb / 1e3), "unit": "bands/s", "ms_per_step": msb / kb,
                   "bands_per_step": nb_tot, "launches_per_step": "1 graph launch",
                   "alg_bytes_per_step": alg, "alg_GBps": alg / (msb / kb / 1e3) / 1e9,
                   "frac_of_hbm": alg / (msb / kb / 1e3) / (peak * 1e9),
                   "serial_direct_ms_per_step": mss / kb,
                   "serial_direct_frac_of_hbm": alg / (mss / kb / 1e3) / (peak * 1e9),
                   "what": "8 instances 48^3..144^3, R = n/4, 64..512 bands, FP32, one CUDA graph "
                           "(instances on up to 4 parallel branches); serial_direct: the same plans' "
                           "applies one after another without a graph; bytes: sum of B5 x bands"}
        del insts, bplans, bcs, bVs, bouts, splans

    # ---- differentiable apply: loss = sum_n <psi_n|V|psi_n> + ||V psi - t||^2,
    # 512 bands at 96^3 FP32, forward + backward (dL/dc, dL/dV)
    autograd = None
    if not args.no_extra:
        na = 512
        ca = c_d[:na].clone().requires_grad_(True)
        Va = V_d.clone().requires_grad_(True)
        ta = (torch.randn(na, info["npw"], dtype=torch.complex64, device="cuda") * 0.01)

        def fwd_bwd():
            ca.grad = None
            Va.grad = None
            o = vloc.vloc_apply(ca, Va, plan)
            L = (torch.conj(ca) * o).real.sum() + ((o - ta).abs() ** 2).sum()
            L.backward()
        ka = max(3, args.steps // 4)
        msa = time_steps(fwd_bwd, ka, 2, stream, dist_on)
        autograd = {"value": world * na / (msa / ka / 1e3), "unit": "bands/s (forward + backward)",
                    "ms_per_step": msa / ka, "bands": na, "what": "96^3 FP32, loss <psi|V|psi> + ||V psi - t||^2"}
        del ca, Va, ta

    # ---- cuFFT comparison (torch.fft on the full grid; comparison only)
    cufft = None
    if not args.no_cufft:
        idx = torch.from_numpy(plan.index_map()).cuda()
        N = GRID[0] * GRID[1] * GRID[2]
        chunk = 64

        def cufft_apply():
            for b0 in range(0, NBANDS, chunk):
                Z = torch.zeros((chunk, N), dtype=torch.complex64, device="cuda")
                Z[:, idx] = c_d[b0:b0 + chunk]
                psi = torch.fft.ifftn(Z.view(chunk, *GRID), dim=(1, 2, 3), norm="forward")
                u = torch.fft.fftn(psi * V_d, dim=(1, 2, 3), norm="forward")
                out_d[b0:b0 + chunk] = u.reshape(chunk, N)[:, idx]
        kc = max(2, args.steps // 5)
        msc = time_steps(cufft_apply, kc, 1, stream, dist_on)
        cufft = {"value": world * NBANDS / (msc / kc / 1e3), "unit": "bands/s",
                 "what": "torch.fft full-grid ifftn/fftn + index scatter/gather, 64-band chunks"}

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = host_cores()
        sample = min(NBANDS, 8 * cores)  # about 10 s of wall time on 16 cores
        rate, used, dt, ref = cpu_oracle_rate(GRID, g, c64, V96.astype(np.float32), sample)
        cpu = {"value": rate, "unit": "bands/s", "cores": used, "kind": "oracle",
               "sample": f"{sample} of the 1024 bands (FP64 C oracle, OpenMP over bands), {dt:.1f} s wall"}
        # accuracy of the timed paths on the same bands (relative L2 per band,
        # max), next to the speeds
        def rel(x):
            x = x.detach().cpu().numpy().astype(np.complex128)
            return float((np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)).max())
        cs = c_d[:sample].contiguous()
        acc_f32 = rel(plan.apply(cs, V_d))
        c64s, V64s = cs.to(torch.complex128), V_d.to(torch.float64)
        acc_f64 = rel(vloc.VlocPlan(GRID, g, torch.complex128).apply(c64s, V64s))
        acc_df = rel(vloc.VlocPlan(GRID, g, torch.complex128, double_float=True).apply(c64s, V64s))
        accuracy = {"bands": sample, "f32_max_rel_l2": acc_f32, "f64_max_rel_l2": acc_f64,
                    "f64_double_float_max_rel_l2": acc_df, "gates": {"f32": 2e-6, "f64": 1e-12},
                    "reference": "FP64 oracle on the same FP32-rounded inputs"}

    # the FP64 legs' headline figures as scalars of the roofline object as well,
    # so that a reader of the line's standard keys sees them
    roofline.update({
        "fp64_native_bands_per_s": round(f64_value, 1),
        "fp64_native_frac_of_measured_dfma_rate": round(f64["roofline"]["frac"], 4),
        "fp64_double_float_bands_per_s": round(df_value, 1),
        "fp64_double_float_frac_of_fp64_B5_roofline": round(f64_df["hbm_frac_of_B5"], 4),
        "measured_dfma_gflops": alu["dfma_gflops"], "measured_ffma2_gflops": alu["ffma2_gflops"],
        "speedup_fp32_over_fp64_double_float": round(value / df_value, 3),
    })
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "bands/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(CONFIG, bands_per_gpu=NBANDS),
            "arm": {"chunk_bands": info["chunk_bands"], "ranks": world},
            "roofline": roofline, "path": path,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "fp64": f64, "fp64_double_float": f64_df, "alu_peaks": alu, "adjoint": {"value": adj, "unit": "bands/s"}, "graph_replay": graph,
            "accuracy": accuracy,
            "grid_96x96x120": {"value": c2_value, "unit": "bands/s"},
            "batched_uneven": batched, "autograd_512": autograd, "gamma_real": gamma, "half_transforms_density": halves, "eigensolve": eig,
            "cufft_comparison": cufft,
        }
        print(json.dumps(line), flush=True)
    if dist_on:
        dist.barrier()
        dist.destroy_process_group()


def main():
    global NBANDS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-cufft", action="store_true", help="skip the torch.fft comparison")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched and autograd legs")
    ap.add_argument("--only", choices=["all", "headline", "density"], default="all",
                    help="headline: only the forward apply steps; density: only the density steps "
                         "(profiler drivers)")
    ap.add_argument("--df", action="store_true", help="with --only headline --prec f64: double-float plan")
    ap.add_argument("--bands", type=int, default=NBANDS, help="bands per GPU per step (default 1024)")
    ap.add_argument("--prec", choices=["f32", "f64"], default="f32", help="precision of --only headline")
    ap.add_argument("--chunk", type=int, default=0, help="bands per workspace chunk (0: the plan's default)")
    ap.add_argument("--generic", action="store_true", help="runtime-radix kernels only (--only headline)")
    ap.add_argument("--grid", default="96,96,96", help="grid of --only headline (n1,n2,n3; R = n/4)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    NBANDS = args.bands
    rank = env_int("RANK", 0)
    world = env_int("WORLD_SIZE", 1)
    local_rank = env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
