"""Autotuner for V_loc plans: measures candidate configurations on the GPU
and caches the fastest per (grid, sphere, precision, band count, GPU).

Candidates:
* workspace chunk (bands per launch);
* kernel family: compile-time-length kernels (where compiled) or the
  runtime-radix kernels;
* for the runtime-radix kernels, the radix schedule of each axis: every
  ordered factorisation into at most three radices of {2,...,16}, tried axis
  by axis (coordinate descent from the planner's default).

Each candidate is timed with CUDA events on seeded synthetic inputs of the
requested shape (the real inputs do not change the timing).  The cache is a
JSON file (``VLOC_TUNE_CACHE``, default ~/.cache/vloc_tune.json).
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os
import time

import numpy as np

RADICES = (16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2)


def factorizations(n: int, max_stages: int = 3):
    """Ordered factorisations of n into supported radices (at most max_stages)."""
    out = []
    for k in range(1, max_stages + 1):
        for combo in itertools.product(RADICES, repeat=k):
            if int(np.prod(combo)) == n:
                out.append(list(combo))
    return out


def cache_path() -> str:
    return os.environ.get("VLOC_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "vloc_tune.json"))


def _key(grid, glist, dtype, nbands, gpu) -> str:
    h = hashlib.sha256(np.ascontiguousarray(np.asarray(glist, dtype=np.int32)).tobytes()).hexdigest()[:12]
    return f"{gpu}|{tuple(grid)}|{h}|{dtype}|{nbands}"


def _time_plan(plan, c, V, out, reps: int) -> float:
    import torch
    plan.apply(c, V, out=out)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        plan.apply(c, V, out=out)
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def tune(grid, glist, dtype=None, nbands: int = 256, *, reps: int = 3, chunks=(64, 128, 256, 512, 1024),
         schedules: bool = True, use_cache: bool = True, verbose: bool = False) -> dict:
    """Return the fastest configuration {"chunk", "generic", "schedule", "ms"}."""
    import torch
    from . import synth, vloc

    dtype = dtype or torch.complex64
    gpu = torch.cuda.get_device_name()
    key = _key(grid, glist, str(dtype), nbands, gpu)
    path = cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except ValueError:
            cache = {}
        if key in cache:
            return cache[key]
    rdtype = torch.float32 if dtype == torch.complex64 else torch.float64
    g = np.asarray(glist, dtype=np.int32)
    c = torch.from_numpy(synth.coefficients(g, nbands, seed=0)).to("cuda", dtype)
    V = torch.from_numpy(synth.potential(*grid, "smooth", 1000)[0]).to("cuda", rdtype)
    out = torch.empty_like(c)
    results = []

    def measure(cfg):
        plan = vloc.VlocPlan(grid, g, dtype, chunk=cfg["chunk"], generic=cfg["generic"])
        if cfg.get("schedule"):
            for a, rad in enumerate(cfg["schedule"]):
                if rad is not None:
                    plan.set_schedule(a, rad)
        ms = _time_plan(plan, c, V, out, reps)
        plan.close()
        results.append(dict(cfg, ms=ms))
        if verbose:
            print(f"  {cfg} -> {ms:.3f} ms", flush=True)
        return ms

    best = None
    for ch in sorted({min(x, nbands) for x in chunks}):
        for generic in (False, True):
            cfg = {"chunk": ch, "generic": generic, "schedule": None}
            ms = measure(cfg)
            if best is None or ms < best["ms"]:
                best = dict(cfg, ms=ms)
    if schedules:
        # coordinate descent over each axis's schedule on the runtime-radix path
        base = {"chunk": best["chunk"], "generic": True}
        plan = vloc.VlocPlan(grid, g, dtype, host_only=True)
        sched = [list(r) for r in plan.info()["radix"]]
        plan.close()
        for a in range(3):
            for rad in factorizations(grid[a]):
                if rad == sched[a]:
                    continue
                trial = [list(x) for x in sched]
                trial[a] = rad
                cfg = dict(base, schedule=trial)
                ms = measure(cfg)
                if ms < best["ms"]:
                    best = dict(cfg, ms=ms)
                    sched = trial
    best["candidates"] = len(results)
    best["when"] = time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())
    if use_cache:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        cache[key] = best
        tmp = path + f".{os.getpid()}"
        json.dump(cache, open(tmp, "w"), indent=1)
        os.replace(tmp, path)
    return best


def tuned_plan(grid, glist, dtype=None, nbands: int = 256, **kw):
    """A VlocPlan built with the tuned configuration (tuning on first use)."""
    from . import vloc
    cfg = tune(grid, glist, dtype, nbands, **kw)
    plan = vloc.VlocPlan(grid, glist, dtype, chunk=cfg["chunk"], generic=cfg["generic"])
    if cfg.get("schedule"):
        for a, rad in enumerate(cfg["schedule"]):
            if rad is not None:
                plan.set_schedule(a, rad)
    return plan, cfg
