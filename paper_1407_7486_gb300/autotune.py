"""Autotuner of the Wilson kernel's work decomposition.

The kernel's shape parameters are searched: radii per lane P and warps per
CTA (register pressure and occupancy against reuse of each staged loop
segment: (P, warps) in (2, 8), (4, 4), (4, 8), (8, 8)), the
float4 rows of loop data per staged chunk (loops-per-CTA tile: 32 loops x
rows), and the number of chunks in flight.  Each candidate is timed with
CUDA events on a probe: the caller's own profiles, truncated to about
`probe_seconds` of kernel time, against the caller's ensemble.  The chain
length (consecutive 32-loop blocks per work item) is left to the library's
planner, which sizes it from the full problem so that every SM gets many
items.  The winner is applied to the context (wln_set_tuning) and cached per
(GPU, points per loop, precision) in ~/.cache/wln/autotune.json.
"""
from __future__ import annotations

import itertools
import json
import os
import time
from typing import Dict, Sequence

import numpy as np

from .inputs import Profile
from . import wln

CACHE = os.path.join(os.path.expanduser("~"), ".cache", "wln", "autotune.json")
CANDIDATES = {"shape": ((2, 8), (4, 4), (4, 8), (8, 8)), "rows": (16, 32, 64),
              "stages": (2, 3, 4)}


def _key(device_name: str, ppl: int, prec: str) -> str:
    return f"{device_name}|ppl={ppl}|{prec}"


def _load_cache() -> Dict[str, dict]:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(key: str, entry: dict):
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        data = _load_cache()
        data[key] = entry
        with open(CACHE, "w") as f:
            json.dump(data, f, indent=1)
    except Exception:
        pass


def _probe(profiles, rho, T, n_loops, ppl, seg_per_s, seconds):
    """A prefix of the caller's points worth about `seconds` of kernel time."""
    target = max(256, int(seconds * seg_per_s / (n_loops * ppl)))
    P, R, TT, n = [], [], [], 0
    for p, r, t in zip(profiles, rho, T):
        if n >= target:
            break
        keep = max(1, min(len(t), (target - n) // max(1, len(r)) + 1))
        P.append(p); R.append(np.asarray(r)); TT.append(np.asarray(t)[:keep])
        n += len(r) * keep
    return P, R, TT, n


def candidates():
    """Every (P, warps, rows, stages) the search times, in a fixed order."""
    return [(P, w, r, st) for (P, w), r, st in itertools.product(
        CANDIDATES["shape"], CANDIDATES["rows"], CANDIDATES["stages"])]


def _gpu_timer(ctx, ens, pr, r, t, n_groups, prec):
    """Time one candidate (already set on ctx) with CUDA events: a warm-up run,
    then the mean of two runs of the probe batch on the context's stream."""
    import torch

    def measure() -> float:
        b = wln.Batch(ctx, ens, pr, r, t, n_groups, prec=prec)
        try:
            b.run(graph=False)                       # warm-up
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(ctx.stream)
            for _ in range(2):
                b.run(graph=False)
            z.record(ctx.stream)
            z.synchronize()
            return a.elapsed_time(z) / 2
        finally:
            b.free()
    return measure


def tune(ctx: "wln.Context", ens: "wln.Ensemble", profiles: Sequence[Profile], rho, T,
         n_groups: int, prec: str = "fp32", probe_seconds: float = 0.05, use_cache: bool = True,
         verbose: bool = False, timer=None, device_name: str = None) -> dict:
    """Pick (P, warps, rows, stages) for this ensemble and precision; returns the choice
    and the probe timings, and leaves it set on ctx.  `timer` (a function of no
    arguments returning milliseconds for the candidate currently set on ctx)
    replaces the CUDA-event timing of the probe; `device_name` the GPU's name in
    the cache key."""
    if prec == "fp64":
        ctx.set_tuning()
        return {"P": 2, "warps": 4, "rows": 32, "stages": 3, "source": "fixed for fp64"}
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    key = _key(device_name, ens.ppl, prec)
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            ctx.set_tuning(hit["P"], hit.get("warps", 8), hit["rows"], hit["stages"], 0)
            return dict(hit, source="cache")
    pr, r, t, n_pts = _probe(profiles, rho, T, ens.n_loops, ens.ppl, 7e11, probe_seconds)
    if timer is None:
        timer = _gpu_timer(ctx, ens, pr, r, t, n_groups, prec)
    results = []
    t0 = time.perf_counter()
    for P, warps, rows, stages in candidates():
        ctx.set_tuning(P, warps, rows, stages, 0)
        ms = float(timer())
        seg = n_pts * ens.n_loops * ens.ppl / (ms / 1e3)
        results.append({"P": P, "warps": warps, "rows": rows, "stages": stages, "ms": ms,
                        "seg_per_s": seg})
        if verbose:
            print(results[-1])
    best = max(results, key=lambda x: x["seg_per_s"])
    ctx.set_tuning(best["P"], best["warps"], best["rows"], best["stages"], 0)
    entry = {"P": best["P"], "warps": best["warps"], "rows": best["rows"], "stages": best["stages"],
             "seg_per_s": best["seg_per_s"], "probe_points": n_pts,
             "tuning_seconds": time.perf_counter() - t0, "candidates": results}
    _store(key, entry)
    return dict(entry, source="measured")
