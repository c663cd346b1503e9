"""Benchmark of the worldline Wilson-loop path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload paper|small] [--prec fp32|fp64]

One step is one pass of the whole path over the paper-scale workload
(10240 unit loops of 2048 points, flux tubes F = 1, 10, 50 with lambda = 1,
64 log-spaced T in [1e-3, 20] x 128 radii in [0, 8], 32 groups):
  loop generation (Philox -> Box-Muller -> closed, centred loops),
  Wilson group sums (FP32 compensated unless --prec fp64),
  group statistics with the full covariance of the spinor loop per profile,
  and the per-group effective action with its group error.
The metric is loop-point evaluations per second (loops x points / step time).
Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1407_7486_gb300 import inputs as I  # noqa: E402

METRIC = "loop-point evals/s (Wilson loops, FP32-compensated, |d<W>| <= 1e-6)"
FP32_LANES_PER_SM = 128
# FP64 FMA lanes per SM: GB300's double-precision pipe issues at 1/64 of the
# FP32 rate (128 / 64 = 2 per SM and clock; 152 SMs x 2 x 2 flops x 2.07 GHz
# = 1.26 TFLOP/s, the part's nominal FP64 figure).
FP64_LANES_PER_SM = 2


def sm_count(dev: int = 0) -> int:
    """Streaming multiprocessors of the device (cudaDevAttrMultiProcessorCount)."""
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def l2_bytes(dev: int = 0) -> int:
    """The device's L2 size (cudaDevAttrL2CacheSize)."""
    import torch
    return int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0) or 128 << 20)


class L2Flush:
    """Between timed iterations whose inputs fit in L2: write a buffer of
    twice the L2's size, outside the iteration's own events, so that every
    iteration starts from DRAM."""

    def __init__(self, dev: int, stream):
        import torch
        self.stream = stream
        self.buf = torch.empty(2 * l2_bytes(dev), dtype=torch.uint8, device=f"cuda:{dev}")

    def __call__(self):
        import torch
        with torch.cuda.stream(self.stream):
            self.buf.fill_(1)


def l2_note(ens_bytes: int, flushed: bool, how: str, dev: int = 0) -> str:
    """The config's statement of how timed iterations meet L2."""
    mb = ens_bytes / 1e6
    if flushed:
        return (f"inputs < L2 (loop ensemble {mb:.1f} MB, {how}): L2 flushed between timed "
                f"iterations ({2 * l2_bytes(dev) / 1e6:.0f} MB written outside their events)")
    return f"inputs > L2 (loop ensemble {mb:.0f} MB, {how})"
# Algorithmic FP32 operations per (segment, point) of the compensated walk,
# counted from the formulas in csrc/wln_wilson.cu (an FMA, a min/max or a
# select each count 1; a product added into a sum is one FMA): 16 per radius
# for the geometry (Q1 and its point 2, B, X, D 3, Q0 + B 1), the closed-form
# integrals (theta = atan2(sqrt(D), Q0 + B): sqrt(D) 1, theta/sqrt(D) 1), the
# spin bracket (B + C, D - B (B + C), the two reciprocal factors, C J1: 5),
# 1/D 1 and the two sums 2; 17 for the arctangent (range fold 2, quotient 1,
# square 1, polynomial 8, octant unfolding 4, plus t*s 1); 11 per segment
# shared by the lane's P = 4 radii (11/4); and two Kahan folds of 4
# operations every 8 segments (1).  The level passes hold P = 4 radii per
# lane too, and a segment of a sub-loop costs the same as one of the loop.
N_ALG_FP32 = 16 + 17 + 11 / 4 + 1
N_ALG_MUFU = 3      # 1/Q, 1/sqrt(D), and the reciprocal inside the arctangent
# The FP64 comparison walk (2 radii per lane): the general form, the shared
# part over 2 radii, no compensated folds.  On blocks with tan(theta) < 0.05
# it takes series long enough for double precision: int dt/Q = r f(t^2) with
# six terms (r^2, t^2, 5 FMAs, r times it) and int dt/Q^2 = 1/(Q0 Q1) +
# C r^3 h(t^2) with five terms of h (r^3, C r^3, 4 FMAs), the two sums: 23
# per radius instead of 33, 10 fewer.
N_ALG_FP64 = 16 + 17 + 11 / 2
N_ALG_FP64_TINY_SAVED = 10
# Where every segment of a block subtends at most pi/4 at the axis the kernel
# takes the arctangent's low form, which needs neither the range fold (2) nor
# the octant unfolding (4): 6 operations fewer per (segment, point).  Below
# tan(theta) = 0.18 it takes int dt/Q = r (1 - t^2/3 + t^4/5 - t^6/7 + t^8/9),
# r = 1/(Q0 + B), t^2 = D r^2 (r^2 1, t^2 1, 4 FMAs, r times it 1) instead of
# sqrt(D) (1), the quotient (1), the degree-7 polynomial (8 + 1) and
# theta/sqrt(D) (1), and 1/D by a reciprocal instead of (1/sqrt(D))^2 (1): 7
# fewer than the low form.  Below tan(theta) = 0.05 three terms of the series
# (2 FMAs fewer), and the spin as int dt/Q^2 = C r^3 (1/3 - 2 t^2/5) +
# 1/(Q0 Q1) (r^3 1, the bracket 1, two FMAs into the sum) in place of the
# bracket and its sum (6, 1/D by no reciprocal at all), with C/3 and 2C/5
# shared by the radii (2/P): 9 + 2 - 2/P fewer than the low form (MUFU: 2).
# Rows per sub-block of the ensemble statistics (kSubRows in csrc/wln_internal.cuh):
# the plain walks choose the form of theta per chunk of at most that many rows.
SUB_ROWS = 64
N_ALG_LOW_SAVED = 6
N_ALG_MID_SAVED = 7


def n_alg_tiny_saved(P: int) -> float:
    """Operations the three-term form saves against the low form, per
    (segment, radius), with P radii per lane sharing C/3 and 2C/5."""
    return 9 + 2 - 2 / P
# FP32 operations per segment of the precision guard's double-float walk
# (csrc/wln_guard.cu, counted with two-sum 6, fast two-sum 3, sum 11, accurate
# sum 20, product 7, product by a float 6, reciprocal 6, reciprocal square
# root 16, negation 0): position 17 + 6, differences 22, C, B, X, D 25 each,
# Q1 36, 1/Q1 6, 1/sqrt(D) 16, the arguments of the angle 18, the angle 153
# (fold 21, table-driven arctangent 106, unfolding 26), int dt/Q 7, the phase
# term and its sum 27, the spin bracket 61 and its sum 34: 503, plus 4 MUFU.
N_ALG_DF = 503


def low_angle_fraction(y32: np.ndarray, profiles, rhos, Ts, P: int, span: float,
                       sub_rows: int = 0):
    """Fractions of the flux-tube segment evaluations of one pass that the
    kernel walks with the pi/4 form of the arctangent or better, with the
    five-term series or better, and with the three-term series: the same
    float32 tests per (tile of P radii at one T, block of 32 loops) that the
    kernel makes from the block's longest segment and largest |y|, and with
    sub_rows > 0 (whole loops in chunks of that many rows) per sub-block of
    sub_rows rows as well: a block that does not take the three-term form
    takes, chunk by chunk, the best of its own and the sub-block's forms up
    to the five-term one (accounting only).  Returns (low, mid, short), each
    a part of the one before."""
    f = np.float32
    n_loops, _, ppl = y32.shape
    n_blocks = (n_loops + 31) // 32
    pad = n_blocks * 32 - n_loops
    up = f(1.0 + 2.0 ** -20)
    seg = np.sqrt(np.sum((np.roll(y32, -1, axis=2) - y32) ** 2, axis=1, dtype=f))   # [loop][k]
    rad = np.sqrt(np.sum(y32 * y32, axis=1, dtype=f))                                # [loop][k]

    def per_block(a, n_sub):
        a = np.concatenate([a, np.zeros((pad, a.shape[1]), f)])
        return a.reshape(n_blocks, 32, n_sub, -1).max(axis=(1, 3)) * up             # [block][sub]

    dm = per_block(seg, 1)
    rm = per_block(rad, 1)
    n_sub = 0
    if sub_rows:
        n_sub = max(1, ppl // (2 * sub_rows))
        ds = per_block(seg, n_sub)                                  # segments starting in the sub-block
        rs = per_block(np.maximum(rad, np.roll(rad, -1, axis=1)), n_sub)   # and their end points
    in_block = np.minimum(32, n_loops - 32 * np.arange(n_blocks)).astype(np.float64)

    def forms(a2, sT, rmin, lam2, d, r):
        gap = np.maximum(f(0.0), rmin[:, None, None] - sT * r[None])
        lhs = a2 * d[None]
        rhs = np.sqrt(f(lam2) + gap * gap)
        return np.where(lhs <= f(0.09) * rhs, 3,
                        np.where(lhs <= f(0.3) * rhs, 2, np.where(lhs <= f(0.9) * rhs, 1, 0)))

    low = mid = tiny = tot = 0.0
    for prof, rho, T in zip(profiles, rhos, Ts):
        if prof.kind != I.PROFILE_FLUX_TUBE:
            continue
        rho = np.asarray(rho, np.float64)
        starts = np.arange(0, len(rho), P)
        rmin = np.array([rho[a:a + P].min() for a in starts], np.float64).astype(f)
        nval = np.array([min(P, len(rho) - a) for a in starts], np.float64)
        lam2 = prof.lam * prof.lam
        for t in np.asarray(T, np.float64):
            a2 = f(2.0 * span * np.sqrt(t))
            sT = f(np.sqrt(t))
            fb = forms(a2, sT, rmin, lam2, dm, rm)                  # [tile][block][1]
            if n_sub:
                fs = forms(a2, sT, rmin, lam2, ds, rs)              # [tile][block][sub]
                fm = np.where(fb == 3, 3, np.maximum(fb, np.minimum(fs, 2)))
            else:
                fm = fb
            w = (nval[:, None] * in_block[None, :])[:, :, None] / fm.shape[2]
            low += float(((fm >= 1) * w).sum())
            mid += float(((fm >= 2) * w).sum())
            tiny += float(((fm == 3) * w).sum())
            tot += float(w.sum()) * fm.shape[2]
    return (low / tot, mid / tot, tiny / tot) if tot else (0.0, 0.0, 0.0)


def _n_alg(base: float, fr, P: int = 4) -> float:
    """Operations per (segment, radius): the general form's count less what
    each cheaper form saves (6 on the pi/4 form; 7 more on the five-term
    series, 11 - 2/P more on the three-term one)."""
    return base - N_ALG_LOW_SAVED * fr[0] - N_ALG_MID_SAVED * fr[1] - \
        (n_alg_tiny_saved(P) - N_ALG_MID_SAVED) * fr[2]


def _workload(name: str) -> I.Workload:
    if name == "paper_mapped":
        return _paper_mapped()
    if name == "sweep":
        return I.sweep(4096)
    return {"paper": I.paper, "small": I.small, "paper_slice": I.paper_slice,
            "batched": I.batched}[name]()


def _paper_mapped() -> I.Workload:
    """The paper ensemble and flux tubes with the paper's own quadrature: T and
    rho_cm on [0, inf) mapped by x = 1/(1 + v/scale) (64 times from a = 1e-3
    with T_max = 1, 128 radii with scale lambda = 1), the small-T part added
    analytically below a.  Grid nodes come from the library (wln_mapped_grid)."""
    from paper_1407_7486_gb300 import build, wln
    build.build()
    wl = I.paper()
    T = wln.mapped_grid(64, 1.0, 1e-3)
    rho = wln.mapped_grid(128, 1.0, 0.0)
    wl.name = ("paper_mapped: 10240 loops x 2048 ppl, flux tubes F=[1.0, 10.0, 50.0] lam=1, "
               "64 T mapped (T_max=1) from 1e-3 x 128 rho mapped (scale 1) from 0, "
               "small-T part below 1e-3, G=32")
    wl.rho = [rho.copy() for _ in wl.profiles]
    wl.T = [T.copy() for _ in wl.profiles]
    wl.meta["quad"] = (wln.GRID_MAPPED, wln.GRID_MAPPED, 1.0, 1.0, True)
    return wl


def _action(ctx, wl: I.Workload, S, lpg: int, where: str = "device", out=None):
    """The effective action of the step: the paper's full form (small-T part,
    mapped grids, LCF comparison) when the workload carries its quadrature,
    else Simpson on the linear/geometric grids."""
    if wl.meta.get("quad"):
        from paper_1407_7486_gb300 import wln
        quad = [wln.Quad(*wl.meta["quad"]) for _ in wl.profiles]
        r = ctx.effective_action_full(wl.profiles, wl.rho, wl.T, S, wl.n_groups, lpg, quad=quad,
                                      spinor=True, where=where)
        r["scalar"] = ctx.effective_action_full(wl.profiles, wl.rho, wl.T, S, wl.n_groups, lpg,
                                                quad=quad, spinor=False, where=where)
        return r["gamma_groups"], r["gamma"], r
    gg, ms = ctx.effective_action(wl.profiles, wl.rho, wl.T, S, wl.n_groups, lpg, spinor=True,
                                  where=where, out=out)
    return gg, ms, None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"sm_max_mhz": 2070.0, "hbm_gbs": 6800.0}, "fallback"


def _kernel_source_hash(src: str = "wln_wilson.cu") -> str:
    with open(os.path.join(ROOT, "paper_1407_7486_gb300", "csrc", src), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _ncu_value(summary: str, key: str = "dram_bytes_per_launch", src: str = "wln_wilson.cu"):
    """A figure (`key: value` line) from the committed ncu summary
    profiles/<summary>.md, or None when the kernel source `src` changed since
    the capture."""
    path = os.path.join(ROOT, "profiles", f"{summary}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    h = k = None
    for line in text.splitlines():
        if line.startswith("kernel_source_sha256_16:"):
            h = line.split(":", 1)[1].strip()
        if line.startswith(key + ":"):
            k = float(line.split(":", 1)[1].strip())
    return k if (h == _kernel_source_hash(src) and k) else None


def _ncu_traffic(summary: str):
    """DRAM bytes per Wilson launch from the committed ncu summary."""
    return _ncu_value(summary)


class ClockSampler:
    """nvidia-smi clock and throttle samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # WLN_CLOCKS_DIR keeps the raw samples somewhere the caller chooses.
        d = os.environ.get("WLN_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_buffers(wl: I.Workload, pinned: bool = True):
    """Page-locked host buffers for every output of a step, allocated once by
    the caller and reused (the fast path for device-to-host copies)."""
    import torch

    def buf(*shape):
        t = torch.empty(shape, dtype=torch.float64, pin_memory=pinned)
        return t.numpy()

    G = wl.n_groups
    b = {"S": buf(wl.n_points, G, 5), "prof": []}
    for r, t in zip(wl.rho, wl.T):
        n = len(r) * len(t)
        b["prof"].append({"ferm": {"mean": buf(n), "sem": buf(n), "jk_var": buf(n),
                                   "cov": buf(n * (n + 1) // 2)},
                          "scal": {"mean": buf(n), "sem": buf(n)}})
    b["gamma"] = (buf(len(wl.profiles), G), buf(len(wl.profiles), 2))
    return b


def run_step(ctx, wl: I.Workload, seed: int, prec: str, where: str = "device", cov: bool = True,
             loop0: int = 0, bufs=None):
    """One pass of the path; returns (outputs, h2d_bytes, d2h_bytes).  With
    `bufs` (host_buffers) every output lands in those caller-owned buffers."""
    ens = ctx.gen_loops(seed, wl.n_loops, wl.ppl, loop0=loop0)
    S = ctx.wilson_avg(ens, wl.profiles, wl.rho, wl.T, wl.n_groups, prec=prec, where=where,
                       out=bufs["S"] if bufs else None)
    lpg = wl.n_loops // wl.n_groups
    outs = {"S": S}
    off = 0
    d2h = S.nbytes if where != "device" else 0
    h2d = sum(r.nbytes + t.nbytes for r, t in zip(wl.rho, wl.T))
    for q, (r, t) in enumerate(zip(wl.rho, wl.T)):
        n = len(r) * len(t)
        Sq = S[off:off + n]
        pb = bufs["prof"][q] if bufs else {}
        jf = ctx.jackknife(Sq, wl.n_groups, lpg, 1, jk_var=True, cov="packed" if cov else False,
                           where=where,
                           out=pb.get("ferm"))
        js = ctx.jackknife(Sq, wl.n_groups, lpg, 0, jk_var=False, cov=False, where=where,
                           out=pb.get("scal"))
        outs[f"ferm{q}"] = jf
        outs[f"scal{q}"] = js
        if where != "device":
            d2h += sum(v.nbytes for v in jf.values() if v is not None)
            d2h += sum(v.nbytes for v in js.values() if v is not None)
            h2d += Sq.nbytes * 2
        off += n
    gg, ms, full = _action(ctx, wl, S, lpg, where=where, out=bufs["gamma"] if bufs else None)
    outs["gamma"] = (gg, ms)
    outs["full"] = full
    if where != "device":
        d2h += gg.nbytes + ms.nbytes
        if full is not None:       # spinor: gamma_groups and gamma counted above
            d2h += full["density"].nbytes + full["integrand"].nbytes
            d2h += sum(v.nbytes for v in full["scalar"].values())
        h2d += S.nbytes
    ens.free()
    return outs, h2d, d2h


def cpu_baseline(wl: I.Workload, gpu_ctx, prec_tol=1e-6, budget_s: float = 15.0):
    """Time the FP64 oracle on the host cores on a bounded sample of the workload
    (one flux tube, a sparse subset of points, loops of the first groups), and
    compare the GPU's group sums on that sample with it."""
    import oracle
    threads = oracle.max_threads()
    q = 1 if len(wl.profiles) > 1 else 0
    prof = wl.profiles[q]
    stride = 1 if wl.n_points <= 1024 else 4        # small configurations run in full
    rho = wl.rho[q][::stride]
    T = wl.T[q][::stride]
    lpg = wl.n_loops // wl.n_groups
    # the oracle works on the GPU ensemble's own float loops (its generator's
    # float copy can differ by one rounding at boundary cases, which would show
    # as an error of the Wilson path)
    ens = gpu_ctx.gen_loops(wl.seed, wl.n_loops, wl.ppl)
    y_all, _ = gpu_ctx.loops_copy(ens)
    # calibrate on one group at every sampled point (enough (point, group) pairs for all threads)
    y = y_all[:lpg].astype(np.float64)
    t0 = time.perf_counter()
    oracle.group_sums(y, prof, rho, T, 1, threads=threads)
    per_group = max(time.perf_counter() - t0, 1e-6)
    n_groups = int(max(1, min(wl.n_groups, budget_s / per_group)))
    y = y_all[:n_groups * lpg].astype(np.float64)
    t0 = time.perf_counter()
    ref = oracle.group_sums(y, prof, rho, T, n_groups, threads=threads)
    dt = time.perf_counter() - t0
    lp = n_groups * lpg * len(rho) * len(T)
    # one thread, one group, at most 32 of the sampled points
    y1 = y[:lpg]
    r1, t1 = rho[:8], T[:4]
    t0 = time.perf_counter()
    oracle.group_sums(y1, prof, r1, t1, 1, threads=1)
    single = lpg * len(r1) * len(t1) / (time.perf_counter() - t0)
    # GPU result on the same sample (same loops: the first n_groups groups of the ensemble)
    err = {}
    cs = _cosh_group_sums(y, prof, rho, T, n_groups)
    for prec in ("fp32", "fp64"):
        S = gpu_ctx.wilson_avg(ens, [prof], [rho], [T], wl.n_groups, prec=prec, where="host")
        S = S[:, :n_groups]
        d = np.abs(S - ref) / lpg
        rel = np.abs(S - ref)[:, :, 1] / np.maximum(np.abs(ref[:, :, 1]), lpg)
        fg, fe = _ferm_scaled_err(S, ref, cs, lpg)
        err[prec] = {"scal_max_abs": float(d[:, :, 0].max()),
                     "ferm_max_rel_to_max(1,<cosh s>)": {"group_means": fg, "mean": fe},
                     "ferm_max_rel_to_max(1,|<W>-1|)": float(rel.max())}
    ens.free()
    return {"value": lp / dt, "unit": "loop-point evals/s", "cores": threads, "kind": "oracle",
            "sample": f"F={prof.F} lam={prof.lam}, {len(rho)} rho x {len(T)} T (every {stride}), "
                      f"{n_groups * lpg} loops ({n_groups} groups) x {wl.ppl} ppl; {dt:.1f} s",
            "single_thread": {"value": single, "unit": "loop-point evals/s",
                              "sample": f"{lpg} loops x {len(r1) * len(t1)} points, 1 thread"},
            "gpu_error_vs_oracle_on_sample": err}


def _cosh_group_sums(y, prof, rho, T, n_groups: int) -> np.ndarray:
    """Sum of cosh(spin) over each group of loops [n_T * n_rho][G] (rho fastest),
    from the oracle's per-loop spins: the scale of the spinor sums, by which
    their error is measured (|d<W_ferm>| / max(1, <cosh s>))."""
    import oracle
    lpg = y.shape[0] // n_groups
    out = np.zeros((len(T) * len(rho), n_groups))
    with np.errstate(over="ignore"):
        for b, t in enumerate(T):
            for a, r in enumerate(rho):
                _, sp = oracle.phase_spin(y, prof, r, t)
                out[b * len(rho) + a] = np.cosh(sp).reshape(n_groups, lpg).sum(axis=1)
    return out


def _ferm_scaled_err(S, ref, cosh_sums, lpg: int):
    """(max over group means, max over the sample's ensemble means) of
    |d<W_ferm>| / max(1, <cosh s>); points whose cosh overflows are skipped."""
    with np.errstate(invalid="ignore", over="ignore"):
        fin = np.isfinite(ref[:, :, 1]) & np.isfinite(S[:, :, 1]) & np.isfinite(cosh_sums)
        d = np.where(fin, np.abs(S[:, :, 1] - ref[:, :, 1]), 0.0)
        g = d / np.maximum(cosh_sums, lpg)
        fe = fin.all(axis=1)
        e = np.where(fe, np.abs(np.where(fin, S[:, :, 1] - ref[:, :, 1], 0.0).sum(axis=1)), 0.0)
        e = e / np.maximum(np.where(fe, cosh_sums.sum(axis=1), 1.0), lpg * S.shape[1])
    return float(g.max()), float(e.max())


def precision_corners(wl: I.Workload, gpu_ctx, n_groups: int = 2):
    """Errors of both GPU precisions against the oracle where the spins are
    largest: for every profile, the largest and the middle T at rho = 0 and at
    the second radius, on the first n_groups groups.  The spinor error is
    measured relative to max(1, <cosh s>): cosh s has relative sensitivity
    ds to the spin, and the float spin carries a relative bias of a few 1e-8
    from the rounding of each segment's terms, so this is where the float form
    is weakest."""
    import oracle
    lpg = wl.n_loops // wl.n_groups
    y32 = oracle.gen_loops(wl.seed, n_groups * lpg, wl.ppl).astype(np.float32)
    y = y32.astype(np.float64)
    ens = gpu_ctx.ensemble_from_host(y32)
    out = []
    for prof, rho, T in zip(wl.profiles, wl.rho, wl.T):
        r_s = rho[[0, 1]] if len(rho) > 1 else rho
        t_s = T[[len(T) // 2, len(T) - 1]] if len(T) > 1 else T
        ref = oracle.group_sums(y, prof, r_s, t_s, n_groups)
        cs = _cosh_group_sums(y, prof, r_s, t_s, n_groups)
        row = {"profile": f"kind={prof.kind} F={prof.F} lam={prof.lam} B={prof.B}",
               "rho": [float(v) for v in r_s], "T": [float(v) for v in t_s],
               "mean_cosh_s_max": float(np.max(cs) / lpg)}
        for prec in ("fp32", "fp64"):
            S = gpu_ctx.wilson_avg(ens, [prof], [r_s], [t_s], n_groups, prec=prec, where="host")
            row[prec] = {"scal_max_abs": float(np.abs(S - ref)[:, :, 0].max() / lpg),
                         "ferm_max_rel_to_max(1,<cosh s>)": _ferm_scaled_err(S, ref, cs, lpg)[0]}
        out.append(row)
    ens.free()
    return {"sample": f"{n_groups} groups x {lpg} loops; per profile rho in {{0, rho_1}} x "
                      f"T in {{T_mid, T_max}}", "rows": out}


def _guard_line(guard: dict, steps: int, loop_points: int) -> dict:
    """Loops the precision guard recomputed in double-float per step (and as a
    fraction of the step's loop-point evaluations), (group, radius)
    selections it left in float because 64 loops would not bring its estimate
    under the budget, and selections dropped because its queue was full."""
    return {"escalated_loops_per_step": guard["escalated_loops"] / steps,
            "fraction_of_loop_points": guard["escalated_loops"] / steps / loop_points,
            "saturated_per_step": guard["saturated"] / steps,
            "overflows": guard["overflows"]}


def sampled_oracle_error(y32, profiles, rhos, Ts, S, n_groups: int, n_samples: int = 16,
                         seed: int = 3):
    """Error of group sums S (points ordered profile, T, rho) against the FP64
    oracle on seeded (profile, point, group) samples, the oracle working on
    the same float loops y32 [n_loops][2][ppl]: max |d<W_scal>| and max
    |d<W_ferm>| / max(1, |<W_ferm> - 1|) over the samples."""
    import oracle
    rng = np.random.default_rng(seed)
    lpg = y32.shape[0] // n_groups
    offs = np.cumsum([0] + [len(r) * len(t) for r, t in zip(rhos, Ts)])
    e_s = e_f = e_c = 0.0
    for _ in range(n_samples):
        q = int(rng.integers(len(profiles)))
        n = len(rhos[q]) * len(Ts[q])
        p, g = int(rng.integers(n)), int(rng.integers(n_groups))
        r, t = rhos[q][p % len(rhos[q])], Ts[q][p // len(rhos[q])]
        yg = y32[g * lpg:(g + 1) * lpg].astype(np.float64)
        ref = oracle.group_sums(yg, profiles[q], [r], [t], 1)[0, 0]
        got = S[offs[q] + p, g]
        e_s = max(e_s, abs(got[0] - ref[0]) / lpg)
        e_f = max(e_f, abs(got[1] - ref[1]) / max(abs(ref[1]), lpg))
        cs = _cosh_group_sums(yg, profiles[q], [r], [t], 1)[0, 0]
        if np.isfinite(cs) and np.isfinite(ref[1]):
            e_c = max(e_c, abs(got[1] - ref[1]) / max(cs, lpg))
    return {"samples": n_samples, "scal_max_abs": float(e_s),
            "ferm_max_rel_to_max(1,<cosh s>)": float(e_c),
            "ferm_max_rel_to_max(1,|<W>-1|)": float(e_f)}


def reference_arm(args, wl: I.Workload):
    """The oracle as it stands on the host cores, each step a bounded sample."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    threads = oracle.max_threads()
    q = 1 if len(wl.profiles) > 1 else 0
    prof, rho, T = wl.profiles[q], wl.rho[q][::16], wl.T[q][::16]
    y = oracle.gen_loops(wl.seed, wl.n_loops, wl.ppl, threads=threads)

    def step():
        oracle.group_sums(y, prof, rho, T, wl.n_groups, threads=threads)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    lp = wl.n_loops * len(rho) * len(T)
    v = lp / dt
    sample = (f"per step: F={prof.F}, {len(rho)} rho x {len(T)} T (every 16th), all {wl.n_loops} "
              f"loops ({wl.n_groups} groups) x {wl.ppl} ppl")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "loop-point evals/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl.name},
        "cpu_baseline": {"value": v, "unit": "loop-point evals/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "loop-point evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wln", choices=["wln", "reference"])
    ap.add_argument("--workload", default="paper",
                    choices=["paper", "small", "paper_slice", "batched", "paper_mapped", "sweep"])
    ap.add_argument("--serve", action="store_true",
                    help="replay the seed-7 Poisson request stream against the serving ensemble")
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--serve-requests", type=int, default=6,
                    help="requests of the bounded serving block in the default line (0: none)")
    ap.add_argument("--rate-scales", default="sat",
                    help="comma list: 'sat' (2000 req/s) and/or fractions of measured capacity")
    ap.add_argument("--correlation", action="store_true",
                    help="time per-loop values, randomised groups and Eq. corrcoef")
    ap.add_argument("--dloops", action="store_true",
                    help="time the d-loop generator (Eqs. yn2, ynk) on the workload's ensemble")
    ap.add_argument("--levels", action="store_true",
                    help="time the discretisation-level pass (N, N/2, N/4) and extrapolation")
    ap.add_argument("--nested", action="store_true",
                    help="with --levels: the nested loops (all, even, 0 mod 4 points)")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-guard", action="store_true",
                    help="turn the precision guard off (a comparison: the FP32 path then misses "
                         "the 1e-6 bar at strong spins)")
    args = ap.parse_args()
    wl = _workload(args.workload)

    if args.impl == "reference":
        return reference_arm(args, wl)

    import torch
    from paper_1407_7486_gb300 import build, wln

    if args.serve:
        return run_serve(args)
    if args.workload == "batched":
        return run_batched(args, wl)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.dloops:
        return run_dloops(args, wl)
    if args.levels:
        return run_levels(args, wl)
    if args.correlation:
        return run_correlation(args, wl)

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    build.build()
    dev = local if ws > 1 else 0
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    ctx = wln.Context(dev, stream)
    if args.no_guard:
        ctx.set_precision_guard(False)
    # weak scaling: rank r holds loops [r N_l, (r+1) N_l) of one ensemble (the
    # Philox counter is the global loop index), so N ranks evaluate N N_l loops
    seed, loop0 = wl.seed, rank * wl.n_loops

    # warm-up (compiles nothing; fills caches, grows scratch)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            run_step(ctx, wl, seed, args.prec, loop0=loop0)
    stream.synchronize()

    # device-resident timed region; an ensemble that fits in L2 gets a flush
    # before every step, outside the step's events
    ens_bytes = wl.n_loops * wl.ppl * 8
    flush = L2Flush(dev, stream) if ens_bytes < l2_bytes(dev) else None
    st = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    wk = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = ctx.launch_count
    ctx.precision_guard_stats(reset=True)
    _barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk, torch.cuda.stream(stream):
        e0.record(stream)
        for i in range(args.steps):
            if flush:
                flush()
            st[i][0].record(stream)
            ens = ctx.gen_loops(seed, wl.n_loops, wl.ppl, loop0=loop0)
            wk[i][0].record(stream)
            S = ctx.wilson_avg(ens, wl.profiles, wl.rho, wl.T, wl.n_groups, prec=args.prec)
            wk[i][1].record(stream)
            lpg = wl.n_loops // wl.n_groups
            off = 0
            for q, (r, t) in enumerate(zip(wl.rho, wl.T)):
                n = len(r) * len(t)
                ctx.jackknife(S[off:off + n], wl.n_groups, lpg, 1, jk_var=True, cov="packed")
                ctx.jackknife(S[off:off + n], wl.n_groups, lpg, 0, jk_var=False, cov=False)
                off += n
            _action(ctx, wl, S, lpg)
            ens.free()
            st[i][1].record(stream)
        e1.record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    _barrier(ws)
    launches = ctx.launch_count - launches0
    guard = ctx.precision_guard_stats(reset=True)
    # the whole timed region, or with flushes the steps' own events
    ms = (sum(a.elapsed_time(b) for a, b in st) if flush else e0.elapsed_time(e1)) / args.steps
    ms = _max_over_ranks(ms, ws)
    wilson_ms = statistics.mean(a.elapsed_time(b) for a, b in wk)
    loop_points = wl.loop_points
    value = loop_points * ws / (ms / 1e3)

    # end to end through the public API with host buffers: page-locked output
    # buffers the caller allocates once (outside the timed region) and reuses
    bufs = host_buffers(wl)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = args.steps
    h2d = d2h = 0
    step_ms = []
    with torch.cuda.stream(stream):
        for _ in range(e2e_steps):
            ts = time.perf_counter()
            outs, h2d, d2h = run_step(ctx, wl, seed, args.prec, where="host", cov=True,
                                      loop0=loop0, bufs=bufs)
            step_ms.append((time.perf_counter() - ts) * 1e3)
    stream.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = _max_over_ranks(e2e_s, ws)

    if rank != 0:
        ctx.close()
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    peaks, peak_kind = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = sm_count() * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12      # T FP32 ops/s
    seg = wl.segment_evals
    n_alg = N_ALG_FP32
    f_low = (0.0, 0.0, 0.0)
    if args.prec == "fp32":
        ens = ctx.gen_loops(seed, wl.n_loops, wl.ppl, loop0=loop0)
        y32, _ = ctx.loops_copy(ens)
        ens.free()
        f_low = low_angle_fraction(y32, wl.profiles, wl.rho, wl.T, 4, 1.0, sub_rows=SUB_ROWS)
        n_alg = _n_alg(N_ALG_FP32, f_low)
    # the Wilson stage (float pass, double-float recomputation, fixup) does
    # the float walk's work on every segment and the double-float walk's on
    # the segments of the loops the guard recomputes
    df_ops = N_ALG_DF * guard["escalated_loops"] / args.steps * wl.ppl if args.prec == "fp32" else 0.0
    achieved = (n_alg * seg + df_ops) / (wilson_ms / 1e3) / 1e12
    traffic = _ncu_traffic(f"wilson_kernel_{args.workload}")
    line = {
        "metric": METRIC, "value": value, "unit": "loop-point evals/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.prec == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": wl.name, "n_loops": wl.n_loops, "ppl": wl.ppl,
                   "n_points": wl.n_points, "n_groups": wl.n_groups,
                   "precision": "fp32 compensated" if args.prec == "fp32" else "fp64",
                   "covariance": "full, spinor, per profile (its upper triangle, packed)",
                   "l2": l2_note(ens_bytes, flush is not None, "regenerated every step", dev)},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_ops,
                     "unit": "T FP32 op/s", "frac": achieved / peak_ops, "traffic": traffic,
                     "kernel": "wilson_kernel<F32Comp,4,8>" if args.prec == "fp32" else "wilson_kernel<F64,2,4>",
                     "kernel_ms": wilson_ms,
                     "segment_evals_per_s": seg / (wilson_ms / 1e3),
                     "n_alg_fp32_per_segment": n_alg,
                     "n_alg_mufu_per_segment": N_ALG_MUFU - f_low[2],
                     "guard_double_float_ops": df_ops,
                     "low_angle_fraction": f_low[0], "mid_series_fraction": f_low[1],
                     "short_series_fraction": f_low[2],
                     "n_alg_basis": f"{N_ALG_FP32:g} per (segment, point), "
                                    f"{N_ALG_LOW_SAVED} fewer on the low-angle form, "
                                    f"{N_ALG_MID_SAVED} or {n_alg_tiny_saved(4):g} fewer again on its "
                                    f"five- or three-term series; plus {N_ALG_DF} per segment "
                                    f"of each loop the precision guard recomputes in double-float",
                     # context only: the same launch counted as if every segment
                     # took the general form (the rate of segment evaluations in
                     # units of the general formula's operations)
                     "general_form_equivalent": {
                         "achieved": N_ALG_FP32 * seg / (wilson_ms / 1e3) / 1e12,
                         "frac": N_ALG_FP32 * seg / (wilson_ms / 1e3) / 1e12 / peak_ops},
                     "peak_basis": f"{sm_count()} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                   f"{sm_mhz:.0f} MHz ({peak_kind} max SM clock)"},
        "e2e": {"value": loop_points * ws / e2e_s, "unit": "loop-point evals/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "step_ms": [round(v, 1) for v in step_ms]},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "precision_guard": _guard_line(guard, args.steps, loop_points)
        if args.prec == "fp32" else None,
    }
    if wl.meta.get("quad"):
        # the step's physics: spinor effective action per flux tube, mean +- group
        # SEM, against the LCF approximation on the same quadrature
        g = outs["gamma"][1]
        gs = outs["full"]["scalar"]["gamma"]
        line["effective_action"] = {
            "note": "lambda = 1 tubes, where the derivative expansion (LCF) is not expected "
                    "to hold; the e^-T/T^3 factor magnifies the statistical error of <W> at "
                    "small T (why the paper splits off the small-T part); for F = 50 the "
                    "spinor's cosh(eB T) outgrows e^-T at large T and the group spread swamps "
                    "the mean (the paper's fermion problem), while the scalar W = cos(phase) "
                    "stays bounded",
            "tubes": [{"F": p.F, "lam": p.lam,
                       "spinor": {"gamma": float(g[q, 0]), "sem": float(g[q, 1]),
                                  "lcf": float(g[q, 2])},
                       "scalar": {"gamma": float(gs[q, 0]), "sem": float(gs[q, 1]),
                                  "lcf": float(gs[q, 2])}} for q, p in enumerate(wl.profiles)]}
    # FP64 GPU path on one profile and a sparse subset of points (it is ~10^2 slower)
    if args.prec == "fp32":
        q = 1 if len(wl.profiles) > 1 else 0
        sub_rho = [wl.rho[q][::8]]
        sub_T = [wl.T[q][::4]]
        ens = ctx.gen_loops(seed, wl.n_loops, wl.ppl)
        ctx.wilson_avg(ens, [wl.profiles[q]], sub_rho, sub_T, wl.n_groups, prec="fp64")
        stream.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.wilson_avg(ens, [wl.profiles[q]], sub_rho, sub_T, wl.n_groups, prec="fp64")
        b.record(stream)
        stream.synchronize()
        n_lp = wl.n_loops * len(sub_rho[0]) * len(sub_T[0])
        f64_s = a.elapsed_time(b) / 1e3
        # the float walk's count in FP64 operations, with the share of segment
        # evaluations on the double-precision series form, against the FP64
        # pipe (the library's atan2, division and square root take more
        # operations than counted, which shows as a lower fraction)
        y64f, _ = ctx.loops_copy(ens)
        f3 = low_angle_fraction(y64f, [wl.profiles[q]], sub_rho, sub_T, 2, 1.0)[2]
        n_alg_64 = N_ALG_FP64 - N_ALG_FP64_TINY_SAVED * f3
        f64_peak = sm_count() * FP64_LANES_PER_SM * sm_mhz * 1e6 / 1e12
        f64_ach = n_alg_64 * n_lp * wl.ppl / f64_s / 1e12
        line["fp64_gpu"] = {"value": n_lp / f64_s, "unit": "loop-point evals/s",
                            "sample": f"F={wl.profiles[q].F}, {len(sub_rho[0])} rho x "
                                      f"{len(sub_T[0])} T, all loops, Wilson kernel only",
                            "roofline": {"bound": "fp64", "achieved": f64_ach, "peak": f64_peak,
                                         "unit": "T FP64 op/s", "frac": f64_ach / f64_peak,
                                         "n_alg_fp64_per_segment": n_alg_64,
                                         "series_fraction": f3,
                                         "peak_basis": f"{sm_count()} SMs x {FP64_LANES_PER_SM} "
                                                       f"FP64 lanes x {sm_mhz:.0f} MHz"},
                            # Wilson kernel rates, FP32 compensated over FP64
                            "fp32_over_fp64_rate": (wl.loop_points / (wilson_ms / 1e3)) / (n_lp / f64_s)}
        ens.free()
    if ws == 1 and args.serve_requests > 0 and args.workload == "paper":
        line["serve"] = serve_block(ctx, args.prec, args.serve_requests)
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(wl, ctx)
        pc = precision_corners(wl, ctx)
        line["precision_corners"] = pc
        # the metric's bar, |d<W>| <= 1e-6 (spinor relative to max(1, <cosh s>)), per profile
        line["bar_1e-6_met"] = {
            r["profile"]: {prec: bool(r[prec]["scal_max_abs"] <= 1e-6 and
                                     r[prec]["ferm_max_rel_to_max(1,<cosh s>)"] <= 1e-6)
                           for prec in ("fp32", "fp64")} for r in pc["rows"]}
    # the paper's own GPU figure, quoted with its hardware (context only: another
    # machine, another workload, so vs_baseline stays null)
    line["paper_context"] = {
        "gpu_rate_loop_point_evals_per_s": 5000 / 0.001315, "hardware": "NVIDIA Tesla C1060",
        "precision": "fp32", "workload": "5000 loops, one (rho_cm, T) point; ppl not stated",
        "speedup_vs_serial_cpu": 4.7553 / 0.001315}
    ctx.close()
    print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _common_line(metric, value, unit, steps, warmup, ms, dtype, config):
    return {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config}


def run_batched(args, wl: I.Workload):
    """64 flux tubes with uneven grids against one ensemble: the autotuner picks
    the kernel shape, then the whole pass (Wilson sums, statistics, per-group
    effective action) is recorded once into a CUDA graph and replayed."""
    import torch
    from paper_1407_7486_gb300 import autotune, build, wln
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream(0)
    ctx = wln.Context(0, stream)
    ens = ctx.gen_loops(wl.seed, wl.n_loops, wl.ppl)
    with torch.cuda.stream(stream):
        tuned = autotune.tune(ctx, ens, wl.profiles, wl.rho, wl.T, wl.n_groups, use_cache=False)
        b = wln.Batch(ctx, ens, wl.profiles, wl.rho, wl.T, wl.n_groups, prec=args.prec)
        b.run(graph=False)      # the first run sizes the precision guard's queue
        for _ in range(args.warmup):
            b.run(graph=True)   # the first records the graph
        stream.synchronize()
        n0 = ctx.launch_count
        ctx.precision_guard_stats(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                b.run(graph=True)
            e1.record(stream)
            stream.synchronize()
    guard = ctx.precision_guard_stats(reset=True)
    ms = e0.elapsed_time(e1) / args.steps
    S, st, g = b.results()
    peaks, peak_kind = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = sm_count() * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    seg = wl.segment_evals
    achieved = N_ALG_FP32 * seg / (ms / 1e3) / 1e12
    line = _common_line(METRIC, wl.loop_points / (ms / 1e3), "loop-point evals/s", args.steps,
                        args.warmup, ms, "f32" if args.prec == "fp32" else "f64",
                        {"workload": wl.name, "n_points": wl.n_points, "n_profiles": len(wl.profiles),
                         "graph": "one CUDA graph per pass (Wilson, reduction, statistics, action)",
                         "l2": l2_note(wl.n_loops * wl.ppl * 8, False, "resident"),
                         "tiles": {"P": b.P, "chain_blocks": b.chain, "rows": tuned["rows"],
                                   "stages": tuned["stages"], "tuner": tuned["source"]}})
    line["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak_ops,
                        "unit": "T FP32 op/s", "frac": achieved / peak_ops, "traffic": None,
                        "kernel_ms": ms, "note": "whole graph pass timed (Wilson > 99%)"}
    line["gpu_launches"] = int(ctx.launch_count - n0)
    line["clocks"] = clk.summary()
    line["precision_guard"] = _guard_line(guard, args.steps, wl.loop_points)
    # end to end through the public API: build the batch from the host grids
    # (work list upload), one graph pass, results read back to the host
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        b2 = wln.Batch(ctx, ens, wl.profiles, wl.rho, wl.T, wl.n_groups, prec=args.prec)
        b2.run(graph=True)
        S2, st2, g2 = b2.results()
        stream.synchronize()
        e2e_s = time.perf_counter() - t0
        b2.free()
    line["e2e"] = {"value": wl.loop_points / e2e_s, "unit": "loop-point evals/s",
                   "h2d_bytes_per_step": int(sum(a.nbytes for a in wl.rho + wl.T)),
                   "d2h_bytes_per_step": int(S2.nbytes + st2.nbytes + g2.nbytes)}
    y32, _ = ctx.loops_copy(ens)
    if args.prec == "fp32":
        f_low = low_angle_fraction(y32, wl.profiles, wl.rho, wl.T, b.P, 1.0, sub_rows=SUB_ROWS)
        n_alg = _n_alg(N_ALG_FP32 + 11 / b.P - 11 / 4, f_low, P=b.P)
        ach = n_alg * wl.segment_evals / (ms / 1e3) / 1e12
        line["roofline"].update({"achieved": ach, "frac": ach / line["roofline"]["peak"],
                                 "n_alg_fp32_per_segment": n_alg, "low_angle_fraction": f_low[0],
                                 "mid_series_fraction": f_low[1],
                                 "short_series_fraction": f_low[2]})
    line["gpu_error_vs_oracle_sampled"] = sampled_oracle_error(
        y32, wl.profiles, wl.rho, wl.T, S2, wl.n_groups)
    line["autotune"] = {k: v for k, v in tuned.items() if k != "candidates"}
    line["autotune_candidates"] = tuned.get("candidates")
    line["finite_gamma"] = bool(np.isfinite(g).all())
    b.free(); ens.free()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, ctx)
    ctx.close()
    print(json.dumps(line))


def run_dloops(args, wl: I.Workload):
    """The paper's d-loop generator (Eqs. yn2, ynk) on the workload's
    ensemble: one step = wln_gen_dloops (Gaussians drawn by short warps, the
    bisection levels built, centre of mass removed, float store, degeneracy
    check and block statistics) and the ensemble freed.  The roofline is the
    FP64 pipe: the draw's work is Philox in integer arithmetic and one
    double-precision Box-Muller (log, sqrt, sincospi) per point, the build's
    a few FP64 additions per point; their FP64 operations per point are
    counted by ncu (the library calls have no count of their own) and read
    from the committed summary while wln_gen.cu is unchanged."""
    import torch
    from paper_1407_7486_gb300 import build, wln
    import oracle
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream(0)
    ctx = wln.Context(0, stream)
    pts = wl.n_loops * wl.ppl
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ctx.gen_dloops(wl.seed, wl.n_loops, wl.ppl).free()
        stream.synchronize()
        n0 = ctx.launch_count
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        inc = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        with ClockSampler(0) as clk:
            for a, b in ev:
                a.record(stream)
                ctx.gen_dloops(wl.seed, wl.n_loops, wl.ppl).free()
                b.record(stream)
            launches = ctx.launch_count - n0
            for a, b in inc:      # the increment generator on the same ensemble, for context
                a.record(stream)
                ctx.gen_loops(wl.seed, wl.n_loops, wl.ppl).free()
                b.record(stream)
            stream.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        inc_ms = statistics.mean(a.elapsed_time(b) for a, b in inc)
        # end to end: the float loops copied to page-locked host memory each step
        host = torch.empty((wl.n_loops, 2, wl.ppl), dtype=torch.float32, pin_memory=True).numpy()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e = ctx.gen_dloops(wl.seed, wl.n_loops, wl.ppl)
            ctx.loops_copy(e, f32=True, out32=host)
            e.free()
        e2e_s = (time.perf_counter() - t0) / args.steps
    # the oracle on the host cores: the same construction for a bounded sample of loops
    threads = oracle.max_threads()
    n_cpu = 64
    t0 = time.perf_counter()
    ref = oracle.gen_dloops(wl.seed, n_cpu, wl.ppl, threads=threads)
    while time.perf_counter() - t0 < 10.0 and n_cpu < wl.n_loops:
        n_cpu = min(wl.n_loops, n_cpu * 2)
        t0 = time.perf_counter()
        ref = oracle.gen_dloops(wl.seed, n_cpu, wl.ppl, threads=threads)
    cpu_s = time.perf_counter() - t0
    e = ctx.gen_dloops(wl.seed, wl.n_loops, wl.ppl, keep_fp64=True)
    _, y64 = ctx.loops_copy(e, f32=False, f64=True)
    e.free()
    err = float(np.abs(y64[:n_cpu] - ref).max())
    peaks, _ = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = sm_count() * FP64_LANES_PER_SM * sm_mhz * 1e6 / 1e9          # G FP64 op/s
    ops_pt = _ncu_value(f"gen_dloops_{args.workload}", "fp64_ops_per_point", "wln_gen.cu")
    achieved = ops_pt * pts / (ms / 1e3) / 1e9 if ops_pt else None
    line = _common_line("loop-points generated/s (d-loops, Eqs. yn2 and ynk)", pts / (ms / 1e3),
                        "loop-points/s", args.steps, args.warmup, ms, "f64",
                        {"workload": f"{wl.name}: the ensemble's {wl.n_loops} loops x {wl.ppl} points "
                                     f"as d-loops", "n_loops": wl.n_loops, "ppl": wl.ppl,
                         "l2": l2_note(pts * 8, False, "written every step")})
    line["roofline"] = {"bound": "fp64", "achieved": achieved, "peak": peak, "unit": "G FP64 op/s",
                        "frac": achieved / peak if achieved else None,
                        "traffic": _ncu_value(f"gen_dloops_{args.workload}", "dram_bytes_per_launch",
                                              "wln_gen.cu"),
                        "kernel": "gen_dgauss_kernel + gen_dbuild_kernel (the whole generation call)",
                        "kernel_ms": ms, "fp64_ops_per_point": ops_pt,
                        "peak_basis": f"{sm_count()} SMs x {FP64_LANES_PER_SM} FP64 lanes x "
                                      f"{sm_mhz:.0f} MHz"}
    line["increments_ms"] = inc_ms
    line["e2e"] = {"value": pts / e2e_s, "unit": "loop-points/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": int(host.nbytes)}
    line["cpu_baseline"] = {"value": n_cpu * wl.ppl / cpu_s, "unit": "loop-points/s",
                            "cores": threads, "kind": "oracle",
                            "sample": f"the first {n_cpu} loops of the ensemble ({cpu_s:.1f} s)"}
    line["gpu_error_vs_oracle_on_sample"] = {"double_copy_max_abs": err}
    line["gpu_launches"] = int(launches)
    line["clocks"] = clk.summary()
    ctx.close()
    print(json.dumps(line))


def run_levels(args, wl: I.Workload):
    """Discretisation levels (Sec. "Estimating the Discretization
    Uncertainties"): per step, draw the ensemble, walk the three interleaved
    sub-loops of every loop at every point (one pass, N segments per loop and
    point), and extrapolate every point to infinitely many points per loop
    with its group error and discretisation uncertainty."""
    import torch
    from paper_1407_7486_gb300 import build, wln
    import oracle
    from oracle import stats as ost
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream(0)
    ctx = wln.Context(0, stream)
    lpg = wl.n_loops // wl.n_groups

    def step(where="device"):
        ens = ctx.gen_loops(wl.seed, wl.n_loops, wl.ppl)
        L = ctx.wilson_levels(ens, wl.profiles, wl.rho, wl.T, wl.n_groups, prec=args.prec,
                              where=where, nested=args.nested)
        X = ctx.extrapolate(L, wl.n_groups, lpg, where=where)
        ens.free()
        return L, X

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        stream.synchronize()
        n0 = ctx.launch_count
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        wk = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        with ClockSampler(0) as clk:
            e0.record(stream)
            for i in range(args.steps):
                ens = ctx.gen_loops(wl.seed, wl.n_loops, wl.ppl)
                wk[i][0].record(stream)
                L = ctx.wilson_levels(ens, wl.profiles, wl.rho, wl.T, wl.n_groups, prec=args.prec,
                                      nested=args.nested)
                wk[i][1].record(stream)
                X = ctx.extrapolate(L, wl.n_groups, lpg)
                ens.free()
            e1.record(stream)
            stream.synchronize()
        launches = ctx.launch_count - n0
        ms = e0.elapsed_time(e1) / args.steps
        kern_ms = statistics.mean(a.elapsed_time(b) for a, b in wk)
        t0 = time.perf_counter()
        e2e_steps = max(1, min(args.steps, 2))
        for _ in range(e2e_steps):
            Lh, Xh = step(where="host")
        stream.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = sum(r.nbytes + t.nbytes for r, t in zip(wl.rho, wl.T)) + Lh.nbytes
    d2h = Lh.nbytes + Xh.nbytes
    peaks, peak_kind = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = sm_count() * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    # paper's levels: circle N/2 + square N/4 + triangle N/4 = N segments per
    # loop and point; nested levels: N + N/2 + N/4
    seg = wl.segment_evals * (1.75 if args.nested else 1.0)
    n_alg, f_low = N_ALG_FP32, (0.0, 0.0, 0.0)
    if args.prec == "fp32":
        ens = ctx.gen_loops(wl.seed, wl.n_loops, wl.ppl)
        y32, _ = ctx.loops_copy(ens)
        ens.free()
        # sub-loop segments join points up to 4 apart
        f_low = low_angle_fraction(y32, wl.profiles, wl.rho, wl.T, 4, 4.0)
        n_alg = _n_alg(N_ALG_FP32, f_low)
    achieved = n_alg * seg / (kern_ms / 1e3) / 1e12
    line = _common_line("loop-point evals/s (discretisation levels N, N/2, N/4 + extrapolation"
                        + (", nested loops)" if args.nested else ")"),
                        wl.loop_points / (ms / 1e3), "loop-point evals/s", args.steps,
                        args.warmup, ms, "f32" if args.prec == "fp32" else "f64",
                        {"workload": wl.name, "n_loops": wl.n_loops, "ppl": wl.ppl,
                         "n_points": wl.n_points, "n_groups": wl.n_groups,
                         "l2": l2_note(wl.n_loops * wl.ppl * 8, False, "regenerated every step")})
    line["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak_ops,
                        "unit": "T FP32 op/s", "frac": achieved / peak_ops,
                        "traffic": _ncu_traffic(("wilson_nested_" if args.nested else "wilson_levels_")
                                                + args.workload),
                        "kernel": "wilson_kernel<F32Comp,4,4,%s>" % ("nested" if args.nested else "levels"),
                        "kernel_ms": kern_ms,
                        "segment_evals_per_s": seg / (kern_ms / 1e3),
                        "n_alg_fp32_per_segment": n_alg, "low_angle_fraction": f_low[0],
                        "mid_series_fraction": f_low[1], "short_series_fraction": f_low[2],
                        "peak_basis": f"{sm_count()} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                      f"{sm_mhz:.0f} MHz ({peak_kind} max SM clock)"}
    line["e2e"] = {"value": wl.loop_points / e2e_s, "unit": "loop-point evals/s",
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    line["gpu_launches"] = int(launches)
    line["clocks"] = clk.summary()
    # the extrapolation on the workload: spread of delta against the group error
    Xa = Xh.reshape(-1, 2, 6)
    line["discretisation"] = {
        "median_delta_over_sem_spinor": float(np.median(Xa[:, 1, 5] / np.maximum(Xa[:, 1, 4], 1e-300))),
        "median_delta_over_sem_scalar": float(np.median(Xa[:, 0, 5] / np.maximum(Xa[:, 0, 4], 1e-300)))}
    if not args.no_cpu_baseline:
        q = 1 if len(wl.profiles) > 1 else 0
        prof, rho, T = wl.profiles[q], wl.rho[q][::4], wl.T[q][::4]
        # the oracle on the GPU ensemble's own float loops
        ens = ctx.gen_loops(wl.seed, wl.n_loops, wl.ppl)
        y32, _ = ctx.loops_copy(ens)
        y = y32.astype(np.float64)
        t0 = time.perf_counter()
        lev = ost.nested_level_sums if args.nested else ost.level_sums
        ref = lev(oracle, y, prof, rho, T, wl.n_groups, threads=oracle.max_threads())
        dt = time.perf_counter() - t0
        G = ctx.wilson_levels(ens, [prof], [rho], [T], wl.n_groups, prec=args.prec, where="host",
                              nested=args.nested)
        ens.free()
        line["cpu_baseline"] = {
            "value": wl.n_loops * len(rho) * len(T) / dt, "unit": "loop-point evals/s",
            "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"F={prof.F}, {len(rho)} rho x {len(T)} T (every 4th), all {wl.n_loops} "
                      f"loops x {wl.ppl} ppl, levels; {dt:.1f} s",
            "gpu_error_vs_oracle_on_sample": {
                "scal_max_abs": float(np.abs(G - ref)[:, :, 0::2].max() / lpg),
                "ferm_max_rel_to_max(1,|<W>-1|)": float(
                    (np.abs(G - ref)[:, :, 1::2] / np.maximum(np.abs(ref[:, :, 1::2]), lpg)).max())}}
    ctx.close()
    print(json.dumps(line))


def _correlation_cpu(ctx, wl: I.Workload, prof, rho, T, W):
    """The oracle on the host cores for the correlation step on a bounded
    sample: every loop's W - 1 (its per-loop values) at every 8th radius and
    time for the first 1024 loops, their contiguous group sums and Eq.
    corrcoef with the sample's mid-T point at rho = 0, timed together; and
    the GPU's per-loop values on that sample against the oracle's."""
    import oracle
    from oracle import stats as ost
    threads = oracle.max_threads()
    ens = ctx.gen_loops(wl.seed, wl.n_loops, wl.ppl)
    y32, _ = ctx.loops_copy(ens)
    ens.free()
    n_cpu = min(1024, wl.n_loops)
    ir, it = np.arange(0, len(rho), 8), np.arange(0, len(T), 8)
    y = y32[:n_cpu].astype(np.float64)
    t0 = time.perf_counter()
    Wc = oracle.loop_values(y, prof, rho[ir], T[it], threads=threads)
    ost.group_sums_perm(Wc, max(2, n_cpu // (wl.n_loops // wl.n_groups)))
    ost.corrcoef_ref(Wc[:, :, 1], (len(it) // 2) * len(ir))
    cpu_s = time.perf_counter() - t0
    pts = (it[:, None] * len(rho) + ir[None, :]).ravel()
    import torch
    Wg = W[torch.as_tensor(pts, device=W.device), :n_cpu].cpu().numpy()
    # each loop's cosh(spin) scales its spinor error (the fermion factor, Sec.
    # "Uncertainties and the Fermion Problem")
    cosh = np.empty(Wc.shape[:2])
    for j, (a, b) in enumerate((t_, r_) for t_ in it for r_ in ir):
        _, sp = oracle.phase_spin(y, prof, float(rho[b]), float(T[a]), threads=threads)
        with np.errstate(over="ignore"):
            cosh[j] = np.cosh(sp)
    with np.errstate(over="ignore", invalid="ignore"):
        fin = np.isfinite(Wc[:, :, 1]) & np.isfinite(Wg[:, :, 1]) & np.isfinite(cosh)
        e_f = float(np.where(fin, np.abs(Wg[:, :, 1] - Wc[:, :, 1]) / np.maximum(1.0, cosh), 0.0).max())
    e_s = float(np.abs(Wg[:, :, 0] - Wc[:, :, 0]).max())
    cpu = {"value": n_cpu * len(pts) / cpu_s, "unit": "loop-point evals/s", "cores": threads,
           "kind": "oracle",
           "sample": f"F={prof.F}, {len(ir)} rho x {len(it)} T (every 8th), the first {n_cpu} loops "
                     f"x {wl.ppl} ppl: per-loop values, group sums, corrcoef; {cpu_s:.1f} s"}
    err = {"per_loop_scalar_max_abs": e_s,
           "per_loop_spinor_max_rel_to_max(1,cosh s)": e_f,
           "loops_x_points": int(n_cpu * len(pts))}
    return cpu, err


def run_correlation(args, wl: I.Workload):
    """Correlations between evaluations and randomised grouping (Sec.
    "Correlations between Wilson Loops", Sec. "Grouping Worldlines"): per
    step, draw the ensemble, write every loop's W - 1 at every point (the
    Wilson kernel in its per-loop mode), regroup the loops at random anew for
    every point, and take Eq. corrcoef of every point with a reference point
    over loops, fixed groups and shuffled groups.  The step's Wilson pass is
    timed on its own for the roofline."""
    import torch
    from paper_1407_7486_gb300 import build, wln
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream(0)
    ctx = wln.Context(0, stream)
    q = 1 if len(wl.profiles) > 1 else 0
    prof, rho, T = [wl.profiles[q]], [wl.rho[q]], [wl.T[q]]       # one tube: 4 GB of values
    n_points = len(rho[0]) * len(T[0])
    ref = (len(T[0]) // 2) * len(rho[0])                           # mid T, rho = 0
    W = torch.empty((n_points, wl.n_loops, 2), dtype=torch.float64, device="cuda:0")

    def step(timer=None):
        ens = ctx.gen_loops(wl.seed, wl.n_loops, wl.ppl)
        if timer:
            timer[0].record(stream)
        ctx.wilson_loops(ens, prof, rho, T, prec=args.prec, out=W)
        if timer:
            timer[1].record(stream)
        S, _ = ctx.group_sums_loops(W, wl.n_groups)
        Ss, _ = ctx.group_sums_loops(W, wl.n_groups, shuffle=True, seed=wl.seed)
        r = [ctx.corrcoef(W, ref, comp=1), ctx.corrcoef(S, ref, comp=1),
             ctx.corrcoef(Ss, ref, comp=1)]
        ens.free()
        return r

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        stream.synchronize()
        n0 = ctx.launch_count
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        wk = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        with ClockSampler(0) as clk:
            e0.record(stream)
            for i in range(args.steps):
                r = step(wk[i])
            e1.record(stream)
            stream.synchronize()
        launches = ctx.launch_count - n0
        ms = e0.elapsed_time(e1) / args.steps
        kern_ms = statistics.mean(a.elapsed_time(b) for a, b in wk)
        # end to end with host buffers: values stay on the device, the three
        # correlation curves come back
        t0 = time.perf_counter()
        e2e_steps = args.steps
        for _ in range(e2e_steps):
            ens = ctx.gen_loops(wl.seed, wl.n_loops, wl.ppl)
            ctx.wilson_loops(ens, prof, rho, T, prec=args.prec, out=W)
            S, _ = ctx.group_sums_loops(W, wl.n_groups)
            Ss, _ = ctx.group_sums_loops(W, wl.n_groups, shuffle=True, seed=wl.seed)
            rh = [ctx.corrcoef(W, ref, comp=1, where="host"), ctx.corrcoef(S, ref, comp=1, where="host"),
                  ctx.corrcoef(Ss, ref, comp=1, where="host")]
            ens.free()
        stream.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
    lp = wl.n_loops * n_points
    peaks, peak_kind = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = sm_count() * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    seg = lp * wl.ppl
    n_alg, f_low = N_ALG_FP32, (0.0, 0.0)
    if args.prec == "fp32":
        ens = ctx.gen_loops(wl.seed, wl.n_loops, wl.ppl)
        y32, _ = ctx.loops_copy(ens)
        ens.free()
        f_low = low_angle_fraction(y32, prof, rho, T, 4, 1.0, sub_rows=SUB_ROWS)
        n_alg = _n_alg(N_ALG_FP32, f_low)
    achieved = n_alg * seg / (kern_ms / 1e3) / 1e12
    line = _common_line("loop-point evals/s (per-loop values + randomised groups + Eq. corrcoef)",
                        lp / (ms / 1e3), "loop-point evals/s", args.steps, args.warmup, ms,
                        "f32" if args.prec == "fp32" else "f64",
                        {"workload": f"{wl.name}; one tube (F={prof[0].F}), per-loop values "
                                     f"{W.numel() * 8 / 1e9:.1f} GB", "n_loops": wl.n_loops,
                         "ppl": wl.ppl, "n_points": n_points, "n_groups": wl.n_groups,
                         "l2": l2_note(wl.n_loops * wl.ppl * 8, False, "regenerated every step")})
    line["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak_ops,
                        "unit": "T FP32 op/s", "frac": achieved / peak_ops,
                        "traffic": _ncu_traffic(f"wilson_loops_{args.workload}"),
                        "kernel": "wilson_kernel<F32Comp,4,4,loops>", "kernel_ms": kern_ms,
                        "segment_evals_per_s": seg / (kern_ms / 1e3),
                        "n_alg_fp32_per_segment": n_alg, "low_angle_fraction": f_low[0],
                        "mid_series_fraction": f_low[1], "short_series_fraction": f_low[2],
                        "peak_basis": f"{sm_count()} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                      f"{sm_mhz:.0f} MHz ({peak_kind} max SM clock)"}
    line["e2e"] = {"value": lp / e2e_s, "unit": "loop-point evals/s", "h2d_bytes_per_step":
                   int(sum(a.nbytes for a in rho + T)), "d2h_bytes_per_step": int(3 * n_points * 8)}
    line["gpu_launches"] = int(launches)
    line["clocks"] = clk.summary()
    if not args.no_cpu_baseline:
        line["cpu_baseline"], line["gpu_error_vs_oracle_on_sample"] = _correlation_cpu(
            ctx, wl, prof[0], rho[0], T[0], W)
    others = np.arange(n_points) != ref
    line["corr_with_reference"] = {
        "reference_point": {"T": float(T[0][ref // len(rho[0])]), "rho": 0.0},
        "median_abs_loops": float(np.nanmedian(np.abs(rh[0][others]))),
        "median_abs_groups": float(np.nanmedian(np.abs(rh[1][others]))),
        "median_abs_shuffled_groups": float(np.nanmedian(np.abs(rh[2][others])))}
    ctx.close()
    print(json.dumps(line))


def run_sweep(args):
    """Precision and discretisation sweep: 8192 loops at ppl = 256 .. 16384,
    flux tubes F in {1, 100} x lambda in {0.1, 1} on a 16 x 16 grid and
    constant fields B in {0.1, 1, 5} at rho = 0.  For every ppl and every
    precision (FP64, FP32 compensated, FP32 naive) the Wilson pass over all
    profiles is timed, and its group sums are compared with the FP64 oracle on
    two groups at a 2 x 2 sub-grid of every profile."""
    import torch
    from paper_1407_7486_gb300 import build, wln
    import oracle
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream(0)
    ctx = wln.Context(0, stream)
    rows = []
    flush = L2Flush(0, stream)
    n0 = ctx.launch_count
    with ClockSampler(0) as clk, torch.cuda.stream(stream):
        for ppl in (256, 1024, 4096, 16384):
            wl = I.sweep(ppl)
            ens_bytes = wl.n_loops * ppl * 8
            flushed = ens_bytes < l2_bytes(0)
            lpg = wl.n_loops // wl.n_groups
            ens = ctx.gen_loops(wl.seed, wl.n_loops, ppl)
            y32, _ = ctx.loops_copy(ens)
            ysub = y32[:2 * lpg].astype(np.float64)
            subs = []
            for prof, rho, T in zip(wl.profiles, wl.rho, wl.T):
                r_s = rho[[0, len(rho) // 2]] if len(rho) > 1 else rho
                t_s = T[[2, len(T) - 3]]
                subs.append((prof, r_s, t_s, oracle.group_sums(ysub, prof, r_s, t_s, 2),
                             _cosh_group_sums(ysub, prof, r_s, t_s, 2)))
            for prec in ("fp64", "fp32", "fp32_naive"):
                reps = 1 if prec == "fp64" else 3
                ctx.wilson_avg(ens, wl.profiles, wl.rho, wl.T, wl.n_groups, prec=prec)
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(reps)]
                for a, b in ev:
                    if flushed:
                        flush()
                    a.record(stream)
                    ctx.wilson_avg(ens, wl.profiles, wl.rho, wl.T, wl.n_groups, prec=prec)
                    b.record(stream)
                stream.synchronize()
                ms = sum(a.elapsed_time(b) for a, b in ev) / reps
                e_s = e_f = e_c = 0.0
                by_prof = []
                for prof, r_s, t_s, ref, cs in subs:
                    S = ctx.wilson_avg(ens, [prof], [r_s], [t_s], wl.n_groups, prec=prec,
                                       where="host")[:, :2]
                    with np.errstate(invalid="ignore", over="ignore"):
                        fin = np.isfinite(ref[:, :, 1]) & np.isfinite(S[:, :, 1])
                        e_s = max(e_s, float(np.abs(S[:, :, 0] - ref[:, :, 0]).max() / lpg))
                        rel = np.abs(S[:, :, 1] - ref[:, :, 1]) / np.maximum(np.abs(ref[:, :, 1]), lpg)
                        e_f = max(e_f, float(np.where(fin, rel, 0.0).max()))
                    by_prof.append(_ferm_scaled_err(S, ref, cs, lpg)[0])
                    e_c = max(e_c, by_prof[-1])
                rows.append({"ppl": ppl, "prec": prec, "ms": ms,
                             "l2": l2_note(ens_bytes, flushed, "resident"),
                             "ferm_max_rel_to_cosh": e_c,
                             "ferm_rel_to_cosh_by_profile": by_prof,
                             "loop_point_evals_per_s": wl.loop_points / (ms / 1e3),
                             "scal_max_abs_err": e_s, "ferm_max_rel_err": e_f})
            ens.free()
    launches = ctx.launch_count - n0
    main = next(r for r in rows if r["ppl"] == 4096 and r["prec"] == "fp32")
    line = _common_line("loop-point evals/s (precision sweep; value: FP32 compensated at ppl 4096)",
                        main["loop_point_evals_per_s"], "loop-point evals/s", 1, 1, main["ms"],
                        "f32", {"workload": "sweep: 8192 loops, ppl 256..16384, 4 flux tubes "
                                            "(F in {1, 100} x lambda in {0.1, 1}, 16 T x 16 rho) "
                                            "+ 3 constant fields at rho = 0 (16 T), G = 32",
                                "errors": "against the FP64 oracle on 2 groups x 2 x 2 points "
                                          "of every profile; spinor relative to max(1, |<W>-1|) and, per group, to "
                                          "max(1, <cosh s>)"})
    line["sweep"] = rows
    line["gpu_launches"] = int(launches)
    line["clocks"] = clk.summary()
    ctx.close()
    print(json.dumps(line))


def _serve_replay(ctx, ens, cfg, reqs, scales, prec):
    """Replay `reqs` through a continuous-batching server at each arrival-rate
    scale ('sat': the stream's own 2000 req/s; a number: that fraction of the
    capacity measured by the saturated run).  Latency runs from a request's
    arrival to its results on the host.  Returns (runs, capacity req/s)."""
    from paper_1407_7486_gb300 import wln
    runs = []
    capacity = None
    for scale in scales:
        if scale == "sat":
            times = [r.arrival_s for r in reqs]
            label = "2000 req/s (saturated)"
        else:
            if capacity is None:
                continue
            rate = float(scale) * capacity
            times = list(np.cumsum(np.random.default_rng(7).exponential(1.0 / rate, len(reqs))))
            label = f"{scale} x capacity = {rate:.3f} req/s"
        sv = wln.Server(ctx, ens, cfg["n_groups"], prec=prec, arena_bytes=16 << 30,
                        tile_groups_per_step=128)
        ctx.precision_guard_stats(reset=True)
        t0 = time.perf_counter()
        pending = list(range(len(reqs)))
        ids, done_at = {}, {}
        with ClockSampler(0) as clk:
            while len(done_at) < len(reqs):
                now = time.perf_counter() - t0
                while pending and times[pending[0]] <= now:
                    i = pending.pop(0)
                    r = reqs[i]
                    ids[i] = sv.submit(r.profile, r.rho, r.T)
                outstanding = len(ids) - len(done_at)
                if outstanding == 0:
                    if pending:
                        time.sleep(max(0.0, times[pending[0]] - (time.perf_counter() - t0)))
                    continue
                n_active, n_queued = sv.step()
                for i, rid in list(ids.items()):
                    if i in done_at:
                        continue
                    state, _ = sv.poll(rid, results=False)
                    if state == sv.DONE:
                        done_at[i] = time.perf_counter() - t0
                        sv.release(rid)
                if n_active == 0 and n_queued == 0:
                    time.sleep(0.0005)          # only finalisations in flight
        makespan = max(done_at.values()) - min(times)
        lat = np.array([done_at[i] - times[i] for i in range(len(reqs))]) * 1e3
        lp = sum(r.n_points for r in reqs) * cfg["n_loops"]
        thr = lp / makespan
        if scale == "sat":
            capacity = len(reqs) / makespan
        guard = ctx.precision_guard_stats(reset=True)
        runs.append({"rate": label, "requests": len(reqs),
                     "p50_ms": float(np.percentile(lat, 50)),
                     "p99_ms": float(np.percentile(lat, 99)), "loop_point_evals_per_s": thr,
                     "makespan_s": makespan, "steps": sv.info()["steps"], "clocks": clk.summary(),
                     "precision_guard": {"escalated_loops": guard["escalated_loops"],
                                         "saturated": guard["saturated"],
                                         "overflows": guard["overflows"]}})
        sv.free()
    return runs, capacity


def _serve_oracle_check(ctx, ens, cfg, req, prec):
    """One request through the server, its sums against the FP64 oracle on
    sampled (point, group) pairs."""
    from paper_1407_7486_gb300 import wln
    sv = wln.Server(ctx, ens, cfg["n_groups"], prec=prec, arena_bytes=16 << 30,
                    tile_groups_per_step=128)
    rid = sv.submit(req.profile, req.rho, req.T)
    for _ in range(100000):
        sv.step()
        state, res = sv.poll(rid)
        if state == sv.DONE:
            break
    y32, _ = ctx.loops_copy(ens)
    out = sampled_oracle_error(y32, [req.profile], [req.rho], [req.T], res[0], cfg["n_groups"])
    sv.release(rid)
    sv.free()
    return out


def serve_block(ctx, prec: str, n_requests: int):
    """The bounded serving measurement carried by the default line: the
    serving ensemble (32768 loops x 4096 points, 32 groups), the first
    n_requests of the seed-7 Poisson stream, saturated and replayed at half the
    measured capacity; p50/p99 latency of the half-capacity replay."""
    cfg = I.serving_ensemble()
    ens = ctx.gen_loops(cfg["seed"], cfg["n_loops"], cfg["ppl"])
    reqs = I.request_stream(n_requests)
    runs, capacity = _serve_replay(ctx, ens, cfg, reqs, ["sat", "0.5"], prec)
    half = runs[-1]
    block = {"workload": f"serving: {cfg['n_loops']} loops x {cfg['ppl']} ppl, G={cfg['n_groups']}, "
                         f"first {len(reqs)} requests of the seed-7 Poisson stream (mean 2000 req/s)",
             "p50_ms": half["p50_ms"], "p99_ms": half["p99_ms"], "rate": half["rate"],
             "loop_point_evals_per_s": half["loop_point_evals_per_s"],
             "capacity_req_per_s": capacity, "saturated": runs[0],
             "gpu_error_vs_oracle_sampled": dict(_serve_oracle_check(ctx, ens, cfg, reqs[0], prec),
                                                 request=0)}
    ens.free()
    return block


def run_serve(args):
    """Continuous batching: replay the seed-7 Poisson stream (2000 req/s) of
    single-profile queries against the serving ensemble (32768 x 4096); each
    request's latency runs from its arrival to its results on the host."""
    import torch
    from paper_1407_7486_gb300 import build, wln
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream(0)
    ctx = wln.Context(0, stream)
    cfg = I.serving_ensemble()
    ens = ctx.gen_loops(cfg["seed"], cfg["n_loops"], cfg["ppl"])
    reqs = I.request_stream(args.requests)
    runs, capacity = _serve_replay(ctx, ens, cfg, reqs, args.rate_scales.split(","), args.prec)
    line = _common_line("serve p50/p99 latency (ms) and loop-point evals/s", runs[0]["loop_point_evals_per_s"],
                        "loop-point evals/s", len(reqs), 0, None, "f32",
                        {"workload": f"serving: {cfg['n_loops']} loops x {cfg['ppl']} ppl, G={cfg['n_groups']}, "
                                     f"first {len(reqs)} requests of the seed-7 Poisson stream",
                         "arena": "16 GiB", "tile_groups_per_step": 128,
                         "l2": l2_note(cfg["n_loops"] * cfg["ppl"] * 8, False, "resident")})
    line["serve"] = runs
    line["capacity_req_per_s"] = capacity
    line["gpu_error_vs_oracle_sampled"] = dict(
        _serve_oracle_check(ctx, ens, cfg, reqs[0], args.prec), request=0)
    ens.free(); ctx.close()
    print(json.dumps(line))


if __name__ == "__main__":
    main()
