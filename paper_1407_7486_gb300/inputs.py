"""Seeded synthetic workloads for the worldline Wilson-loop path.

This module only builds inputs: grids of centre-of-mass radii and proper
times, field-profile parameters and request streams.  It holds none of the
method's arithmetic (no loops, no Wilson phases, no statistics), so both the
CUDA path and the CPU oracle can be fed from it.

Units follow the paper's cylindrical set-up (Sec. "Cylindrical Worldline
Numerics"): e = m = 1, so lambda and rho are in Compton wavelengths and the
critical field is 1.  F is the raw flux of the tube, A_phi = F f(rho)/(2 pi rho)
with f = rho^2/(lambda^2 + rho^2); the dimensionless flux is F/(2 pi).

Workloads (all loop ensembles are drawn on the device from (seed, n_loops,
ppl); nothing here stores loop coordinates):

  small      512 loops x 512 ppl, F = 10, lambda = 1, 16 log-spaced T in
             [0.01, 10], 16 linear rho in [0, 5], 8 groups.
  paper      10240 loops x 2048 ppl, F in {1, 10, 50}, lambda = 1, 64
             log-spaced T in [1e-3, 20], 128 linear rho in [0, 8], 32 groups.
  sweep      8192 loops, ppl in {256, 1024, 4096, 16384}, flux tubes with
             F in {1, 100} x lambda in {0.1, 1}, constant fields B in
             {0.1, 1, 5} at rho = 0, grids of the small workload, 32 groups.
  batched    16384 loops x 4096 ppl, 64 flux tubes drawn with host seed 4
             (F log-uniform in [0.1, 100], lambda uniform in [0.2, 3], rho
             count uniform in 8..256 over [0, 5 lambda], T count uniform in
             8..128 over [0.01, 10], log-spaced), 32 groups.
  serving    32768 loops x 4096 ppl; Poisson arrivals (mean 2000 / s, seed 7)
             of single-profile requests drawn like the batched profiles but
             with rho count 1..256 and T count 1..128; 32 groups.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np

PROFILE_FLUX_TUBE = 0
PROFILE_CONST_B = 1


@dataclass(frozen=True)
class Profile:
    """One background field.  kind 0: flux tube (F, lam); kind 1: constant B."""
    kind: int
    F: float = 0.0
    lam: float = 1.0
    B: float = 0.0


@dataclass
class Workload:
    name: str
    seed: int
    n_loops: int
    ppl: int
    n_groups: int
    profiles: List[Profile]
    rho: List[np.ndarray]          # per profile, float64
    T: List[np.ndarray]            # per profile, float64
    meta: dict = field(default_factory=dict)

    @property
    def n_points(self) -> int:
        return int(sum(len(r) * len(t) for r, t in zip(self.rho, self.T)))

    @property
    def loop_points(self) -> int:
        return self.n_points * self.n_loops

    @property
    def segment_evals(self) -> int:
        return self.loop_points * self.ppl


def log_grid(t_min: float, t_max: float, n: int) -> np.ndarray:
    """n proper times spaced evenly in ln T, end points included."""
    if n == 1:
        return np.array([t_min], dtype=np.float64)
    j = np.arange(n, dtype=np.float64)
    return t_min * (t_max / t_min) ** (j / (n - 1))


def lin_grid(a: float, b: float, n: int) -> np.ndarray:
    """n evenly spaced radii on [a, b], end points included."""
    if n == 1:
        return np.array([a], dtype=np.float64)
    return a + (b - a) * np.arange(n, dtype=np.float64) / (n - 1)


def small() -> Workload:
    return Workload("small: 512 loops x 512 ppl, flux tube F=10 lam=1, 16 T x 16 rho, G=8",
                    seed=1, n_loops=512, ppl=512, n_groups=8,
                    profiles=[Profile(PROFILE_FLUX_TUBE, F=10.0, lam=1.0)],
                    rho=[lin_grid(0.0, 5.0, 16)], T=[log_grid(0.01, 10.0, 16)])


def paper(fluxes: Sequence[float] = (1.0, 10.0, 50.0), n_loops: int = 10240,
          ppl: int = 2048, n_T: int = 64, n_rho: int = 128) -> Workload:
    profs = [Profile(PROFILE_FLUX_TUBE, F=float(F), lam=1.0) for F in fluxes]
    return Workload(f"paper: {n_loops} loops x {ppl} ppl, flux tubes F={list(fluxes)} lam=1, "
                    f"{n_T} T in [1e-3,20] x {n_rho} rho in [0,8], G=32",
                    seed=1, n_loops=n_loops, ppl=ppl, n_groups=32, profiles=profs,
                    rho=[lin_grid(0.0, 8.0, n_rho) for _ in profs],
                    T=[log_grid(1e-3, 20.0, n_T) for _ in profs])


def paper_slice() -> Workload:
    """The paper-scale ensemble against one flux tube (F = 10) on every 4th
    proper time and radius (16 x 32 points): a launch of ~1/50 the size, for
    profiling the Wilson kernel."""
    return Workload("paper slice: 10240 loops x 2048 ppl, F=10 lam=1, 16 T in [1e-3,20] x "
                    "32 rho in [0,8], G=32",
                    seed=1, n_loops=10240, ppl=2048, n_groups=32,
                    profiles=[Profile(PROFILE_FLUX_TUBE, F=10.0, lam=1.0)],
                    rho=[lin_grid(0.0, 8.0, 128)[::4]], T=[log_grid(1e-3, 20.0, 64)[::4]])


def sweep(ppl: int) -> Workload:
    profs, rhos, Ts = [], [], []
    for F in (1.0, 100.0):
        for lam in (0.1, 1.0):
            profs.append(Profile(PROFILE_FLUX_TUBE, F=F, lam=lam))
            rhos.append(lin_grid(0.0, 5.0, 16))
            Ts.append(log_grid(0.01, 10.0, 16))
    for B in (0.1, 1.0, 5.0):
        profs.append(Profile(PROFILE_CONST_B, B=B))
        rhos.append(np.zeros(1))
        Ts.append(log_grid(0.01, 10.0, 16))
    return Workload(f"sweep: 8192 loops x {ppl} ppl, 4 flux tubes + 3 constant fields, G=32",
                    seed=1, n_loops=8192, ppl=ppl, n_groups=32,
                    profiles=profs, rho=rhos, T=Ts)


def _draw_profile(rng: np.random.Generator, rho_lo: int, rho_hi: int, t_lo: int, t_hi: int):
    F = float(10.0 ** rng.uniform(-1.0, 2.0))
    lam = float(rng.uniform(0.2, 3.0))
    n_rho = int(rng.integers(rho_lo, rho_hi + 1))
    n_T = int(rng.integers(t_lo, t_hi + 1))
    return Profile(PROFILE_FLUX_TUBE, F=F, lam=lam), lin_grid(0.0, 5.0 * lam, n_rho), \
        log_grid(0.01, 10.0, n_T)


def batched(n_profiles: int = 64, n_loops: int = 16384, ppl: int = 4096,
            host_seed: int = 4) -> Workload:
    rng = np.random.default_rng(host_seed)
    profs, rhos, Ts = [], [], []
    for _ in range(n_profiles):
        p, r, t = _draw_profile(rng, 8, 256, 8, 128)
        profs.append(p); rhos.append(r); Ts.append(t)
    return Workload(f"batched: {n_profiles} flux tubes (host seed {host_seed}), "
                    f"{n_loops} loops x {ppl} ppl, G=32",
                    seed=1, n_loops=n_loops, ppl=ppl, n_groups=32,
                    profiles=profs, rho=rhos, T=Ts, meta={"host_seed": host_seed})


@dataclass
class Request:
    arrival_s: float
    profile: Profile
    rho: np.ndarray
    T: np.ndarray

    @property
    def n_points(self) -> int:
        return len(self.rho) * len(self.T)


def request_stream(n_requests: int, rate_per_s: float = 2000.0, seed: int = 7,
                   max_rho: int = 256, max_T: int = 128) -> List[Request]:
    """Poisson arrivals of single-profile queries (exponential gaps)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += float(rng.exponential(1.0 / rate_per_s))
        p, r, tt = _draw_profile(rng, 1, max_rho, 1, max_T)
        out.append(Request(t, p, r, tt))
    return out


def serving_ensemble() -> dict:
    return {"seed": 1, "n_loops": 32768, "ppl": 4096, "n_groups": 32}
