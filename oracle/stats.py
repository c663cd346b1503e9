"""Group statistics and effective-action quadrature of the oracle (plain numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Inputs are group sums S[p][g][c] as produced by ``oracle.group_sums``:
c = 0: sum (W_scal - 1), 1: sum (W_ferm - 1), 2: sum sin(phase),
3: sum (W_scal - 1)^2, 4: sum (W_ferm - 1)^2, over the loops of group g
(Sec. "Grouping Worldlines": group g holds loops g n/G .. (g+1) n/G - 1).
"""
from __future__ import annotations

import math

import numpy as np


def group_means(S: np.ndarray, loops_per_group: int, comp: int) -> np.ndarray:
    """<W>_{G_j} - 1 (or the mean of component comp) per point and group:
    (N_G / N_l) times the group's sum (Sec. "Grouping Worldlines")."""
    return S[:, :, comp] / float(loops_per_group)


def mean_sem(S: np.ndarray, loops_per_group: int, comp: int):
    """Ensemble mean and its standard error from the spread of the group means
    (Sec. "Grouping Worldlines": the uncertainty is the standard error in the
    mean of the groups, sqrt(sum_i (<W>_Gi - <W>)^2 / (N_G (N_G - 1))))."""
    m = group_means(S, loops_per_group, comp)
    G = m.shape[1]
    mean = m.mean(axis=1)
    sem = np.sqrt(((m - mean[:, None]) ** 2).sum(axis=1) / (G * (G - 1)))
    return mean, sem


def jackknife_var(S: np.ndarray, loops_per_group: int, comp: int) -> np.ndarray:
    """Delete-one-group jackknife variance of the mean (the resampling view the
    paper names in Sec. "Grouping Worldlines"): the mean without group g,
    (G <W> - <W>_g)/(G - 1), spread as (G-1)/G sum_g (. - <W>)^2."""
    m = group_means(S, loops_per_group, comp)
    G = m.shape[1]
    mean = m.mean(axis=1)
    loo = (G * mean[:, None] - m) / (G - 1)
    return (G - 1) / G * ((loo - mean[:, None]) ** 2).sum(axis=1)


def covariance(S: np.ndarray, loops_per_group: int, comp: int) -> np.ndarray:
    """Covariance of the ensemble means between points p and q from the groups:
    sum_g (m_g(p) - <m>(p)) (m_g(q) - <m>(q)) / (G (G - 1)).  Its diagonal is
    the squared group standard error; normalising it gives the correlation
    coefficients of Eq. corrcoef for grouped loops."""
    m = group_means(S, loops_per_group, comp)
    G = m.shape[1]
    dev = m - m.mean(axis=1, keepdims=True)
    return dev @ dev.T / (G * (G - 1))


def loop_sem(S: np.ndarray, n_loops: int, comp_sum: int, comp_sq: int) -> np.ndarray:
    """Standard error in the mean over individual loops (Sec. "The Worldline
    Ensemble Distribution is not Normal"): sqrt(sum_i (W_i - <W>)^2 /
    (N_l (N_l - 1))), from the sums of (W - 1) and (W - 1)^2."""
    s1 = S[:, :, comp_sum].sum(axis=1)
    s2 = S[:, :, comp_sq].sum(axis=1)
    ss = s2 - s1 * s1 / n_loops
    return np.sqrt(np.maximum(ss, 0.0) / (n_loops * (n_loops - 1)))


# --------------------------------------------------------------------------
# Quadrature (Sec. "Computing an Effective Action": Simpson's method).
# --------------------------------------------------------------------------
def simpson_weights(n: int, h: float) -> np.ndarray:
    """Weights of composite Simpson on n equally spaced points of spacing h.
    An even n (odd number of intervals) ends with one Simpson 3/8 panel over
    the last three intervals; n = 2 is the trapezoid; n = 1 integrates over
    an empty interval."""
    w = np.zeros(n, np.float64)
    if n == 1:
        return w
    if n == 2:
        w[:] = h / 2.0
        return w
    m = n if n % 2 == 1 else n - 3     # points covered by the 1-4-2-...-4-1 part
    if m >= 3:
        w[0] += h / 3.0
        w[m - 1] += h / 3.0
        for j in range(1, m - 1):
            w[j] += (4.0 if j % 2 == 1 else 2.0) * h / 3.0
    if n % 2 == 0:
        for j, c in zip(range(n - 4, n), (1.0, 3.0, 3.0, 1.0)):
            w[j] += 3.0 * h / 8.0 * c
    return w


def eB_profile(profile, rho: np.ndarray) -> np.ndarray:
    """e B at radius rho: the flux tube's 2 calF lambda^2/(lambda^2 + rho^2)^2
    (from eB = 2 calF f'(rho^2), Sec. "Fermion Part"), or the constant B."""
    rho = np.asarray(rho, np.float64)
    if profile.kind == 1:
        return np.full_like(rho, profile.B)
    calF = profile.F / (2.0 * math.pi)
    l2 = profile.lam ** 2
    return 2.0 * calF * l2 / (l2 + rho * rho) ** 2


def quadrature_weights(rho: np.ndarray, T: np.ndarray):
    """w[b][a] such that sum_ab w[b][a] g(rho_a, T_b) approximates
    int rho drho int dT g: Simpson in rho on the evenly spaced radii, and
    Simpson in u = ln T on the log-spaced proper times, dT = T du (the
    paper maps its T range to a finite interval before Simpson; this grid
    does the same job with the map u = ln T)."""
    rho = np.asarray(rho, np.float64)
    T = np.asarray(T, np.float64)
    n_r, n_t = len(rho), len(T)
    h_r = (rho[-1] - rho[0]) / (n_r - 1) if n_r > 1 else 0.0
    h_u = math.log(T[-1] / T[0]) / (n_t - 1) if n_t > 1 else 0.0
    wr = simpson_weights(n_r, h_r) * rho
    wt = simpson_weights(n_t, h_u) * T
    return wt[:, None] * wr[None, :]


def effective_action_groups(S: np.ndarray, loops_per_group: int, profile, rho, T,
                            spinor: bool = True) -> np.ndarray:
    """Per-group effective action density (Eq. cylEA), one value per group:
    (1/4 pi) int rho drho int dT e^{-T}/T^3 {<W>_g - 1 - (eB T)^2/3} for the
    spinor loop; the scalar loop uses <W_scal>_g - 1 + (eB T)^2/6 (the
    counterterm of Eq. scalI).  Sec. "Grouping Worldlines": the integrals are
    done separately for every group and the spread of the results gives the
    error bar."""
    rho = np.asarray(rho, np.float64)
    T = np.asarray(T, np.float64)
    comp = 1 if spinor else 0
    m = group_means(S, loops_per_group, comp)            # [n_T * n_rho][G]
    G = m.shape[1]
    m = m.reshape(len(T), len(rho), G)
    eB = eB_profile(profile, rho)[None, :]
    TT = T[:, None]
    ct = (eB * TT) ** 2 / 3.0 if spinor else -(eB * TT) ** 2 / 6.0
    pref = np.exp(-TT) / TT ** 3
    w = quadrature_weights(rho, T)
    integrand = pref[:, :, None] * (m - ct[:, :, None])
    return (w[:, :, None] * integrand).sum(axis=(0, 1)) / (4.0 * math.pi)


def effective_action(S, loops_per_group, profile, rho, T, spinor=True):
    """(mean over groups, standard error over groups) of effective_action_groups."""
    g = effective_action_groups(S, loops_per_group, profile, rho, T, spinor)
    G = len(g)
    return g.mean(), math.sqrt(((g - g.mean()) ** 2).sum() / (G * (G - 1)))
