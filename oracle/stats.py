"""Group statistics and effective-action quadrature of the oracle (plain numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Inputs are group sums S[p][g][c] as produced by ``oracle.group_sums``:
c = 0: sum (W_scal - 1), 1: sum (W_ferm - 1), 2: sum sin(phase),
3: sum (W_scal - 1)^2, 4: sum (W_ferm - 1)^2, over the loops of group g
(Sec. "Grouping Worldlines": group g holds loops g n/G .. (g+1) n/G - 1).
"""
from __future__ import annotations

import functools
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


# --------------------------------------------------------------------------
# Discretisation levels (Sec. "Estimating the Discretization Uncertainties").
# --------------------------------------------------------------------------
EXTRAPOLATION = (8.0 / 3.0, -2.0, 1.0 / 3.0)   # weights of W_N, W_N/2, W_N/4


def level_terms(phase_o, spin_o, phase_sq, spin_sq, phase_tr, spin_tr):
    """Per-loop W - 1 (scalar, spinor) at the paper's three levels from the
    integrals over the three interleaved sub-loops (circle: even points, N/2;
    square: points 1 mod 4, N/4; triangle: points 3 mod 4, N/4):
      W_N/4 = e^{i (tri + sq)/2},  W_N/2 = e^{i circ},
      W_N   = e^{i circ/2} e^{i sq/4} e^{i tri/4};
    the spin integrals are combined with the same weights.  Returns
    [n][6] = (scal_N, ferm_N, scal_N/2, ferm_N/2, scal_N/4, ferm_N/4)."""
    lv = [(phase_o / 2 + phase_sq / 4 + phase_tr / 4, spin_o / 2 + spin_sq / 4 + spin_tr / 4),
          (phase_o, spin_o),
          ((phase_sq + phase_tr) / 2, (spin_sq + spin_tr) / 2)]
    out = []
    for ph, sp in lv:
        h = np.sin(0.5 * ph)
        scal = -2.0 * h * h
        sh = np.sinh(0.5 * sp)
        out += [scal, np.cos(ph) * 2.0 * sh * sh + scal]
    return np.stack(out, axis=-1)


def level_sums(oracle_mod, y, profile, rho, T, n_groups, threads=0):
    """Group sums [n_T * n_rho][G][6] of level_terms (rho fastest), with the
    sub-loop integrals from the oracle's closed-form phase and spin of each
    sub-loop (a closed polygon through its points, each segment taking proper
    time T/N', N' its point count)."""
    y = np.ascontiguousarray(y, np.float64)
    subs = [np.ascontiguousarray(y[:, :, 0::2]), np.ascontiguousarray(y[:, :, 1::4]),
            np.ascontiguousarray(y[:, :, 3::4])]
    n = y.shape[0]
    lpg = n // n_groups
    out = np.zeros((len(T) * len(rho), n_groups, 6))
    for b, t in enumerate(T):
        for a, r in enumerate(rho):
            ps = [oracle_mod.phase_spin(sub, profile, r, t, threads) for sub in subs]
            w = level_terms(ps[0][0], ps[0][1], ps[1][0], ps[1][1], ps[2][0], ps[2][1])
            out[b * len(rho) + a] = w.reshape(n_groups, lpg, 6).sum(axis=1)
    return out


def extrapolate(level_S):
    """Group sums of W_inf - 1 and of |W_N - W_inf| per (point, group) from
    level sums: the quadratic in 1/N through W_N, W_N/2, W_N/4 evaluated at
    1/N = 0 (the weights sum to one, so W - 1 sums combine the same way).
    Returns [n_points][G][2] (scalar, spinor) of extrapolated W - 1 sums."""
    a, b, c = EXTRAPOLATION
    return a * level_S[:, :, 0:2] + b * level_S[:, :, 2:4] + c * level_S[:, :, 4:6]


# --------------------------------------------------------------------------
# Full effective action (Sec. "Renormalization": small-T split; Sec.
# "Computing an Effective Action": integrals over [0, inf) mapped to a finite
# interval by x = 1/(1 + T/T_max); Sec. "Verification and Validation": LCF).
# --------------------------------------------------------------------------
GRID_LINEAR, GRID_LOG, GRID_MAPPED = 0, 1, 2


def mapped_nodes(n: int, scale: float, start: float) -> np.ndarray:
    """n ascending nodes of [start, inf) under x = 1/(1 + v/scale): x runs over
    x_k = x0 k/n, k = n .. 1 (x0 = 1/(1 + start/scale)), v = scale (1/x - 1).
    The node x = 0 (v = inf) is not stored: the integrand vanishes there."""
    x0 = 1.0 / (1.0 + start / scale)
    x = x0 * (n - np.arange(n)) / n
    v = scale * (1.0 / x - 1.0)
    v[0] = start
    return v


def mapped_weights(n: int, scale: float, start: float) -> np.ndarray:
    """Weights w such that sum_j w_j g(v_j) approximates int_start^inf g(v) dv
    on mapped_nodes: Simpson in x over the n + 1 nodes x_0 = 0 .. x_n = x0
    (g = 0 at x = 0), times dv/dx = scale / x^2."""
    x0 = 1.0 / (1.0 + start / scale)
    h = x0 / n
    ws = simpson_weights(n + 1, h)                # over x_0 .. x_n
    k = n - np.arange(n)                          # node j sits at x_k
    x = x0 * k / n
    return ws[k] * scale / (x * x)


def _bernoulli_even(n_max: int):
    """B_0, B_2, .., B_{2 n_max} as exact fractions (Akiyama-Tanigawa)."""
    from fractions import Fraction
    m_top = 2 * n_max
    a = [Fraction(0)] * (m_top + 1)
    B = []
    for m in range(m_top + 1):
        a[m] = Fraction(1, m + 1)
        for j in range(m, 0, -1):
            a[j - 1] = j * (a[j - 1] - a[j])
        B.append(a[0])                            # B_m (with B_1 = +1/2)
    return [B[2 * k] for k in range(n_max + 1)]


@functools.lru_cache(maxsize=None)
def _series_coeffs(spinor: bool, n_terms: int = 12):
    """Coefficients c_k of x^{2k}, k = 2.., of x coth x - 1 - x^2/3 (spinor) or
    x / sinh x - 1 + x^2/6 (scalar), from x coth x = sum 2^{2k} B_2k x^{2k}/(2k)!
    and x / sinh x = sum -(2^{2k} - 2) B_2k x^{2k}/(2k)!."""
    B = _bernoulli_even(n_terms + 2)
    out = []
    for k in range(2, n_terms + 2):
        f = math.factorial(2 * k)
        c = (2 ** (2 * k)) * B[k] / f if spinor else -(2 ** (2 * k) - 2) * B[k] / f
        out.append(float(c))
    return tuple(out)


def lcf_bracket(x, spinor: bool = True):
    """The constant-field bracket of the LCF integrand (Eq. LCFferm and its
    scalar counterpart): x coth x - 1 - x^2/3, or x / sinh x - 1 + x^2/6, with
    x = eB T.  Below |x| = 0.5 from the exact Taylor series (the closed form
    cancels to ~x^4 there)."""
    x = np.abs(np.asarray(x, np.float64))
    c = _series_coeffs(spinor)
    small = x < 0.5
    xs = np.where(small, x, 0.0)
    ser = np.zeros_like(x)
    for k, ck in reversed(list(enumerate(c, start=2))):
        ser = ser * xs * xs + ck
    ser = ser * xs ** 4
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        xl = np.where(small, 1.0, x)
        direct = (xl / np.tanh(xl) - 1.0 - xl * xl / 3.0) if spinor else (
            xl / np.sinh(xl) - 1.0 + xl * xl / 6.0)
    return np.where(small, ser, direct)


def small_T_integral(eB, a: float, spinor: bool = True):
    """int_0^a of the small-T expansion of the integrand, Eq. fermI (spinor)
    or Eq. scalI (scalar), m = 1, term by term."""
    b4 = np.asarray(eB, np.float64) ** 4
    b6 = np.asarray(eB, np.float64) ** 6
    if spinor:
        c = (-b4 / 45.0, b4 / 45.0, 2.0 * b6 / 945.0 - b4 / 90.0, (7.0 * b4 - 4.0 * b6) / 1890.0)
    else:
        c = (7.0 * b4 / 360.0, -7.0 * b4 / 360.0, (147.0 * b4 - 31.0 * b6) / 15120.0,
             (31.0 * b6 - 49.0 * b4) / 15120.0)
    # the term c_i T^(i+1) integrates to c_i a^(i+2) / (i+2)
    return sum(ci * a ** (i + 2) / (i + 2) for i, ci in enumerate(c))


def axis_weights(kind: int, v: np.ndarray, scale: float = 0.0) -> np.ndarray:
    """Quadrature weights of one axis (without the rho factor of rho drho):
    LINEAR: Simpson on evenly spaced v; LOG: Simpson in ln v (dv = v du);
    MAPPED: mapped_weights with start v[0]."""
    v = np.asarray(v, np.float64)
    n = len(v)
    if kind == GRID_LINEAR:
        return simpson_weights(n, (v[-1] - v[0]) / (n - 1) if n > 1 else 0.0)
    if kind == GRID_LOG:
        return simpson_weights(n, math.log(v[-1] / v[0]) / (n - 1) if n > 1 else 0.0) * v
    return mapped_weights(n, scale, v[0])


def full_effective_action(S, loops_per_group: int, profile, rho, T, rho_kind: int,
                          T_kind: int, rho_scale: float = 0.0, T_scale: float = 0.0,
                          small_T: bool = True, spinor: bool = True):
    """Per group g, the T integral at every radius,
      D_g(rho) = int_0^a I_series dT + sum_j w_j e^{-T_j}/T_j^3 (<W>_g - 1 - c (eB T_j)^2)
    (a = T_0 when small_T, Eq. fermI/scalI; c = 1/3 spinor, -1/6 scalar), and
    the action Gamma_g = (1/4 pi) sum_i w_i rho_i D_g(rho_i) (Eq. cylEA).  The
    same with the constant-field value of the bracket at eB(rho) T in place
    of <W> - 1 - c (eB T)^2 gives the LCF approximation (Eq. LCFferm).
    Returns dict: D [n_rho][G], gamma [G], D_lcf [n_rho], gamma_lcf, and the
    integrand I [n_T][n_rho][G], I_lcf [n_T][n_rho]."""
    rho = np.asarray(rho, np.float64)
    T = np.asarray(T, np.float64)
    comp = 1 if spinor else 0
    m = group_means(S, loops_per_group, comp).reshape(len(T), len(rho), -1)
    eB = eB_profile(profile, rho)
    x = eB[None, :] * T[:, None]
    ct = x * x / 3.0 if spinor else -x * x / 6.0
    pref = (np.exp(-T) / T ** 3)[:, None]
    I = pref[:, :, None] * (m - ct[:, :, None])
    I_lcf = pref * lcf_bracket(x, spinor)
    wT = axis_weights(T_kind, T, T_scale)
    wr = axis_weights(rho_kind, rho, rho_scale) * rho
    small = small_T_integral(eB, T[0], spinor) if small_T else np.zeros_like(rho)
    D = np.einsum("j,jig->ig", wT, I) + small[:, None]
    D_lcf = wT @ I_lcf + small
    return {"D": D, "gamma": wr @ D / (4.0 * math.pi), "D_lcf": D_lcf,
            "gamma_lcf": float(wr @ D_lcf / (4.0 * math.pi)), "I": I, "I_lcf": I_lcf}


# --------------------------------------------------------------------------
# Correlations between evaluations and randomised grouping (Sec.
# "Correlations between Wilson Loops", Eq. corrcoef; Sec. "Grouping
# Worldlines": new random groups for every evaluation of the integrand).
# --------------------------------------------------------------------------
def group_sums_perm(W: np.ndarray, n_groups: int, perm=None) -> np.ndarray:
    """Group sums S[p][g][c] of per-loop values W[p][l][c]: group g of point p
    holds loops perm[p][g n/G .. (g+1) n/G - 1] (perm None: loops in order,
    the contiguous groups), summed in that order."""
    n_pts, n_loops, n_c = W.shape
    lpg = n_loops // n_groups
    S = np.zeros((n_pts, n_groups, n_c))
    for p in range(n_pts):
        order = np.arange(n_loops) if perm is None else perm[p]
        for g in range(n_groups):
            acc = np.zeros(n_c)
            for k in range(g * lpg, (g + 1) * lpg):
                acc += W[p, order[k]]
            S[p, g] = acc
    return S


def corrcoef_ref(X: np.ndarray, ref: int) -> np.ndarray:
    """Eq. corrcoef between row ref and every row of X[p][n] over the n
    samples (loops, or group means):
      r_p = sum_n (X_pn - <X_p>)(X_rn - <X_r>) / sqrt(sum_n (X_pn - <X_p>)^2 sum_n (X_rn - <X_r>)^2).
    A row without spread gives NaN."""
    X = np.asarray(X, np.float64)
    d = X - X.mean(axis=1, keepdims=True)
    num = d @ d[ref]
    den = np.sqrt((d * d).sum(axis=1) * (d[ref] * d[ref]).sum())
    with np.errstate(invalid="ignore", divide="ignore"):
        return num / den


def nested_level_sums(oracle_mod, y, profile, rho, T, n_groups, threads=0):
    """Group sums [n_T * n_rho][G][6] of W - 1 (scalar, spinor) at three
    nested discretisations of every loop: all N points, the even points
    (N/2) and the points 0 mod 4 (N/4), each a closed polygon with proper time
    T/N' per segment.  These are genuine levels of one loop, so the parabola
    of EXTRAPOLATION applies to them (the paper's own combination of
    interleaved sub-loops, level_sums, is not a discretisation hierarchy)."""
    y = np.ascontiguousarray(y, np.float64)
    subs = [y, np.ascontiguousarray(y[:, :, 0::2]), np.ascontiguousarray(y[:, :, 0::4])]
    n = y.shape[0]
    lpg = n // n_groups
    out = np.zeros((len(T) * len(rho), n_groups, 6))
    for b, t in enumerate(T):
        for a, r in enumerate(rho):
            cols = []
            for sub in subs:
                ph, sp = oracle_mod.phase_spin(sub, profile, r, t, threads)
                h = np.sin(0.5 * ph)
                scal = -2.0 * h * h
                sh = np.sinh(0.5 * sp)
                cols += [scal, np.cos(ph) * 2.0 * sh * sh + scal]
            w = np.stack(cols, axis=-1)
            out[b * len(rho) + a] = w.reshape(n_groups, lpg, 6).sum(axis=1)
    return out
