"""Pins of the oracle's statistics and quadrature.

  * Grouped jackknife (Sec. "Grouping Worldlines"): brute-force delete-one
    group means on small G; the delete-one variance equals the squared group
    standard error for a mean (an algebraic identity); the covariance
    diagonal is that square; every off-diagonal entry equals the explicit
    double sum over groups (brute force on G <= 4, and the closed form
    (m_1(p) - m_2(p)) (m_1(q) - m_2(q)) / 4 at G = 2) and the delete-one
    jackknife covariance; group means reproduce the loop mean.
  * Simpson's rule (Sec. "Computing an Effective Action"): exact on cubics
    for every point count, including the trailing 3/8 panel for even counts.
  * The effective-action quadrature (Eq. cylEA) of the locally constant
    field approximation (Eq. LCFferm) agrees with scipy's adaptive dblquad
    over the same finite domain.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import stats as ost
from paper_1407_7486_gb300.inputs import Profile, PROFILE_FLUX_TUBE, lin_grid, log_grid


def _fake_sums(rng, n_points, G, lpg):
    w = rng.normal(size=(n_points, G, lpg)) * 0.3 - 0.1
    S = np.zeros((n_points, G, 5))
    S[:, :, 0] = w.sum(axis=2)
    S[:, :, 3] = (w * w).sum(axis=2)
    return S, w


@pytest.mark.parametrize("G", [2, 3, 4])
def test_jackknife_brute_force(G):
    rng = np.random.default_rng(G)
    lpg = 5
    S, w = _fake_sums(rng, 3, G, lpg)
    mean, sem = ost.mean_sem(S, lpg, 0)
    jk = ost.jackknife_var(S, lpg, 0)
    for p in range(3):
        loops = w[p].ravel()
        assert mean[p] == pytest.approx(loops.mean(), rel=1e-13)
        loo = [np.delete(w[p], g, axis=0).ravel().mean() for g in range(G)]
        brute = (G - 1) / G * sum((x - loops.mean()) ** 2 for x in loo)
        assert jk[p] == pytest.approx(brute, rel=1e-12)
        gm = w[p].mean(axis=1)
        assert sem[p] == pytest.approx(math.sqrt(((gm - gm.mean()) ** 2).sum() / (G * (G - 1))),
                                       rel=1e-13)
        assert jk[p] == pytest.approx(sem[p] ** 2, rel=1e-12)


def test_covariance_diagonal_and_symmetry():
    rng = np.random.default_rng(9)
    S, _ = _fake_sums(rng, 6, 8, 4)
    C = ost.covariance(S, 4, 0)
    _, sem = ost.mean_sem(S, 4, 0)
    assert np.allclose(np.diag(C), sem ** 2, rtol=1e-13)
    assert np.array_equal(C, C.T)
    assert np.all(np.linalg.eigvalsh(C) > -1e-15)


@pytest.mark.parametrize("G", [2, 3, 4])
def test_covariance_off_diagonal_brute_force(G):
    """Each C(p, q), p != q, against the explicit double sum over groups of the
    products of deviations from the ensemble mean, divided by G (G - 1), and
    against the delete-one-group jackknife covariance (Sec. "Grouping
    Worldlines"; a linear statistic, so the two agree exactly)."""
    rng = np.random.default_rng(100 + G)
    lpg, n_points = 3, 5
    S, w = _fake_sums(rng, n_points, G, lpg)
    S[:, :, 0] += rng.normal(size=(n_points, G)) * 0.7   # uneven group means
    C = ost.covariance(S, lpg, 0)
    assert C.shape == (n_points, n_points)
    m = [[S[p, g, 0] / lpg for g in range(G)] for p in range(n_points)]
    for p in range(n_points):
        for q in range(n_points):
            mp, mq = sum(m[p]) / G, sum(m[q]) / G
            brute = sum((m[p][g] - mp) * (m[q][g] - mq) for g in range(G)) / (G * (G - 1))
            assert C[p, q] == pytest.approx(brute, rel=1e-12, abs=1e-15)
            loo_p = [(G * mp - m[p][g]) / (G - 1) for g in range(G)]
            loo_q = [(G * mq - m[q][g]) / (G - 1) for g in range(G)]
            jk = (G - 1) / G * sum((a - mp) * (b - mq) for a, b in zip(loo_p, loo_q))
            assert C[p, q] == pytest.approx(jk, rel=1e-11, abs=1e-15)
            if G == 2:
                closed = (m[p][0] - m[p][1]) * (m[q][0] - m[q][1]) / 4
                assert C[p, q] == pytest.approx(closed, rel=1e-12, abs=1e-15)
    off = C[~np.eye(n_points, dtype=bool)]
    assert np.any(np.abs(off) > 1e-3)   # the cross terms are exercised


def test_covariance_hand_values():
    """Three points, two groups of one loop each, values chosen by hand:
    group means (1, 3), (2, 2), (0, -4) give deviations (-1, 1), (0, 0),
    (2, -2); C(p, q) = sum_g dev_p dev_q / 2 = [[1, 0, -2], [0, 0, 0],
    [-2, 0, 4]]."""
    S = np.zeros((3, 2, 5))
    S[:, :, 0] = [[1.0, 3.0], [2.0, 2.0], [0.0, -4.0]]
    C = ost.covariance(S, 1, 0)
    assert np.array_equal(C, np.array([[1.0, 0.0, -2.0], [0.0, 0.0, 0.0], [-2.0, 0.0, 4.0]]))


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8, 16, 17, 64, 128])
def test_simpson_exact_on_cubics(n):
    a, b = -0.3, 1.9
    x = np.linspace(a, b, n)
    w = ost.simpson_weights(n, (b - a) / (n - 1))
    polys = [lambda t: 1 + 0 * t, lambda t: t] + ([lambda t: t ** 2, lambda t: t ** 3] if n >= 3 else [])
    exact = [b - a, (b ** 2 - a ** 2) / 2, (b ** 3 - a ** 3) / 3, (b ** 4 - a ** 4) / 4]
    for f, e in zip(polys, exact):
        assert np.dot(w, f(x)) == pytest.approx(e, rel=1e-13, abs=1e-14)


def test_simpson_single_point_is_zero():
    assert ost.simpson_weights(1, 0.0).tolist() == [0.0]


def test_lcf_effective_action_quadrature():
    # Flux tube, lambda = 1, F = 2 pi * 10 (calF = 10 as in Fig. igrandvsT).
    prof = Profile(PROFILE_FLUX_TUBE, F=2 * math.pi * 10.0, lam=1.0)
    t0, t1, r1 = 0.05, 4.0, 3.0
    rho = lin_grid(0.0, r1, 129)
    T = log_grid(t0, t1, 129)
    G, lpg = 2, 1
    eB = ost.eB_profile(prof, rho)
    x = eB[None, :] * T[:, None]
    lcf = x / np.tanh(x) - 1.0                      # <W> - 1 with the local constant field
    S = np.zeros((len(T) * len(rho), G, 5))
    S[:, :, 1] = lcf.reshape(-1, 1)
    g, err = ost.effective_action(S, lpg, prof, rho, T, spinor=True)
    assert err == 0.0

    def integrand(t, r):
        e = float(ost.eB_profile(prof, np.array([r]))[0]) * t
        return r * math.exp(-t) / t ** 3 * (e / math.tanh(e) - 1.0 - e * e / 3.0) / (4 * math.pi)

    ref, _ = integrate.dblquad(integrand, 0.0, r1, t0, t1, epsabs=1e-13, epsrel=1e-10)
    assert g == pytest.approx(ref, rel=1e-6)


def test_scalar_lcf_effective_action_quadrature():
    # Scalar loop: <W_scal> - 1 + (eB T)^2/6 with the constant-field x/sinh x (Eq. scalI).
    prof = Profile(PROFILE_FLUX_TUBE, F=2 * math.pi * 3.0, lam=1.5)
    t0, t1, r1 = 0.02, 6.0, 4.0
    rho = lin_grid(0.0, r1, 128)
    T = log_grid(t0, t1, 128)
    eB = ost.eB_profile(prof, rho)
    x = eB[None, :] * T[:, None]
    S = np.zeros((len(T) * len(rho), 2, 5))
    S[:, :, 0] = (x / np.sinh(x) - 1.0).reshape(-1, 1)
    g, _ = ost.effective_action(S, 1, prof, rho, T, spinor=False)

    def integrand(t, r):
        e = float(ost.eB_profile(prof, np.array([r]))[0]) * t
        return r * math.exp(-t) / t ** 3 * (e / math.sinh(e) - 1.0 + e * e / 6.0) / (4 * math.pi)

    ref, _ = integrate.dblquad(integrand, 0.0, r1, t0, t1, epsabs=1e-13, epsrel=1e-10)
    assert g == pytest.approx(ref, rel=1e-6)


def test_flux_tube_field_matches_eq_bwln():
    import sympy as sp
    F, lam = 9.0, 0.6
    r = sp.symbols("r", positive=True)
    A_phi = F * (r ** 2 / (lam ** 2 + r ** 2)) / (2 * sp.pi * r)
    Bf = sp.lambdify(r, A_phi / r + sp.diff(A_phi, r), "numpy")
    rho = np.array([0.0, 0.1, 0.5, 1.0, 3.0, 8.0])
    got = ost.eB_profile(Profile(PROFILE_FLUX_TUBE, F=F, lam=lam), rho)
    want = np.array([Bf(max(x, 1e-12)) for x in rho])
    assert np.allclose(got, want, rtol=1e-12)


def test_extrapolation_weights_are_the_quadratic_in_one_over_N():
    # Lagrange interpolation in x = 1/N through N, N/2, N/4, evaluated at x = 0
    N = 512.0
    xs = np.array([1 / N, 2 / N, 4 / N])
    for coeffs in ([1.0, 0.0, 0.0], [0.3, -2.0, 5.0], [1.0, 7.0, -40.0]):
        f = np.polyval(coeffs[::-1], xs)        # f(x) = c0 + c1 x + c2 x^2
        got = np.dot(ost.EXTRAPOLATION, f)
        assert got == pytest.approx(coeffs[0], rel=1e-12, abs=1e-12)
    assert sum(ost.EXTRAPOLATION) == pytest.approx(1.0)


def test_half_loop_level_matches_exact_constant_field_average():
    import oracle
    from paper_1407_7486_gb300.inputs import PROFILE_CONST_B
    # the circle sub-loop (every other point) is an N/2-point loop, so in a
    # constant field <W_N/2> is the exact finite-N average at N/2 points
    N, n_loops, G, b = 64, 12800, 32, 1.5
    y = oracle.gen_loops(61, n_loops, N)
    L = ost.level_sums(oracle, y, Profile(PROFILE_CONST_B, B=b), [0.0], [1.0], G)
    m, e = ost.mean_sem(L, n_loops // G, 2)
    k = np.arange(1, N // 2)
    exact = float(np.prod((1.0 + (b / ((N // 2) * np.tan(np.pi * k / (N // 2)))) ** 2) ** -0.5))
    assert abs(1.0 + m[0] - exact) < 5 * e[0]


def _regular_polygon(n, R):
    k = np.arange(n)
    return np.stack([R * np.cos(2 * np.pi * k / n), R * np.sin(2 * np.pi * k / n)])[None]


def test_levels_of_a_regular_polygon_in_a_constant_field():
    import oracle
    from paper_1407_7486_gb300.inputs import PROFILE_CONST_B
    # the sub-loops of a regular 16-gon are a regular 8-gon (even points) and
    # two regular 4-gons (1 mod 4, 3 mod 4); in a constant field each phase
    # is B times the enclosed area (n/2) R^2 sin(2 pi/n), each spin is B T
    R, B, T = 0.6, 1.7, 1.0
    y = _regular_polygon(16, R)
    area = lambda n: 0.5 * n * R * R * np.sin(2 * np.pi / n)
    L = ost.level_sums(oracle, y, Profile(PROFILE_CONST_B, B=B), [0.0], [T], 1)[0, 0]
    phases = [B * (area(8) / 2 + area(4) / 4 + area(4) / 4), B * area(8), B * area(4)]
    for lv, ph in enumerate(phases):
        assert L[2 * lv] == pytest.approx(np.cos(ph) - 1.0, rel=1e-12, abs=1e-14)
        assert L[2 * lv + 1] == pytest.approx(np.cos(ph) * np.cosh(B * T) - 1.0, rel=1e-12)


def test_levels_of_a_wide_flux_tube_approach_the_constant_field():
    import oracle
    from paper_1407_7486_gb300.inputs import PROFILE_CONST_B
    # near the axis of a tube much wider than the loop the field is uniform,
    # e B = F / (pi lambda^2); the sub-loop spins then sum T/N' per segment to
    # B T on every sub-loop (a wrong proper time per segment scales them by
    # N'/N), and the phases approach B times the areas
    lam, Beff, T = 1.0e3, 0.7, 1.3
    F = Beff * np.pi * lam * lam
    y = oracle.gen_loops(3, 4, 64)
    tube = ost.level_sums(oracle, y, Profile(0, F=F, lam=lam), [0.0], [T], 4)
    const = ost.level_sums(oracle, y, Profile(PROFILE_CONST_B, B=Beff), [0.0], [T], 4)
    np.testing.assert_allclose(tube, const, rtol=1e-5, atol=1e-9)


def test_small_T_series_integral_matches_sympy_expansion():
    sp = pytest.importorskip("sympy")
    T, b, a = sp.symbols("T b a", positive=True)
    for spinor in (True, False):
        br = b * T / sp.tanh(b * T) - 1 - (b * T) ** 2 / 3 if spinor else \
            b * T / sp.sinh(b * T) - 1 + (b * T) ** 2 / 6
        ser = sp.series(sp.exp(-T) / T ** 3 * br, T, 0, 5).removeO()
        integral = sp.integrate(ser, (T, 0, a))
        for bv, av in ((0.7, 0.05), (3.0, 0.01), (0.2, 0.3)):
            want = float(integral.subs({b: bv, a: av}))
            got = float(ost.small_T_integral(bv, av, spinor))
            assert got == pytest.approx(want, rel=1e-12, abs=1e-300)


def test_lcf_bracket_matches_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for x in (1e-6, 1e-3, 0.1, 0.4999, 0.5001, 1.0, 7.0, 40.0, 400.0):
        f = float(x * mp.coth(x) - 1 - mp.mpf(x) ** 2 / 3)
        s = float(x / mp.sinh(x) - 1 + mp.mpf(x) ** 2 / 6)
        assert float(ost.lcf_bracket(x, True)) == pytest.approx(f, rel=1e-12)
        assert float(ost.lcf_bracket(x, False)) == pytest.approx(s, rel=1e-12, abs=1e-300)


def test_mapped_quadrature_on_known_integrals():
    # int_a^inf e^{-v} dv = e^{-a};  int_a^inf v^2 e^{-v} dv = (a^2 + 2a + 2) e^{-a}:
    # Simpson in x converges at least like h^4 (the mapped integrand is smooth
    # at x = 0, where every derivative vanishes)
    cases = ((lambda v: np.exp(-v), lambda a: np.exp(-a)),
             (lambda v: v * v * np.exp(-v), lambda a: (a * a + 2 * a + 2) * np.exp(-a)))
    for scale, a in ((1.0, 0.01), (3.0, 0.2), (0.5, 0.0)):
        for f, F in cases:
            err = []
            for n in (64, 128, 256):
                v = ost.mapped_nodes(n, scale, a)
                w = ost.mapped_weights(n, scale, a)
                assert np.all(np.diff(v) > 0) and v[0] == a
                err.append(abs(w @ f(v) / F(a) - 1.0))
            assert err[2] < 1e-9
            assert err[1] <= max(err[0] / 16.0, 1e-11) and err[2] <= max(err[1] / 16.0, 1e-11)
    # an even node count (odd interval count) takes the 3/8 panel
    v, w = ost.mapped_nodes(129, 1.0, 0.1), ost.mapped_weights(129, 1.0, 0.1)
    assert w @ np.exp(-v) == pytest.approx(np.exp(-0.1), rel=1e-8)


def test_full_lcf_action_matches_adaptive_quadrature():
    sc = pytest.importorskip("scipy.integrate")
    # flux tube, LCF: (1/4 pi) int_0^inf rho drho int_0^inf dT e^{-T}/T^3 bracket(eB(rho) T)
    prof = Profile(0, F=2 * np.pi * 10.0, lam=1.0)
    for spinor in (True, False):
        a = 0.01
        T = ost.mapped_nodes(96, 1.0, a)
        rho = ost.mapped_nodes(96, 1.5, 0.0)
        S = np.zeros((len(T) * len(rho), 2, 5))
        r = ost.full_effective_action(S, 10, prof, rho, T, ost.GRID_MAPPED, ost.GRID_MAPPED,
                                      rho_scale=1.5, T_scale=1.0, spinor=spinor)

        def inner(rr):
            eB = float(ost.eB_profile(prof, np.array([rr]))[0])
            f = lambda t: np.exp(-t) / t ** 3 * float(ost.lcf_bracket(eB * t, spinor))
            return sc.quad(f, 0, 1, epsabs=0, epsrel=1e-11, limit=200)[0] + \
                sc.quad(f, 1, np.inf, epsabs=0, epsrel=1e-11, limit=200)[0]

        # T integral at a few radii (small-T series + mapped Simpson vs adaptive)
        for i in (0, 20, 60):
            assert r["D_lcf"][i] == pytest.approx(inner(rho[i]), rel=2e-5)
        want = sc.quad(lambda rr: rr * inner(rr), 0, np.inf, epsabs=0, epsrel=1e-8,
                       limit=200)[0] / (4 * np.pi)
        assert r["gamma_lcf"] == pytest.approx(want, rel=1e-4)


def test_full_action_of_constant_field_averages_equals_lcf():
    # with the continuum constant-field averages as <W>, every group reproduces
    # the LCF result exactly (same quadrature): W_ferm - 1 = x coth x - 1 and
    # W_scal - 1 = x / sinh x - 1 at x = eB(rho) T
    prof = Profile(0, F=20.0, lam=0.7)
    T = ost.mapped_nodes(24, 1.0, 0.02)
    rho = np.linspace(0.0, 3.0, 17)
    eB = ost.eB_profile(prof, rho)
    x = eB[None, :] * T[:, None]
    G, lpg = 4, 8
    S = np.zeros((len(T) * len(rho), G, 5))
    S[:, :, 1] = ((ost.lcf_bracket(x, True) + x * x / 3.0).reshape(-1) * lpg)[:, None]
    S[:, :, 0] = ((ost.lcf_bracket(x, False) - x * x / 6.0).reshape(-1) * lpg)[:, None]
    for spinor in (True, False):
        r = ost.full_effective_action(S, lpg, prof, rho, T, ost.GRID_LINEAR, ost.GRID_MAPPED,
                                      T_scale=1.0, spinor=spinor)
        np.testing.assert_allclose(r["D"], np.repeat(r["D_lcf"][:, None], G, 1), rtol=1e-9,
                                   atol=1e-12)
        np.testing.assert_allclose(r["gamma"], r["gamma_lcf"], rtol=1e-9)


def test_shuffle_is_a_uniform_permutation():
    import oracle
    from itertools import permutations
    for n in (1, 2, 7, 100, 1000):
        a = oracle.shuffle(11, 3, n)
        assert sorted(a.tolist()) == list(range(n))
    # all 24 orders of 4 loops, equally often over 24000 evaluations (chi-square)
    idx = {p: i for i, p in enumerate(permutations(range(4)))}
    counts = np.zeros(24)
    for point in range(24000):
        counts[idx[tuple(oracle.shuffle(5, point, 4).tolist())]] += 1
    chi2 = ((counts - 1000.0) ** 2 / 1000.0).sum()
    assert chi2 < 60.0          # 23 degrees of freedom: P(chi2 > 60) ~ 4e-5
    # every loop lands in every position equally often (n = 10)
    pos = np.zeros((10, 10))
    for point in range(20000):
        a = oracle.shuffle(9, point, 10)
        pos[a, np.arange(10)] += 1
    assert np.abs(pos / 2000.0 - 1.0).max() < 0.12
    # different evaluations, different orders; the same evaluation, the same order
    assert not np.array_equal(oracle.shuffle(1, 0, 50), oracle.shuffle(1, 1, 50))
    assert np.array_equal(oracle.shuffle(1, 7, 50), oracle.shuffle(1, 7, 50))


def test_grouping_by_permutation():
    rng = np.random.default_rng(3)
    W = rng.normal(size=(3, 12, 2))
    # identity order = the contiguous groups of the paper's default grouping
    S = ost.group_sums_perm(W, 4)
    np.testing.assert_allclose(S, W.reshape(3, 4, 3, 2).sum(axis=2), rtol=1e-15)
    perm = np.stack([rng.permutation(12) for _ in range(3)])
    Sp = ost.group_sums_perm(W, 4, perm)
    np.testing.assert_allclose(Sp.sum(axis=1), W.sum(axis=1), rtol=1e-13)   # totals kept
    for p in range(3):
        for g in range(4):
            np.testing.assert_allclose(Sp[p, g], W[p, perm[p, 3 * g:3 * g + 3]].sum(axis=0),
                                       rtol=1e-15)


def test_corrcoef_definition():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(6, 500))
    X[1] = 3.0 * X[0] + 2.0          # exact linear relation: +1
    X[2] = -0.5 * X[0]               # exact inverse relation: -1
    r = ost.corrcoef_ref(X, 0)
    assert r[0] == pytest.approx(1.0, abs=1e-14)
    assert r[1] == pytest.approx(1.0, abs=1e-14) and r[2] == pytest.approx(-1.0, abs=1e-14)
    assert np.all(np.abs(r[3:]) < 5.0 / np.sqrt(500))     # independent rows: ~0
    np.testing.assert_allclose(r, np.corrcoef(X)[0], rtol=1e-12, atol=1e-15)
    assert np.isnan(ost.corrcoef_ref(np.vstack([X[:1], np.ones((1, 500))]), 0)[1])


def test_shuffled_groups_remove_point_to_point_correlation():
    # Fig. corr: W at two evaluations built on the same loops is correlated loop by
    # loop, and so are the means of fixed groups; new random groups for every
    # evaluation remove the correlation between the group means
    import oracle
    rng = np.random.default_rng(6)
    n_loops, G = 6400, 64
    z = rng.normal(size=n_loops)
    W = np.stack([z + 0.3 * rng.normal(size=n_loops) for _ in range(8)])[:, :, None]
    lpg = n_loops // G
    loops = ost.corrcoef_ref(W[:, :, 0], 0)
    fixed = ost.corrcoef_ref(ost.group_sums_perm(W, G)[:, :, 0] / lpg, 0)
    perm = np.stack([oracle.shuffle(21, p, n_loops) for p in range(8)])
    shuffled = ost.corrcoef_ref(ost.group_sums_perm(W, G, perm)[:, :, 0] / lpg, 0)
    assert np.all(loops[1:] > 0.85) and np.all(fixed[1:] > 0.8)
    assert np.all(np.abs(shuffled[1:]) < 4.0 / np.sqrt(G))


def test_loop_values_sum_to_group_sums():
    import oracle
    y = oracle.gen_loops(8, 24, 64)
    prof, rho, T = Profile(0, F=10.0, lam=1.0), np.array([0.0, 0.7]), np.array([0.1, 2.0])
    W = oracle.loop_values(y, prof, rho, T)
    S = oracle.group_sums(y, prof, rho, T, 3)
    np.testing.assert_allclose(ost.group_sums_perm(W, 3), S[:, :, :2], rtol=1e-13, atol=1e-15)


def _exact_const(b, N):
    k = np.arange(1, N)
    return float(np.prod((1.0 + (b / (N * np.tan(np.pi * k / N))) ** 2) ** -0.5))


def test_nested_levels_are_the_exact_finite_N_averages_and_extrapolate():
    import oracle
    from paper_1407_7486_gb300.inputs import PROFILE_CONST_B
    # constant field: every nested level is a genuine N'-point loop, so its
    # average is the exact finite-N' product; the bias is ~ b^2 / (2 N') at
    # O(b^2), so the parabola through N, N/2, N/4 recovers the continuum
    # b / sinh b far better than the finest level
    N, n_loops, G, b = 32, 25600, 32, 1.0
    y = oracle.gen_loops(71, n_loops, N)
    L = ost.nested_level_sums(oracle, y, Profile(PROFILE_CONST_B, B=b), [0.0], [1.0], G)
    lpg = n_loops // G
    for lv, n in enumerate((N, N // 2, N // 4)):
        m, e = ost.mean_sem(L, lpg, 2 * lv)
        assert abs(1.0 + m[0] - _exact_const(b, n)) < 5 * e[0], (n, m[0], e[0])
    E = ost.extrapolate(L)
    m_inf, e_inf = ost.mean_sem(E, lpg, 0)
    m_N, _ = ost.mean_sem(L, lpg, 0)
    cont = b / math.sinh(b) - 1.0
    assert abs(m_inf[0] - cont) < 5 * e_inf[0]
    assert abs(m_inf[0] - cont) < 0.2 * abs(m_N[0] - cont)
    # the exact finite-N values themselves extrapolate to the continuum
    ex = [_exact_const(b, n) for n in (N, N // 2, N // 4)]
    assert abs(np.dot(ost.EXTRAPOLATION, ex) - (1.0 + cont)) < 0.02 * abs(ex[0] - (1.0 + cont))


def test_paper_levels_are_not_a_discretisation_hierarchy():
    # the printed combination e^{i(circ/2 + sq/4 + tri/4)} is a point-weighted
    # mean of sub-loop phases, not the N-point loop: the N-point polygon's
    # area is not (1/2) A_circ + (1/4)(A_sq + A_tri)
    import oracle
    y = oracle.gen_loops(3, 1, 64)[0]

    def area(p):
        return 0.5 * np.sum(p[0] * np.roll(p[1], -1) - np.roll(p[0], -1) * p[1])

    A = area(y)
    mix = 0.5 * area(y[:, 0::2]) + 0.25 * (area(y[:, 1::4]) + area(y[:, 3::4]))
    assert abs(A - mix) > 0.05 * abs(A)
