"""Pins of the oracle's statistics and quadrature.

  * Grouped jackknife (Sec. "Grouping Worldlines"): brute-force delete-one
    group means on small G; the delete-one variance equals the squared group
    standard error for a mean (an algebraic identity); the covariance
    diagonal is that square; group means reproduce the loop mean.
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
