"""Ensemble-level pins in a constant magnetic field (Sec. "Renormalization";
Sec. "Estimating the Statistical Uncertainties").

For Gaussian closed loops of N points the Wilson loop average in a constant
field is known exactly at finite N.  With b = eBT, the shoelace area is a
quadratic form of two independent discrete Brownian bridges; diagonalising it
in the Fourier basis gives
    <W_scal>_N = prod_{k=1}^{N-1} (1 + (b cot(pi k/N)/N)^2)^(-1/2),
    <W_ferm>_N = cosh(b) <W_scal>_N,
whose N -> infinity limits are the paper's b/sinh(b) and b coth(b).  The flux
b * area through a loop follows f(Phi) = pi/(4 b cosh^2(pi Phi/(2 b))) in the
continuum (Sec. "Uncertainties and the Fermion Problem").  The oracle's
ensemble means, with their group standard errors, are compared with these.
"""
import math

import numpy as np
import pytest
from scipy import stats as sst

import oracle
from oracle import stats as ost
from paper_1407_7486_gb300.inputs import Profile, PROFILE_CONST_B


def exact_scalar_finite_N(b, N):
    k = np.arange(1, N)
    return float(np.prod((1.0 + (b / (N * np.tan(np.pi * k / N))) ** 2) ** -0.5))


def test_finite_N_product_tends_to_continuum():
    # The discretisation bias is first order in 1/N, of relative size ~ b^2/(2N).
    for b in (0.3, 1.0, 3.0):
        cont = b / math.sinh(b)
        e1 = exact_scalar_finite_N(b, 1 << 14) - cont
        e2 = exact_scalar_finite_N(b, 1 << 15) - cont
        assert 0 < e2 < e1 < b * b / (1 << 14) * cont
        assert e1 / e2 == pytest.approx(2.0, rel=1e-3)


@pytest.mark.parametrize("b,N", [(0.5, 64), (2.0, 64), (6.0, 256)])
def test_constant_field_ensemble_matches_exact(b, N):
    n_loops, G = 16000, 32
    y = oracle.gen_loops(1, n_loops, N)
    S = oracle.group_sums(y, Profile(PROFILE_CONST_B, B=b), [0.0], [1.0], G)
    lpg = n_loops // G
    m_s, e_s = ost.mean_sem(S, lpg, 0)
    m_f, e_f = ost.mean_sem(S, lpg, 1)
    ex = exact_scalar_finite_N(b, N)
    assert abs(1.0 + m_s[0] - ex) < 5 * e_s[0]
    assert abs(1.0 + m_f[0] - math.cosh(b) * ex) < 5 * e_f[0]
    # the imaginary part averages to zero
    m_i, e_i = ost.mean_sem(S, lpg, 2)
    assert abs(m_i[0]) < 5 * e_i[0]


def test_spinor_average_matches_b_coth_b_within_jackknife_error():
    # At large N the discretisation bias ~ b^2/(2N) is far below the error bar.
    n_loops, G, N = 8192, 32, 1024
    y = oracle.gen_loops(2, n_loops, N)
    Ts = np.array([0.25, 0.5, 1.0, 2.0])
    S = oracle.group_sums(y, Profile(PROFILE_CONST_B, B=1.0), [0.0], Ts, G)
    m, e = ost.mean_sem(S, n_loops // G, 1)
    for i, b in enumerate(Ts):
        assert abs(1.0 + m[i] - b / math.tanh(b)) < 5 * e[i]


def test_flux_distribution_of_constant_field_loops():
    # 5120 loops, as in the paper's histograms (Fig. hists caption).
    N, b = 1024, 2.0
    y = oracle.gen_loops(3, 5120, N)
    ph, _ = oracle.phase_spin(y, Profile(PROFILE_CONST_B, B=b), 0.0, 1.0)
    cdf = lambda x: 0.5 * (1.0 + np.tanh(np.pi * x / (2.0 * b)))
    assert sst.kstest(ph, cdf).pvalue > 1e-4


def test_group_means_reproduce_loop_mean_and_sems_agree():
    # Sec. "Grouping Worldlines": equal groups leave the mean unchanged.  For
    # independent loops the per-loop standard error and the group standard
    # error estimate the same quantity, so their ratio is 1 within the
    # sampling error of the group estimate (about 1/sqrt(2(G-1))).
    n_loops, G, N, b = 6400, 64, 128, 6.0
    y = oracle.gen_loops(4, n_loops, N)
    ph, spn = oracle.phase_spin(y, Profile(PROFILE_CONST_B, B=b), 0.0, 1.0)
    S = oracle.group_sums(y, Profile(PROFILE_CONST_B, B=b), [0.0], [1.0], G)
    w = np.cos(ph) - 1.0
    m, e = ost.mean_sem(S, n_loops // G, 0)
    assert m[0] == pytest.approx(w.mean(), rel=1e-12, abs=1e-15)
    loop_sem = ost.loop_sem(S, n_loops, 0, 3)[0]
    assert loop_sem == pytest.approx(w.std(ddof=1) / math.sqrt(n_loops), rel=1e-9)
    assert abs(e[0] / loop_sem - 1.0) < 5 / math.sqrt(2 * (G - 1))


def test_groups_are_contiguous_ranges_of_loops():
    # Sec. "Grouping Worldlines": group i holds loops i N_l/N_G .. (i+1) N_l/N_G - 1.
    n_loops, G, N = 96, 6, 32
    y = oracle.gen_loops(8, n_loops, N)
    prof = Profile(0, F=10.0, lam=1.0)
    rho, T = [0.0, 0.7], [0.3, 2.0]
    S = oracle.group_sums(y, prof, rho, T, G)
    lpg = n_loops // G
    for b, t in enumerate(T):
        for a, r in enumerate(rho):
            ph, spn = oracle.phase_spin(y, prof, r, t)
            w = np.array([oracle.wilson_terms(p, s) for p, s in zip(ph, spn)])
            for g in range(G):
                want = w[g * lpg:(g + 1) * lpg].sum(axis=0)
                assert np.allclose(S[b * len(rho) + a, g], want, rtol=1e-13, atol=1e-15)
