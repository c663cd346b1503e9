"""Pins of the oracle's unit-loop generator (Sec. "Loop Generation").

What the paper fixes and what is checked here:
  * Box-Muller output is standard normal (moments, Kolmogorov-Smirnov).
  * Loops are closed and have zero centre of mass (d-loop step 5).
  * The d-loop construction (Eqs. yn2, ynk): with N_k points, a new midpoint
    is Gaussian about the mean of its two neighbours with variance 1/N_k per
    component, independent of them.  The increment construction used here
    must give the same joint law, so at the finest level the midpoint
    residual has variance 1/N and is uncorrelated with the neighbours; the
    N = 2 loop has separation variance 1/2 (Eq. yn2).
  * Every other point forms an N/2 loop with the N/2 statistics (Sec.
    "Estimating the Discretization Uncertainties").
  * Closed-form moments of the discrete Brownian bridge: increment variance
    (2/N)(1 - 1/N), point variance (N^2 - 1)/(6 N^2), area variance
    (N - 1)(N - 2)/(3 N^2).
Statistical checks use 5-sigma bounds on fixed seeds.
"""
import math

import numpy as np
import pytest
from scipy import stats as sst

import oracle

# Both generators must give the law of the discretised closed loop: the
# increment construction of the hot path and the paper's d-loop (Eqs. yn2, ynk).
GENERATORS = {"increments": oracle.gen_loops, "dloop": oracle.gen_dloops}


def _z_from_raw(seed, n_loops, ppl):
    xi = np.stack([oracle.raw_increments(seed, l, ppl) for l in range(n_loops)])
    return xi / math.sqrt(2.0 / ppl)


def test_box_muller_is_standard_normal():
    z = _z_from_raw(11, 400, 256).ravel()          # 204800 samples
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(sst.kurtosis(z, fisher=False) - 3.0) < 5 * math.sqrt(24.0 / n)
    assert sst.kstest(z, "norm").pvalue > 1e-4
    # x and y components independent
    zz = _z_from_raw(12, 200, 256)
    r = np.corrcoef(zz[:, 0, :].ravel(), zz[:, 1, :].ravel())[0, 1]
    assert abs(r) < 5 / math.sqrt(zz[:, 0, :].size)


@pytest.mark.parametrize("gen", list(GENERATORS))
@pytest.mark.parametrize("ppl", [4, 64, 1024])
def test_loops_closed_and_centred(ppl, gen):
    y = GENERATORS[gen](3, 50, ppl)
    d = np.roll(y, -1, axis=2) - y
    assert np.abs(d.sum(axis=2)).max() < 1e-13
    assert np.abs(y.sum(axis=2)).max() < 1e-15 * ppl * 10


@pytest.mark.parametrize("gen", list(GENERATORS))
def test_two_point_loop_variance(gen):
    # Eq. yn2: with N_1 = 2 the separation has weight exp(-(2/4) 2 dy^2), variance 1/2.
    y = GENERATORS[gen](5, 40000, 2)
    sep = y[:, :, 1] - y[:, :, 0]
    n = sep.size
    assert abs(sep.var() - 0.5) < 5 * 0.5 * math.sqrt(2.0 / n)
    assert np.allclose(y[:, :, 0], -y[:, :, 1])


@pytest.mark.parametrize("gen", list(GENERATORS))
@pytest.mark.parametrize("ppl", [16, 128])
def test_midpoint_law_matches_dloop(ppl, gen):
    # Eq. ynk at the finest level: y_{2m+1} ~ N((y_{2m} + y_{2m+2})/2, 1/N).
    y = GENERATORS[gen](9, 8000, ppl)
    even = y[:, :, 0::2]
    odd = y[:, :, 1::2]
    nxt = np.roll(even, -1, axis=2)
    resid = odd - 0.5 * (even + nxt)
    n = resid.size
    assert abs(resid.var() - 1.0 / ppl) < 5 * (1.0 / ppl) * math.sqrt(2.0 / n)
    # The residual is unchanged by the centre-of-mass shift (its weights sum to
    # zero), so it must be independent of the coarse loop's shape and of the
    # other residuals, as the d-loop draws each midpoint afresh.
    c1 = np.corrcoef(resid.ravel(), (nxt - even).ravel())[0, 1]
    c2 = np.corrcoef(resid.ravel(), np.roll(nxt - even, 1, axis=2).ravel())[0, 1]
    c3 = np.corrcoef(resid.ravel(), np.roll(resid, 1, axis=2).ravel())[0, 1]
    for c in (c1, c2, c3):
        assert abs(c) < 5 / math.sqrt(n)


def _area(y):
    x, yy = y[:, 0, :], y[:, 1, :]
    return 0.5 * (x * np.roll(yy, -1, axis=1) - yy * np.roll(x, -1, axis=1)).sum(axis=1)


@pytest.mark.parametrize("gen", list(GENERATORS))
@pytest.mark.parametrize("ppl", [8, 64, 256])
def test_bridge_moments(ppl, gen):
    N = ppl
    n_loops = 20000 if ppl <= 64 else 6000
    y = GENERATORS[gen](21, n_loops, ppl)
    d = np.roll(y, -1, axis=2) - y
    v_d = (2.0 / N) * (1.0 - 1.0 / N)
    nd = d.size
    assert abs(d.var() - v_d) < 6 * v_d * math.sqrt(2.0 / nd) * 2
    v_y = (N * N - 1) / (6.0 * N * N)
    # one coordinate per loop keeps the samples independent
    s = y[:, :, 0].ravel()
    assert abs(s.var() - v_y) < 5 * v_y * math.sqrt(2.0 / s.size)
    a = _area(y)
    v_a = (N - 1) * (N - 2) / (3.0 * N * N)
    if N > 2:
        # area = sum of products: kurtosis ~ 6 (logistic tail), so 5 sigma with that
        assert abs(a.var() - v_a) < 5 * v_a * math.sqrt((6.0 + 2.0) / a.size)
    assert abs(a.mean()) < 5 * math.sqrt(v_a / a.size)


@pytest.mark.parametrize("gen", list(GENERATORS))
def test_every_other_point_is_half_loop(gen):
    N, M = 128, 64
    y = GENERATORS[gen](31, 10000, N)[:, :, 0::2]
    d = np.roll(y, -1, axis=2) - y
    v_d = (2.0 / M) * (1.0 - 1.0 / M)
    assert abs(d.var() - v_d) < 10 * v_d * math.sqrt(2.0 / d.size)
    a = _area(y - y.mean(axis=2, keepdims=True))
    v_a = (M - 1) * (M - 2) / (3.0 * M * M)
    assert abs(a.var() - v_a) < 5 * v_a * math.sqrt(8.0 / a.size)


def test_loops_are_counter_based():
    a = oracle.gen_loops(77, 10, 32, loop0=100)
    b = oracle.gen_loops(77, 3, 32, loop0=105)
    assert np.array_equal(a[5:8], b)
    c = oracle.gen_loops(78, 3, 32, loop0=105)
    assert not np.allclose(b, c)


def test_dloop_coarse_levels_follow_eq_ynk():
    # Level k of the d-loop: the points q N/N_k (q odd) about their level-(k-1)
    # neighbours, residual variance 1/N_k per component.
    N = 64
    y = oracle.gen_dloops(41, 8000, N)
    for Nk in (4, 8, 16):
        st = N // Nk
        mid = y[:, :, st::2 * st]
        nb = y[:, :, 0::2 * st]
        resid = mid - 0.5 * (nb + np.roll(nb, -1, axis=2))
        v = resid.var()
        assert abs(v - 1.0 / Nk) < 5 * (1.0 / Nk) * math.sqrt(2.0 / resid.size)


def test_generators_give_the_same_area_law():
    # two-sample KS of the loop areas of the two constructions
    a = _area(oracle.gen_loops(51, 6000, 128))
    b = _area(oracle.gen_dloops(52, 6000, 128))
    assert sst.ks_2samp(a, b).pvalue > 1e-3
