"""The bound behind the Wilson kernel's low-angle forms, checked on the CPU.

For a segment from r to r + d and Q(t) = lambda^2 + |r + t d|^2, the angle
theta = atan2(sqrt(D), Q0 + B) (B = r.d, D = lambda^2 |d|^2 + (r x d)^2)
obeys tan(theta) <= u / (1 - u) with u = |d| / sqrt(Q0): sqrt(D) <=
sqrt(Q0) |d| (Lagrange) and Q0 + B >= Q0 - sqrt(Q0) |d|.  The kernel takes the
low form (no octant unfolding) for 2u <= 0.9, the five-term series for
2u <= 0.3 and the three-term series for 2u <= 0.09, with u bounded per block
through |d| <= sqrt(T) |d|max and Q0 >= lambda^2 + (rho - sqrt(T) |y|max)_+^2.
Checked here:
  * the bound itself, by brute force over random and adversarial segments
    (short and long, near and across the axis, thin and wide tubes);
  * that the three thresholds give theta <= pi/4, tan(theta) < 0.18 and
    tan(theta) < 0.05;
  * the remainders of the series 1 - t^2/3 + t^4/5 (below t^6/7) and
    1 - t^2/3 + t^4/5 - t^6/7 + t^8/9 (below t^10/11) of atan(t)/t;
  * the three-term form's spin integral int dt/Q^2 = 1/(Q0 Q1) +
    C r^3 (1/3 - 2 t^2/5), against the closed form and a quadrature;
  * the per-block reading of u on a real ensemble against every segment's u;
  * the bench's accounting of the forms at the extremes (all or nothing).
"""
import numpy as np
import pytest

import oracle
from paper_1407_7486_gb300 import inputs as I


def _theta_u(r, d, lam):
    B = np.sum(r * d, axis=-1)
    X = r[..., 0] * d[..., 1] - r[..., 1] * d[..., 0]
    C = np.sum(d * d, axis=-1)
    D = lam * lam * C + X * X
    Q0 = lam * lam + np.sum(r * r, axis=-1)
    theta = np.arctan2(np.sqrt(D), Q0 + B)
    u = np.sqrt(C / Q0)
    return theta, u


def test_tan_theta_bound_brute_force():
    rng = np.random.default_rng(5)
    n = 400000
    for lam in (1e-3, 0.1, 1.0, 10.0):
        r = rng.normal(size=(n, 2)) * 10.0 ** rng.uniform(-3, 1, size=(n, 1))
        d = rng.normal(size=(n, 2)) * 10.0 ** rng.uniform(-4, 1, size=(n, 1))
        # adversarial: segments pointing straight at the axis
        d[: n // 4] = -r[: n // 4] * rng.uniform(0.0, 0.9, size=(n // 4, 1))
        theta, u = _theta_u(r, d, lam)
        ok = u < 1.0
        assert np.all(np.tan(theta[ok]) <= u[ok] / (1.0 - u[ok]) * (1 + 1e-12) + 1e-300)


def test_thresholds_give_the_forms():
    rng = np.random.default_rng(6)
    n = 400000
    r = rng.normal(size=(n, 2)) * 10.0 ** rng.uniform(-2, 1, size=(n, 1))
    d = rng.normal(size=(n, 2))
    d *= (10.0 ** rng.uniform(-3, 0, size=(n, 1))) / np.linalg.norm(d, axis=1, keepdims=True)
    theta, u = _theta_u(r, d, 0.7)
    low, mid, short = 2 * u <= 0.9, 2 * u <= 0.3, 2 * u <= 0.09
    assert low.any() and mid.any() and short.any() and (~low).any()
    assert np.all(theta[low] <= np.pi / 4)
    assert np.all(np.tan(theta[mid]) < 0.18)
    assert np.all(np.tan(theta[short]) < 0.05)


def test_series_remainder():
    t = np.linspace(1e-6, 0.05, 20001)
    series = 1.0 - t * t / 3.0 + t ** 4 / 5.0
    # an alternating series: the remainder is below the first omitted term
    # (plus the double rounding of both sides, a few ulps of 1)
    assert np.all(np.abs(np.arctan(t) / t - series) <= t ** 6 / 7.0 + 1e-15)
    assert (0.05 ** 6) / 7.0 < 2.3e-9
    t = np.linspace(1e-6, 0.18, 20001)
    s2 = t * t
    series5 = 1.0 - s2 / 3.0 + s2 ** 2 / 5.0 - s2 ** 3 / 7.0 + s2 ** 4 / 9.0
    assert np.all(np.abs(np.arctan(t) / t - series5) <= t ** 10 / 11.0 + 1e-15)
    assert (0.18 ** 10) / 11.0 < 3.3e-9


def test_block_bound_covers_every_segment():
    y = oracle.gen_loops(3, 96, 256)                       # 3 blocks of 32 loops
    d = np.roll(y, -1, axis=2) - y
    seg = np.sqrt(np.sum(d * d, axis=1))                   # [loop][segment]
    rad = np.sqrt(np.sum(y * y, axis=1))
    lam = 0.5
    for T in (1e-3, 0.3, 4.0):
        for rho in (0.0, 1.0, 6.0):
            for b in range(3):
                sl = slice(32 * b, 32 * b + 32)
                dm, rm = seg[sl].max(), rad[sl].max()
                gap = max(0.0, rho - np.sqrt(T) * rm)
                u_block = np.sqrt(T) * dm / np.sqrt(lam * lam + gap * gap)
                r = np.stack([rho + np.sqrt(T) * y[sl, 0], np.sqrt(T) * y[sl, 1]], axis=-1)
                dd = np.sqrt(T) * np.stack([d[sl, 0], d[sl, 1]], axis=-1)
                _, u = _theta_u(r, dd, lam)
                assert np.all(u <= u_block * (1 + 1e-12))


def test_sub_block_bound_covers_every_segment():
    """The per-chunk form takes a sub-block's statistics: the longest segment
    starting in its 64 rows (128 points; the last one ends at the next
    sub-block's first point) and the largest |y| of those points and that
    next point.  Every segment a chunk walks stays within that bound."""
    y = oracle.gen_loops(5, 64, 512)                       # 2 blocks, 4 sub-blocks each
    d = np.roll(y, -1, axis=2) - y                         # segment k: point k -> k + 1
    seg = np.sqrt(np.sum(d * d, axis=1))
    rad = np.sqrt(np.sum(y * y, axis=1))
    rad_end = np.maximum(rad, np.roll(rad, -1, axis=1))
    lam = 0.7
    for T in (1e-3, 0.5, 6.0):
        for rho in (0.0, 2.0, 9.0):
            for b in range(2):
                lo = slice(32 * b, 32 * b + 32)
                for c in range(4):
                    ks = slice(128 * c, 128 * c + 128)
                    dm, rm = seg[lo, ks].max(), rad_end[lo, ks].max()
                    gap = max(0.0, rho - np.sqrt(T) * rm)
                    u_sub = np.sqrt(T) * dm / np.sqrt(lam * lam + gap * gap)
                    r = np.stack([rho + np.sqrt(T) * y[lo, 0, ks], np.sqrt(T) * y[lo, 1, ks]], axis=-1)
                    dd = np.sqrt(T) * np.stack([d[lo, 0, ks], d[lo, 1, ks]], axis=-1)
                    _, u = _theta_u(r, dd, lam)
                    assert np.all(u <= u_sub * (1 + 1e-12))


def test_sub_block_accounting():
    """Per-chunk forms only improve on the block's, never reach the
    three-term form the block does not take, and change nothing where a
    block is a single sub-block."""
    import bench
    prof = I.Profile(I.PROFILE_FLUX_TUBE, F=10.0, lam=1.0)
    rho = I.lin_grid(0.0, 4.0, 9)
    T = I.log_grid(0.01, 10.0, 7)
    y32 = oracle.gen_loops(6, 96, 1024).astype(np.float32)
    blk = bench.low_angle_fraction(y32, [prof], [rho], [T], 4, 1.0)
    sub = bench.low_angle_fraction(y32, [prof], [rho], [T], 4, 1.0, sub_rows=64)
    assert sub[0] >= blk[0] and sub[1] >= blk[1] and sub[1] > blk[1]
    assert sub[2] == blk[2]
    y32 = oracle.gen_loops(6, 96, 128).astype(np.float32)
    assert (bench.low_angle_fraction(y32, [prof], [rho], [T], 4, 1.0, sub_rows=64) ==
            bench.low_angle_fraction(y32, [prof], [rho], [T], 4, 1.0))


def test_accounting_extremes():
    import bench
    y32 = oracle.gen_loops(4, 64, 128).astype(np.float32)
    prof = I.Profile(I.PROFILE_FLUX_TUBE, F=10.0, lam=1.0)
    rho = I.lin_grid(0.0, 3.0, 7)
    low, mid, short = bench.low_angle_fraction(y32, [prof], [rho], [np.array([1e-8])], 4, 1.0)
    assert low == 1.0 and mid == 1.0 and short == 1.0
    low, mid, short = bench.low_angle_fraction(y32, [prof], [np.zeros(1)], [np.array([1e4])], 4, 1.0)
    assert low == 0.0 and mid == 0.0 and short == 0.0
    const = I.Profile(I.PROFILE_CONST_B, B=1.0)
    assert bench.low_angle_fraction(y32, [const], [np.zeros(1)], [np.ones(1)], 4, 1.0) == (0.0, 0.0, 0.0)
    # the operation count: 6 fewer on the low form, 13 on the five-term series,
    # 6 + 9 + 2 - 2/P on the three-term one (its spin series, C/3 and 2C/5
    # shared by P radii)
    base = bench.N_ALG_FP32
    assert base == 16 + 17 + 11 / 4 + 1
    assert bench._n_alg(base, (1.0, 1.0, 1.0)) == base - 16.5
    assert bench._n_alg(base, (1.0, 1.0, 0.0)) == base - 13
    assert bench._n_alg(base, (1.0, 0.0, 0.0)) == base - 6
    assert bench._n_alg(base, (1.0, 1.0, 1.0), P=2) == pytest.approx(base - 16)


@pytest.mark.parametrize("u_max,terms,bound", [(0.045, 3, 2.3e-9), (0.15, 5, 3.3e-9)])
def test_series_forms_of_int_dt_over_q(u_max, terms, bound):
    """The kernel's series forms: int_0^1 dt/Q = theta / sqrt(D) =
    r atan(t)/t, r = 1/(Q0 + B), t^2 = D r^2, from three terms of the series
    on segments with 2u <= 0.09 and five on segments with 2u <= 0.3 -- checked
    against the closed form and against a 400-point Gauss-Legendre rule of
    the integral itself."""
    rng = np.random.default_rng(8)
    n = 20000
    lam = 0.8
    r = rng.normal(size=(n, 2)) * 3.0
    d = rng.normal(size=(n, 2))
    Q0 = lam * lam + np.sum(r * r, axis=1)
    d *= (u_max * np.sqrt(Q0) * rng.uniform(0.01, 1.0, size=n) / np.linalg.norm(d, axis=1))[:, None]
    theta, u = _theta_u(r, d, lam)
    assert np.all(u <= u_max * (1 + 1e-12))
    B = np.sum(r * d, axis=1)
    X = r[:, 0] * d[:, 1] - r[:, 1] * d[:, 0]
    D = lam * lam * np.sum(d * d, axis=1) + X * X
    rr = 1.0 / (Q0 + B)
    t2 = D * rr * rr
    coef = [1.0, -1.0 / 3.0, 1.0 / 5.0, -1.0 / 7.0, 1.0 / 9.0][:terms]
    series = rr * sum(c * t2 ** k for k, c in enumerate(coef))
    closed = theta / np.sqrt(D)
    assert np.all(np.abs(series - closed) <= bound * closed + 1e-15 * closed)
    x, w = np.polynomial.legendre.leggauss(400)
    tq = 0.5 * (x + 1.0)
    Q = lam * lam + np.sum((r[:, None, :] + tq[None, :, None] * d[:, None, :]) ** 2, axis=2)
    quad = 0.5 * np.sum(w[None, :] / Q, axis=1)
    assert np.all(np.abs(series - quad) <= bound * quad + 1e-14 * quad)


def test_series_form_of_int_dt_over_q2():
    """The three-term form's spin integral: int_0^1 dt/Q^2 = -d/d(lambda^2)
    int_0^1 dt/Q.  Shifting lambda^2 by e moves Q0 + B by e and D by C e, so
    with int dt/Q = r f(t^2), f(u) = atan(sqrt u)/sqrt u, it is
    r^2 [f - (C r - 2 t^2) f'] = 1/(Q0 Q1) + C r^3 h(t^2), h = -f' =
    1/3 - 2u/5 + 3u^2/7 - ...  (r^2/(1 + t^2) = 1/(Q0 Q1)).  Two terms of h,
    on segments with 2u <= 0.09, against the closed form
    [(C + B)/Q1 - B/Q0 + C int dt/Q] / (2D) and a 400-point Gauss-Legendre
    rule of the integral; the remainder bound is 3.6e-9 relative."""
    rng = np.random.default_rng(9)
    n = 20000
    for lam in (0.1, 0.8, 3.0):
        r = rng.normal(size=(n, 2)) * 3.0
        d = rng.normal(size=(n, 2))
        Q0 = lam * lam + np.sum(r * r, axis=1)
        d *= (0.045 * np.sqrt(Q0) * rng.uniform(0.3, 1.0, size=n) /
              np.linalg.norm(d, axis=1))[:, None]
        theta, u = _theta_u(r, d, lam)
        B = np.sum(r * d, axis=1)
        C = np.sum(d * d, axis=1)
        X = r[:, 0] * d[:, 1] - r[:, 1] * d[:, 0]
        D = lam * lam * C + X * X
        Q1 = Q0 + 2 * B + C
        rr = 1.0 / (Q0 + B)
        t2 = D * rr * rr
        series = 1.0 / (Q0 * Q1) + C * rr ** 3 * (1.0 / 3.0 - 0.4 * t2)
        x, w = np.polynomial.legendre.leggauss(400)
        tq = 0.5 * (x + 1.0)
        Q = lam * lam + np.sum((r[:, None, :] + tq[None, :, None] * d[:, None, :]) ** 2, axis=2)
        quad = 0.5 * np.sum(w[None, :] / Q ** 2, axis=1)
        assert np.all(np.abs(series - quad) <= 3.6e-9 * quad + 1e-14 * quad)
        # the closed form, where it keeps its digits (it cancels for short segments)
        closed = ((C + B) / Q1 - B / Q0 + C * theta / np.sqrt(D)) / (2 * D)
        ok = C / Q0 > 1e-4
        assert ok.sum() > n // 4
        assert np.all(np.abs(series - closed)[ok] <= 1e-8 * closed[ok])
