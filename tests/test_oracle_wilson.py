"""Pins of the oracle's per-loop Wilson phase and spin factor.

The oracle integrates A.dr and B along each straight segment in closed form
(Sec. "Wilson Loop", Eqs. rhoi-Ci; Sec. "Fermion Part", Eq. Wfermfpl).  The
checks below reach the same numbers by other routes:
  * Gauss-Legendre quadrature of A.dr, with A built from the paper's
    A_phi = F f(rho)/(2 pi rho), and of B obtained by differentiating A_phi
    symbolically through Eq. BWLN (B = A_phi/rho + dA_phi/drho);
  * the lambda -> 0 limit, where the phase is calF times the winding angle
    of the polygon about the axis (an independent angle sum);
  * a hand-integrated square centred on the axis;
  * the constant field, where the phase is B times the polygon area and the
    spin integral is B T;
  * exact symmetries (reflection, reversal, cyclic relabelling, rotation
    about the axis) and the zero-field case W = 1 exactly.
"""
import math

import numpy as np
import pytest
import sympy as sp

import oracle
from paper_1407_7486_gb300.inputs import Profile, PROFILE_CONST_B, PROFILE_FLUX_TUBE


def _field_functions(F, lam):
    r = sp.symbols("r", positive=True)
    f = r**2 / (lam**2 + r**2)                       # Sec. Verification and Validation
    A_phi = F * f / (2 * sp.pi * r)                  # Sec. Cylindrical Magnetic Fields
    B = sp.simplify(A_phi / r + sp.diff(A_phi, r))   # Eq. BWLN
    return sp.lambdify(r, A_phi, "numpy"), sp.lambdify(r, B, "numpy")


def _gl_phase_spin(y, F, lam, rho_cm, T, n_gl=200):
    A_phi, Bf = _field_functions(F, lam)
    t, w = np.polynomial.legendre.leggauss(n_gl)
    t = 0.5 * (t + 1.0); w = 0.5 * w
    N = y.shape[1]
    r = np.stack([rho_cm + math.sqrt(T) * y[0], math.sqrt(T) * y[1]])
    d = np.roll(r, -1, axis=1) - r
    ph = sp_ = 0.0
    for k in range(N):
        pts = r[:, k:k + 1] + d[:, k:k + 1] * t[None, :]
        rr = np.hypot(pts[0], pts[1])
        # A = A_phi * phi_hat, phi_hat = (-y, x)/rho
        Ax = -A_phi(rr) * pts[1] / rr
        Ay = A_phi(rr) * pts[0] / rr
        ph += np.sum(w * (Ax * d[0, k] + Ay * d[1, k]))
        sp_ += (T / N) * np.sum(w * Bf(rr))
    return ph, sp_


@pytest.mark.parametrize("case", [
    dict(N=8, F=10.0, lam=1.0, rho=0.0, T=1.0),
    dict(N=16, F=3.0, lam=0.7, rho=0.5, T=2.0),
    dict(N=32, F=50.0, lam=1.5, rho=2.0, T=5.0),
    dict(N=64, F=1.0, lam=1.0, rho=8.0, T=0.1),
    dict(N=16, F=100.0, lam=0.5, rho=1.0, T=0.5),
])
def test_closed_forms_match_gauss_legendre(case):
    y = oracle.gen_loops(101, 3, case["N"])
    prof = Profile(PROFILE_FLUX_TUBE, F=case["F"], lam=case["lam"])
    for l in range(3):
        ph, spn = oracle.loop_phase_spin(y[l], prof, case["rho"], case["T"])
        ph_gl, sp_gl = _gl_phase_spin(y[l], case["F"], case["lam"], case["rho"], case["T"])
        assert ph == pytest.approx(ph_gl, rel=1e-10, abs=1e-12)
        assert spn == pytest.approx(sp_gl, rel=1e-10, abs=1e-14)


def _winding_angle(y, rho_cm, T):
    r = np.stack([rho_cm + math.sqrt(T) * y[0], math.sqrt(T) * y[1]])
    rn = np.roll(r, -1, axis=1)
    return np.arctan2(r[0] * rn[1] - r[1] * rn[0], r[0] * rn[0] + r[1] * rn[1]).sum()


def test_thin_tube_phase_is_flux_times_winding():
    # lambda -> 0: int_0^1 dt/(lambda^2 + rho^2) * X -> subtended angle of the
    # segment; the correction is of order lambda^2 / (closest approach)^2.
    F, lam = 7.0, 1e-9
    y = oracle.gen_loops(202, 40, 64)
    windings = []
    for l in range(40):
        for rho_cm in (0.0, 0.3):
            r = np.stack([rho_cm + y[l][0], y[l][1]])
            d = np.roll(r, -1, axis=1) - r
            t = np.clip(-(r * d).sum(0) / (d * d).sum(0), 0.0, 1.0)
            closest = np.hypot(*(r + d * t)).min()
            if closest < 1e-4:
                continue
            ph, _ = oracle.loop_phase_spin(y[l], Profile(PROFILE_FLUX_TUBE, F=F, lam=lam), rho_cm, 1.0)
            ang = _winding_angle(y[l], rho_cm, 1.0)
            assert ph == pytest.approx(F / (2 * math.pi) * ang, abs=1e-9)
            windings.append(round(ang / (2 * math.pi)))
    assert 0 in windings and any(w != 0 for w in windings)


def test_square_on_axis_by_hand():
    # Square of side a centred on the axis, counter-clockwise, N = 4, T = 1.
    a, lam, F = 0.7, 0.4, 3.0
    calF = F / (2 * math.pi)
    y = np.array([[a / 2, a / 2, -a / 2, -a / 2], [-a / 2, a / 2, a / 2, -a / 2]])
    ph, spn = oracle.loop_phase_spin(y, Profile(PROFILE_FLUX_TUBE, F=F, lam=lam), 0.0, 1.0)
    h = math.sqrt(lam**2 + a**2 / 4)
    assert ph == pytest.approx(4 * calF * (a / h) * math.atan(a / (2 * h)), rel=1e-13)
    # each side: (1/a) int_{-a/2}^{a/2} du/(h^2+u^2)^2
    J2 = ((a / 2) / (h**2 * (h**2 + a**2 / 4)) + math.atan(a / (2 * h)) / h**3) / a
    assert spn == pytest.approx((1.0 / 4) * 2 * calF * lam**2 * 4 * J2, rel=1e-13)
    # thin-tube limit: 2 pi calF
    ph0, _ = oracle.loop_phase_spin(y, Profile(PROFILE_FLUX_TUBE, F=F, lam=1e-9), 0.0, 1.0)
    assert ph0 == pytest.approx(2 * math.pi * calF, rel=1e-9)
    # square of side a off the axis in a constant field: phase = B a^2
    phc, spc = oracle.loop_phase_spin(y, Profile(PROFILE_CONST_B, B=0.8), 4.0, 1.0)
    assert phc == pytest.approx(0.8 * a * a, rel=1e-13)
    assert spc == 0.8 * 1.0


@pytest.mark.parametrize("rho_cm", [0.0, 2.5])
def test_constant_field_phase_is_B_times_area(rho_cm):
    y = oracle.gen_loops(303, 20, 128)
    T, B = 1.7, 0.9
    for l in range(20):
        x = rho_cm + math.sqrt(T) * y[l][0]
        yy = math.sqrt(T) * y[l][1]
        # trapezoid form of Green's theorem, area = sum (x_k + x_{k+1})/2 (y_{k+1} - y_k)
        area = np.sum(0.5 * (x + np.roll(x, -1)) * (np.roll(yy, -1) - yy))
        ph, spn = oracle.loop_phase_spin(y[l], Profile(PROFILE_CONST_B, B=B), rho_cm, T)
        assert ph == pytest.approx(B * area, rel=1e-11, abs=1e-13)
        assert spn == pytest.approx(B * T, rel=1e-15)


def test_wide_tube_is_constant_field_near_axis():
    lam, F = 40.0, 5.0
    B0 = 2 * (F / (2 * math.pi)) / lam**2           # eB(0) = 2 calF f'(0)
    y = oracle.gen_loops(404, 10, 64)
    for l in range(10):
        ph, spn = oracle.loop_phase_spin(y[l], Profile(PROFILE_FLUX_TUBE, F=F, lam=lam), 0.0, 0.5)
        phc, spc = oracle.loop_phase_spin(y[l], Profile(PROFILE_CONST_B, B=B0), 0.0, 0.5)
        assert ph == pytest.approx(phc, rel=2e-3)
        assert spn == pytest.approx(spc, rel=2e-3)


def test_zero_flux_gives_unit_wilson_loop_exactly():
    y = oracle.gen_loops(505, 5, 32)
    for l in range(5):
        ph, spn = oracle.loop_phase_spin(y[l], Profile(PROFILE_FLUX_TUBE, F=0.0, lam=1.0), 1.3, 2.0)
        assert ph == 0.0 and spn == 0.0
        assert np.all(oracle.wilson_terms(ph, spn) == 0.0)


def test_wilson_terms_identities():
    for ph, spn in [(0.3, 0.0), (2.0, 1.5), (-7.0, 30.0), (1e-5, 1e-4)]:
        w = oracle.wilson_terms(ph, spn)
        assert w[0] == pytest.approx(math.cos(ph) - 1.0, rel=1e-12, abs=1e-16)
        assert w[1] == pytest.approx(math.cos(ph) * math.cosh(spn) - 1.0, rel=1e-12, abs=1e-16)
        assert w[2] == pytest.approx(math.sin(ph))
        assert w[3] == pytest.approx(w[0] ** 2) and w[4] == pytest.approx(w[1] ** 2)


def _rot(y, a):
    c, s = math.cos(a), math.sin(a)
    return np.stack([c * y[0] - s * y[1], s * y[0] + c * y[1]])


def test_symmetries():
    prof = Profile(PROFILE_FLUX_TUBE, F=10.0, lam=1.0)
    y = oracle.gen_loops(606, 6, 32)
    for l in range(6):
        L = y[l]
        ph, spn = oracle.loop_phase_spin(L, prof, 0.8, 1.5)
        # reflection about the x axis (x_cm stays on it): phase flips, spin stays
        ph_r, sp_r = oracle.loop_phase_spin(np.stack([L[0], -L[1]]), prof, 0.8, 1.5)
        assert ph_r == pytest.approx(-ph, rel=1e-12, abs=1e-14)
        assert sp_r == pytest.approx(spn, rel=1e-12)
        # orientation reversal
        ph_v, sp_v = oracle.loop_phase_spin(L[:, ::-1].copy(), prof, 0.8, 1.5)
        assert ph_v == pytest.approx(-ph, rel=1e-12, abs=1e-14)
        assert sp_v == pytest.approx(spn, rel=1e-12)
        # cyclic relabelling of the starting point
        ph_c, sp_c = oracle.loop_phase_spin(np.roll(L, 5, axis=1).copy(), prof, 0.8, 1.5)
        assert ph_c == pytest.approx(ph, rel=1e-12, abs=1e-14)
        assert sp_c == pytest.approx(spn, rel=1e-12)
        # rotating loop and centre of mass together about the field axis
        a = 0.37 + l
        Tq = 1.5
        shifted = _rot(L, a) + (_rot(np.array([[0.8], [0.0]]), a) / math.sqrt(Tq))
        ph_q, sp_q = oracle.loop_phase_spin(shifted, prof, 0.0, Tq)
        assert ph_q == pytest.approx(ph, rel=1e-11, abs=1e-13)
        assert sp_q == pytest.approx(spn, rel=1e-11)


def test_repeated_point_still_accumulates_spin():
    # A loop that rests at one point for one step: the phase is unchanged,
    # the spin integral gains eB(rho^2) T/N for that step (Eq. Wfermfpl).
    F, lam, T = 6.0, 0.8, 1.3
    calF = F / (2 * math.pi)
    base = oracle.gen_loops(707, 1, 8)[0]
    rep = np.concatenate([base[:, :3], base[:, 2:3], base[:, 3:]], axis=1)   # point 2 twice, N = 9
    prof = Profile(PROFILE_FLUX_TUBE, F=F, lam=lam)
    ph9, sp9 = oracle.loop_phase_spin(rep, prof, 0.4, T)
    ph8, sp8 = oracle.loop_phase_spin(base, prof, 0.4, T)
    assert ph9 == pytest.approx(ph8, rel=1e-13)
    r2 = (0.4 + math.sqrt(T) * base[0, 2]) ** 2 + (math.sqrt(T) * base[1, 2]) ** 2
    eB = 2 * calF * lam**2 / (lam**2 + r2) ** 2
    assert sp9 == pytest.approx(sp8 * 8 / 9 + eB * T / 9, rel=1e-12)


def test_phase_abs_sum_of_segment_magnitudes():
    # phase_abs is the sum over segments of |segment phase| (it sizes the
    # rounding bars of the float path)
    rng = np.random.default_rng(17)
    F = 2 * math.pi * 3.0                      # calF = 3
    # thin tube: each segment's phase is calF times the angle it subtends at the axis
    prof = Profile(PROFILE_FLUX_TUBE, F=F, lam=1e-9)
    for _ in range(5):
        y = oracle.gen_loops(int(rng.integers(1 << 30)), 1, 64)[0]
        rho, T = 0.3, 0.5
        r = np.stack([rho + math.sqrt(T) * y[0], math.sqrt(T) * y[1]])
        if np.min(np.hypot(r[0], r[1])) < 1e-3:
            continue
        ang = np.arctan2(r[1], r[0])
        d = np.diff(np.append(ang, ang[0]))
        d = (d + math.pi) % (2 * math.pi) - math.pi
        want = 3.0 * np.abs(d).sum()
        assert oracle.phase_abs(y[None], prof, rho, T)[0] == pytest.approx(want, rel=1e-7)
    # |phase| <= phase_abs, equal for a convex polygon around the axis, and
    # linear in the flux
    prof = Profile(PROFILE_FLUX_TUBE, F=F, lam=0.7)
    k = np.arange(12)
    poly = np.stack([0.8 * np.cos(2 * np.pi * k / 12), 0.5 * np.sin(2 * np.pi * k / 12)])[None]
    ph, _ = oracle.phase_spin(poly, prof, 0.0, 1.0)
    assert oracle.phase_abs(poly, prof, 0.0, 1.0)[0] == pytest.approx(abs(ph[0]), rel=1e-13)
    y = oracle.gen_loops(5, 40, 128)
    ph, _ = oracle.phase_spin(y, prof, 0.4, 2.0)
    pa = oracle.phase_abs(y, prof, 0.4, 2.0)
    assert np.all(pa >= np.abs(ph) * (1 - 1e-13)) and np.any(pa > 1.5 * np.abs(ph))
    pa2 = oracle.phase_abs(y, Profile(PROFILE_FLUX_TUBE, F=2 * F, lam=0.7), 0.4, 2.0)
    np.testing.assert_allclose(pa2, 2 * pa, rtol=1e-13)
