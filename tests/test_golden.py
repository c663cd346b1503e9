"""Stored values: the numbers the paper prints, and one oracle regression case.

  * tests/golden/paper_printed_values.txt holds the small-T coefficients of
    Eqs. fermI and scalI and the extrapolation weights of Sec. "Estimating
    the Discretization Uncertainties", as printed.  Each is checked twice:
    against the mathematics that fixes it (the Bernoulli series of x coth x
    and x / sinh x times e^{-T}; the parabola in 1/N through N, N/2, N/4
    extrapolated to 1/N = 0), and against the oracle's use of it.
  * tests/golden/oracle_small_case.txt is the oracle's group sums for one
    fixed small case, written by tests/golden/make_oracle_small_case.py: a
    change to the oracle's arithmetic shows up here.
"""
import os
import re
from fractions import Fraction

import numpy as np

from oracle import stats as ost

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _printed():
    """name -> function of x (Fraction in, Fraction out) for every printed line."""
    out = {}
    with open(os.path.join(GOLDEN, "paper_printed_values.txt")) as f:
        for line in f:
            line = line.split("[")[0].strip()
            if not line or line.startswith("#"):
                continue
            name, expr = (s.strip() for s in line.split("=", 1))
            expr = re.sub(r"\d+", lambda m: f"F({m.group()})", expr.replace("^", "**"))
            out[name] = (lambda e: lambda x: eval(e, {"F": Fraction, "x": Fraction(x)}))(expr)
    return out


def _series_of_integrand(spinor, n, x):
    """Coefficient of T^n in e^{-T} / T^3 * bracket(x T), exactly: the bracket
    x coth x - 1 - x^2/3 = sum_k 2^{2k} B_2k x^{2k} / (2k)!, or
    x / sinh x - 1 + x^2/6 = -sum_k (2^{2k} - 2) B_2k x^{2k} / (2k)!, k >= 2."""
    import math
    B = ost._bernoulli_even(6)
    c = Fraction(0)
    for k in range(2, 6):
        j = n - (2 * k - 3)                   # power taken from e^{-T}
        if j < 0:
            continue
        bk = (Fraction(2 ** (2 * k)) if spinor else -Fraction(2 ** (2 * k) - 2)) * B[k]
        bk /= math.factorial(2 * k)
        c += bk * Fraction(x) ** (2 * k) * Fraction((-1) ** j, math.factorial(j))
    return c


def test_printed_small_T_coefficients_follow_from_the_series():
    P = _printed()
    for x in (Fraction(1, 3), Fraction(1), Fraction(5, 2), Fraction(7)):
        for i in range(4):
            assert P[f"ferm_c{i + 1}"](x) == _series_of_integrand(True, i + 1, x), (x, i)
            assert P[f"scal_c{i + 1}"](x) == _series_of_integrand(False, i + 1, x), (x, i)


def test_oracle_small_T_integral_uses_the_printed_coefficients():
    P = _printed()
    for eB in (0.3, 1.0, 2.5):
        for a in (0.01, 0.05, 0.2):
            for spinor, tag in ((True, "ferm"), (False, "scal")):
                want = sum(float(P[f"{tag}_c{i + 1}"](Fraction(eB))) * a ** (i + 2) / (i + 2)
                           for i in range(4))
                got = float(ost.small_T_integral(eB, a, spinor=spinor))
                assert abs(got - want) <= 1e-14 * abs(want), (eB, a, spinor, got, want)


def test_printed_extrapolation_weights():
    P = _printed()
    w = [P[k](0) for k in ("extrap_a", "extrap_b", "extrap_c")]
    # Lagrange weights at h = 0 of the parabola through h, 2h, 4h (h = 1/N)
    nodes = [Fraction(1), Fraction(2), Fraction(4)]
    for i, hi in enumerate(nodes):
        li = Fraction(1)
        for j, hj in enumerate(nodes):
            if j != i:
                li *= (0 - hj) / (hi - hj)
        assert w[i] == li
    assert tuple(float(v) for v in w) == ost.EXTRAPOLATION


def test_oracle_small_case_regression():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_oracle_small_case", os.path.join(GOLDEN, "make_oracle_small_case.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    stored = np.loadtxt(os.path.join(GOLDEN, "oracle_small_case.txt"))
    S = mod.compute()
    n_pts, G = len(mod.RHO) * len(mod.T), mod.G
    assert stored.shape == (n_pts * G, 7)
    want = stored[:, 2:].reshape(n_pts, G, 5)
    assert np.array_equal(stored[:, 0], np.repeat(np.arange(n_pts), G))
    # libm differs between hosts in the last bit: hold to a few ulps of the scale
    scale = np.abs(want).max(axis=(0, 1), keepdims=True) + 1e-300
    assert np.all(np.abs(S - want) <= 1e-13 * scale), float((np.abs(S - want) / scale).max())
