"""The Wilson kernel's float arctangent (atan_unit and atan2_pos in
csrc/wln_wilson.cu): the polynomial coefficients in the source, evaluated in
float32 the way the kernel does, stay within 1.5 float ulps of the
double-precision arctangent over every octant, and they match what
gen_atan_poly.py derives.  The low-angle form (atan2_low, for 0 < y <= x) is
the same quotient and polynomial, so it is covered by the first octant."""
import os
import re
import subprocess
import sys

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_1407_7486_gb300", "csrc")


def _coeffs():
    text = open(os.path.join(SRC, "wln_wilson.cu")).read()
    body = text[text.index("float atan_unit"):text.index("float atan2_pos")]
    q0 = float(re.search(r"float q = ([-0-9.e]+)f;", body).group(1))
    rest = [float(v) for v in re.findall(r"q = fmaf\(q, s, ([-0-9.e]+)f\);", body)]
    return [q0] + rest


def _atan2_pos_f32(y, x, q):
    y = y.astype(np.float32); x = x.astype(np.float32)
    ax = np.abs(x)
    mn, mx = np.minimum(y, ax), np.maximum(y, ax)
    t = (mn * (np.float32(1) / mx)).astype(np.float32)
    s = (t * t).astype(np.float32)
    p = np.full_like(s, np.float32(q[0]))
    for k in q[1:]:
        p = (p * s + np.float32(k)).astype(np.float32)
    r = (t + (t * s).astype(np.float32) * p).astype(np.float32)
    r = np.where(y > ax, np.float32(np.pi / 2) - r, r).astype(np.float32)
    return np.where(x < 0, np.float32(np.pi) - r, r).astype(np.float32)


def test_polynomial_error_bound():
    q = _coeffs()
    assert len(q) == 8
    rng = np.random.default_rng(0)
    ang = rng.uniform(1e-6, np.pi - 1e-6, 400000)
    rad = 10.0 ** rng.uniform(-8, 8, ang.size)
    y, x = (rad * np.sin(ang)).astype(np.float32), (rad * np.cos(ang)).astype(np.float32)
    got = _atan2_pos_f32(y, x, q).astype(np.float64)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    # the reciprocal in the kernel is an approximation good to 1 ulp: allow 1.5 + 1
    assert np.max(np.abs(got - ref) / ulp) < 2.5


def test_coefficients_come_from_the_generator():
    out = subprocess.run([sys.executable, os.path.join(SRC, "gen_atan_poly.py"), "7"],
                         capture_output=True, text=True, check=True).stdout
    gen = [float(v.strip().rstrip("f")) for v in out.strip().splitlines()[-1].split(",")]
    assert np.allclose(gen, _coeffs(), rtol=1e-6, atol=0)
