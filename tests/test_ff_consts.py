"""The float-pair constants of the precision guard's double-float walk
(csrc/wln_guard.cu): atan(j/16), j = 0..16, pi, pi/2 and 1/3 as hi + lo.

Each is re-derived at 50 digits (mpmath) by csrc/gen_ff_consts.py and
compared bit for bit with the literal in the source; hi + lo must carry the
value to within 2^-48 of it (a double-float number's precision), and hi must
be the float nearest to the value.
"""
import os
import re
import sys

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1407_7486_gb300", "csrc")
sys.path.insert(0, CSRC)
import gen_ff_consts  # noqa: E402


def _source_constants():
    text = open(os.path.join(CSRC, "wln_guard.cu")).read()
    body = text[text.index("kAtanTable[17] = {"):]
    body = body[:body.index("};")]
    table = [(np.float32(a), np.float32(b))
             for a, b in re.findall(r"\{([-0-9.e+]+)f, ([-0-9.e+]+)f\}", body)]
    named = {}
    for name in ("PI", "PI_2", "THIRD"):
        m = re.search(rf"k{name}_HI = ([-0-9.e+]+)f, k{name}_LO = ([-0-9.e+]+)f", text)
        named[name] = (np.float32(m.group(1)), np.float32(m.group(2)))
    return table, named


def test_constants_match_their_derivation_bit_for_bit():
    table, named = _source_constants()
    want_table, want_named = gen_ff_consts.constants()
    assert len(table) == 17
    for (h, l), (wh, wl) in zip(table, want_table):
        assert h.view(np.uint32) == wh.view(np.uint32) and l.view(np.uint32) == wl.view(np.uint32)
    for k, (h, l) in named.items():
        wh, wl = want_named[k]
        assert h.view(np.uint32) == wh.view(np.uint32) and l.view(np.uint32) == wl.view(np.uint32)


def test_pairs_carry_the_values():
    mpmath.mp.dps = 50
    table, named = _source_constants()
    exact = [mpmath.atan(mpmath.mpf(j) / 16) for j in range(17)]
    exact_named = {"PI": mpmath.pi, "PI_2": mpmath.pi / 2, "THIRD": mpmath.mpf(1) / 3}
    pairs = list(zip(table, exact)) + [(named[k], exact_named[k]) for k in named]
    for (h, l), x in pairs:
        got = mpmath.mpf(float(h)) + mpmath.mpf(float(l))
        assert abs(got - x) <= abs(x) * mpmath.mpf(2) ** -48
        # hi is the float nearest to x
        for nb in (np.nextafter(h, np.float32(-np.inf)), np.nextafter(h, np.float32(np.inf))):
            assert abs(mpmath.mpf(float(h)) - x) <= abs(mpmath.mpf(float(nb)) - x)
