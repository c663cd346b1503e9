"""Generate the float-pair constants of the double-float (float-float) walk.

    python paper_1407_7486_gb300/csrc/gen_ff_consts.py

Every constant c is written as hi + lo with hi the float nearest to c and lo
the float nearest to c - hi, from 50-digit values (mpmath): the arctangents
atan(j/16), j = 0..16, of the table-driven arctangent, and pi, pi/2, 1/3.
Prints C++ initialisers in the form used by csrc/wln_guard.cu; a CPU test
re-derives them and compares bit patterns.
"""
import mpmath
import numpy as np

mpmath.mp.dps = 50


def nearest_f32(x) -> np.float32:
    """The float32 nearest to the mpmath number x (ties to even)."""
    c = np.float32(float(x))
    best = c
    for cand in (np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))):
        d, db = abs(mpmath.mpf(float(cand)) - x), abs(mpmath.mpf(float(best)) - x)
        if d < db or (d == db and int(cand.view(np.uint32)) % 2 == 0):
            best = cand
    return best


def split(x):
    hi = nearest_f32(x)
    lo = nearest_f32(x - mpmath.mpf(float(hi)))
    return hi, lo


def constants():
    table = [split(mpmath.atan(mpmath.mpf(j) / 16)) for j in range(17)]
    named = {"PI": split(mpmath.pi), "PI_2": split(mpmath.pi / 2), "THIRD": split(mpmath.mpf(1) / 3)}
    return table, named


def _lit(v: np.float32) -> str:
    return f"{float(v):.9e}f" if v != 0 else "0.0f"


if __name__ == "__main__":
    table, named = constants()
    print("// atan(j/16), j = 0..16, as (hi, lo)")
    for j, (h, l) in enumerate(table):
        print(f"    {{{_lit(h)}, {_lit(l)}}},   // j = {j}")
    for k, (h, l) in named.items():
        print(f"constexpr float k{k}_HI = {_lit(h)}, k{k}_LO = {_lit(l)};")
