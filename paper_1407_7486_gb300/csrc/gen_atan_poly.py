"""Generate the minimax polynomial used by the Wilson kernel's arctangent.

    python paper_1407_7486_gb300/csrc/gen_atan_poly.py [degree]

atan(t) = t + t^3 Q(t^2) on t in [0, 1]: the leading term is kept exact so
small angles (short, distant segments: most of them) carry only the rounding
of t.  Q of the given degree minimises the maximum relative error of the
arctangent, by the Remez exchange algorithm on the weighted error
w(s) (Q(s) - g(s)), s = t^2, g = (atan(t)/t - 1)/s, w = s t/atan(t).
Prints the coefficients of Q (highest degree first) as float literals and the
error of the float32 evaluation against the double arctangent.
"""
import sys

import numpy as np


def _g(s):
    t = np.sqrt(s)
    return np.where(s > 1e-12, (np.arctan(t) / np.maximum(t, 1e-300) - 1.0) / np.maximum(s, 1e-300),
                    -1.0 / 3.0 + s / 5.0)


def _w(s):
    t = np.sqrt(s)
    return np.where(s > 1e-12, s * t / np.maximum(np.arctan(t), 1e-300), s)


def remez(deg: int, iters: int = 60):
    n = deg + 2
    lo = 1e-4
    x = lo + (1 - lo) * (0.5 - 0.5 * np.cos(np.pi * np.arange(n) / (n - 1)))
    dense = np.concatenate([np.linspace(0.0, 1e-3, 2001), np.linspace(1e-3, 1.0, 400001)])
    best = None
    for _ in range(iters):
        A = np.zeros((n, n))
        for i in range(n):
            A[i, :deg + 1] = x[i] ** np.arange(deg + 1)
            A[i, deg + 1] = (-1) ** i / _w(x[i])
        sol = np.linalg.solve(A, _g(x))
        c = sol[:deg + 1]
        err = _w(dense) * (np.polyval(c[::-1], dense) - _g(dense))
        e = np.abs(err).max()
        if best is None or e < best[1]:
            best = (c.copy(), e)
        idx = np.where(np.diff(np.sign(err)) != 0)[0]
        bounds = np.concatenate([[0], idx + 1, [len(dense)]])
        ext = [b0 + np.argmax(np.abs(err[b0:b1])) for b0, b1 in zip(bounds[:-1], bounds[1:])]
        if len(ext) < n:
            break
        ext = sorted(ext, key=lambda j: -abs(err[j]))[:n]
        x = np.sort(dense[ext])
    return best


def float32_ulps(q_high_first):
    q = np.array(q_high_first, np.float32)
    t = np.linspace(0, 1, 2000001).astype(np.float32)
    s = (t * t).astype(np.float32)
    p = np.full_like(s, q[0])
    for k in q[1:]:
        p = (p * s + k).astype(np.float32)
    r = (t + (t * s).astype(np.float32) * p).astype(np.float32)
    ref = np.arctan(t.astype(np.float64))
    ok = ref > 0
    ulp = np.spacing(ref[ok].astype(np.float32)).astype(np.float64)
    return np.max(np.abs(r[ok] - ref[ok]) / ulp)


if __name__ == "__main__":
    deg = int(sys.argv[1]) if len(sys.argv) > 1 else 7
    c, e = remez(deg)
    q = [float(np.float32(v)) for v in c[::-1]]
    print(f"// degree {deg}: max relative error {e:.3e} (exact arithmetic); "
          f"float32 evaluation within {float32_ulps(q):.2f} ulp")
    print(", ".join(f"{np.float32(v)!r}f".replace("np.float32(", "").replace(")", "") for v in q))
