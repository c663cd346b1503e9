"""Writes oracle_small_case.txt: the oracle's group sums for one small fixed
case, as a regression fixture of the oracle itself (a later change to the
oracle's arithmetic shows up as a mismatch and must name the passage that
justifies it).  Calls only oracle/.

    python tests/golden/make_oracle_small_case.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

SEED, N_LOOPS, PPL, G = 1, 64, 64, 4
PROFILE = {"kind": 0, "F": 10.0, "lam": 1.0, "B": 0.0}
RHO = [0.0, 0.5, 2.0]
T = [0.05, 1.0, 5.0]


class _P:
    def __init__(self, d):
        self.kind, self.F, self.lam, self.B = d["kind"], d["F"], d["lam"], d["B"]


def loops():
    """The ensemble, rounded to float32 as the GPU stores it."""
    return oracle.gen_loops(SEED, N_LOOPS, PPL).astype(np.float32).astype(np.float64)


def compute():
    return oracle.group_sums(loops(), _P(PROFILE), RHO, T, G)


if __name__ == "__main__":
    S = compute()
    with open(os.path.join(HERE, "oracle_small_case.txt"), "w") as f:
        f.write("# oracle.group_sums: seed 1, 64 loops x 64 points rounded to float32, flux tube\n")
        f.write("# F = 10, lambda = 1,\n")
        f.write("# rho in {0, 0.5, 2}, T in {0.05, 1, 5} (point p = iT * 3 + i_rho), 4 groups;\n")
        f.write("# columns: point group sum(W_scal-1) sum(W_ferm-1) sum(sin) sum(W_scal-1)^2 sum(W_ferm-1)^2\n")
        f.write("# written by tests/golden/make_oracle_small_case.py (Sec. \"Wilson Loop\", Eqs. rhoi-Ci,\n")
        f.write("# Eq. Wfermfpl; Sec. \"Grouping Worldlines\")\n")
        for p in range(S.shape[0]):
            for g in range(S.shape[1]):
                f.write(f"{p} {g} " + " ".join(f"{v:.17g}" for v in S[p, g]) + "\n")
