"""The cheaper forms of theta (wln_set_low_angle).

Where every segment of a 32-loop block subtends a small angle at the field
axis, the float walks skip the arctangent's range fold and octant unfolding
(level 1) and, below tan(theta) = 0.05, take three terms of its series
(level 2, the default).  On the grids below the smallest proper times
certainly qualify for both (u = sqrt(T) |d|max / lambda ~ 0.01 for 512-point
loops, |d|max ~ 0.3) and T = 50 at the axis certainly does not (u ~ 2), so
a pass mixes the forms.
  * Level 1 gives the same angle bit for bit: every mode and float precision
    equals the general form (level 0) exactly.
  * Level 2 moves the angle by float rounding only: group sums and per-loop
    values stay within the per-loop rounding bars of the parity tests.
"""
import numpy as np
import pytest

import oracle
from paper_1407_7486_gb300 import inputs as I
from paper_1407_7486_gb300 import wln
from test_gpu_parity import F32_REL, _bars, _compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

N_LOOPS, PPL, G = 333, 512, 9       # ragged last block


@pytest.fixture(scope="module")
def setup():
    from paper_1407_7486_gb300 import build
    build.build()
    c = wln.Context(0)
    y32 = oracle.gen_loops(12, N_LOOPS, PPL).astype(np.float32)
    ens = c.ensemble_from_host(y32)
    yield c, y32, ens
    ens.free()
    c.close()


PROFS = [I.Profile(0, F=10.0, lam=1.0), I.Profile(0, F=50.0, lam=0.3), I.Profile(1, B=2.0)]
RHOS = [I.lin_grid(0.0, 8.0, 23), I.lin_grid(0.0, 3.0, 9), np.zeros(1)]
TS = [I.log_grid(1e-3, 50.0, 13), I.log_grid(1e-3, 20.0, 7), I.log_grid(0.01, 5.0, 4)]


def _run(ctx, ens, mode, prec, level, profs=PROFS, rhos=RHOS, Ts=TS):
    ctx.set_low_angle(level)
    try:
        if mode == "sums":
            return ctx.wilson_avg(ens, profs, rhos, Ts, G, prec=prec, where="host")
        if mode in ("levels", "nested"):
            return ctx.wilson_levels(ens, profs, rhos, Ts, G, prec=prec, where="host",
                                     nested=mode == "nested")
        return ctx.wilson_loops(ens, profs, rhos, Ts, prec=prec, where="host")
    finally:
        ctx.set_low_angle(2)


@pytest.mark.parametrize("prec", ["fp32", "fp32_naive"])
@pytest.mark.parametrize("mode", ["sums", "levels", "nested", "loops"])
def test_level1_is_bitwise_neutral(setup, prec, mode):
    ctx, _, ens = setup
    a = _run(ctx, ens, mode, prec, 1)
    b = _run(ctx, ens, mode, prec, 0)
    assert np.isfinite(a).any()
    assert np.array_equal(a, b, equal_nan=True)


@pytest.mark.parametrize("mode", ["sums", "loops"])
def test_level2_within_rounding_bars(setup, mode):
    ctx, y32, ens = setup
    prof, rho, T = PROFS[0], RHOS[0], TS[0]
    a = _run(ctx, ens, mode, "fp32", 2, [prof], [rho], [T])
    b = _run(ctx, ens, mode, "fp32", 0, [prof], [rho], [T])
    if mode == "sums":
        _compare(a, b, N_LOOPS // G, _bars(y32, prof, rho, T, G, 1e-6, F32_REL), what="level 2")
    else:
        bars = _bars(y32, prof, rho, T, N_LOOPS, 1e-6, F32_REL)      # groups of one loop
        for c in (0, 1):
            assert np.all(np.abs(a[:, :, c] - b[:, :, c]) <= bars[c][0]), c


def test_low_angle_rejects_other_levels(setup):
    ctx, _, _ = setup
    from paper_1407_7486_gb300.wln import load
    assert load().wln_set_low_angle(ctx.handle, 3) != 0
    assert load().wln_set_low_angle(ctx.handle, -1) != 0
    ctx.set_low_angle(2)
