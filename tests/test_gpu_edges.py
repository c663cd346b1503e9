"""Edge cases of the Wilson pass, through the C ABI.

  * A single radius and a single proper time (a tile with one valid radius).
  * A ragged last block (33 loops: one full block of 32 and one loop) with
    groups of 11 loops straddling the block boundary.
  * The smallest loops (ppl = 4) and the largest (ppl = 16384).
  * Extreme but valid parameters against the oracle: tiny and huge proper
    times, a radius far outside the tube, a very thin tube.  For the thin
    tube (lambda = 1e-4) only the scalar parts are held to the bar: segments
    passing within ~lambda of the axis make the spin integral ill-conditioned
    (relative sensitivity |r|/h to the rounding of the points, h the distance
    of closest approach), and as lambda -> 0 the spinor loop meets a
    delta-function field; its spinor sums must still be finite where the
    oracle's are.
  * F -> -F: the phase and the spin change sign exactly, so the sums of
    W_scal - 1, W_ferm - 1 and their squares are bitwise unchanged and the sum
    of sin(phase) is exactly negated.
  * One loop per group: the group sums are the per-loop values of
    wln_wilson_loops, bit for bit (same arithmetic, one addition to zero).
  * Empty inputs (no profile, no radius, no loops) are refused.
"""
import numpy as np
import pytest

import oracle
from paper_1407_7486_gb300 import inputs as I
from paper_1407_7486_gb300 import wln
from test_gpu_parity import F32_REL, F64_REL, _bars, _compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def ctx():
    from paper_1407_7486_gb300 import build
    build.build()
    c = wln.Context(0)
    yield c
    c.close()


def _ens(ctx, seed, n_loops, ppl):
    y = oracle.gen_loops(seed, n_loops, ppl).astype(np.float32)
    return y, ctx.ensemble_from_host(y)


EDGE = [
    # (n_loops, ppl, G, profile, rho, T)
    (64, 128, 4, I.Profile(0, F=10.0, lam=1.0), np.array([0.7]), np.array([0.9])),
    (33, 64, 3, I.Profile(0, F=10.0, lam=1.0), I.lin_grid(0.0, 3.0, 5), I.log_grid(0.05, 5.0, 3)),
    (96, 4, 4, I.Profile(0, F=10.0, lam=1.0), I.lin_grid(0.0, 3.0, 6), I.log_grid(0.05, 5.0, 3)),
    (64, 128, 4, I.Profile(0, F=10.0, lam=1.0), np.array([0.0, 0.5]), np.array([1e-6, 50.0])),
    (64, 128, 4, I.Profile(0, F=10.0, lam=1.0), np.array([1e4]), np.array([0.1, 10.0])),
    (64, 256, 4, I.Profile(0, F=1.0, lam=1e-4), I.lin_grid(0.0, 1.0, 3), np.array([0.5, 2.0])),  # scalar
    (32, 16384, 2, I.Profile(0, F=50.0, lam=1.0), np.array([0.0, 2.0]), np.array([0.01, 1.0])),
]


@pytest.mark.parametrize("case", range(len(EDGE)))
@pytest.mark.parametrize("prec,tol,rel", [("fp64", 1e-12, F64_REL), ("fp32", 1e-6, F32_REL)])
def test_edge_cases_match_oracle(ctx, case, prec, tol, rel):
    n_loops, ppl, G, prof, rho, T = EDGE[case]
    y32, ens = _ens(ctx, 71 + case, n_loops, ppl)
    gpu = ctx.wilson_avg(ens, [prof], [rho], [T], G, prec=prec, where="host")
    ref = oracle.group_sums(y32.astype(np.float64), prof, rho, T, G)
    bars = _bars(y32, prof, rho, T, G, tol, rel)
    if prof.kind == 0 and prof.lam < 1e-3:
        assert np.array_equal(np.isfinite(gpu), np.isfinite(ref))
        lpg = n_loops // G
        for c in (0, 2, 3):                            # scalar parts only
            d = np.abs(gpu[:, :, c] - ref[:, :, c]) / lpg
            assert np.all(d <= bars[c][0]), (prec, c, float((d / bars[c][0]).max()))
    else:
        _compare(gpu, ref, n_loops // G, bars, what=f"{prec} edge {case}")
    ens.free()


@pytest.mark.parametrize("prec", ["fp32", "fp64", "fp32_naive"])
@pytest.mark.parametrize("mode", ["sums", "levels", "loops"])
def test_flux_reversal_is_exact(ctx, prec, mode):
    # spins up to ~320 (F = 50, T = 20 on the axis): cosh beyond float range
    _, ens = _ens(ctx, 8, 96, 256)
    rho, T = I.lin_grid(0.0, 4.0, 7), I.log_grid(0.01, 20.0, 5)
    pos = [I.Profile(0, F=50.0, lam=1.0), I.Profile(1, B=3.0)]
    neg = [I.Profile(0, F=-50.0, lam=1.0), I.Profile(1, B=-3.0)]
    if mode == "sums":
        call = lambda p: ctx.wilson_avg(ens, p, [rho, rho], [T, T], 4, prec=prec, where="host")
    elif mode == "levels":
        call = lambda p: ctx.wilson_levels(ens, p, [rho, rho], [T, T], 4, prec=prec, where="host")
    else:
        call = lambda p: ctx.wilson_loops(ens, p, [rho, rho], [T, T], prec=prec, where="host")
    a, b = call(pos), call(neg)
    assert not np.any(np.isnan(a)) and not np.any(np.isnan(b))
    if mode == "sums":
        for c in (0, 1, 3, 4):
            assert np.array_equal(a[:, :, c], b[:, :, c]), c
        assert np.array_equal(a[:, :, 2], -b[:, :, 2])
    else:
        assert np.array_equal(a, b)
    ens.free()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_one_loop_per_group_equals_loop_values(ctx, prec):
    n_loops = 64
    _, ens = _ens(ctx, 9, n_loops, 128)
    prof, rho, T = I.Profile(0, F=10.0, lam=1.0), I.lin_grid(0.0, 3.0, 6), I.log_grid(0.05, 5, 4)
    S = ctx.wilson_avg(ens, [prof], [rho], [T], n_loops, prec=prec, where="host")
    W = ctx.wilson_loops(ens, [prof], [rho], [T], prec=prec, where="host")
    assert np.array_equal(S[:, :, 0], W[:, :, 0]) and np.array_equal(S[:, :, 1], W[:, :, 1])
    ens.free()


def test_empty_inputs_are_refused(ctx):
    _, ens = _ens(ctx, 10, 32, 64)
    prof = I.Profile(0, F=1.0, lam=1.0)
    with pytest.raises(wln.WlnError):
        ctx.wilson_avg(ens, [], [], [], 2)                              # no profile
    with pytest.raises(wln.WlnError):
        ctx.wilson_avg(ens, [prof], [np.zeros(0)], [np.ones(1)], 2)     # no radius
    with pytest.raises(wln.WlnError):
        ctx.wilson_avg(ens, [prof], [np.zeros(1)], [np.zeros(0)], 2)    # no proper time
    with pytest.raises(wln.WlnError):
        ctx.gen_loops(1, 0, 64)                                         # no loops
    ens.free()
