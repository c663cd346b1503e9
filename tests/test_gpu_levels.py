"""GPU parity of the discretisation levels (Sec. "Estimating the Discretization
Uncertainties") against the FP64 oracle, through the C ABI.

  * wln_wilson_levels: group means of W - 1 at the levels N, N/2, N/4 against
    oracle.stats.level_sums on the same float points.  Per-loop bars as for
    the plain pass: a level's phase and spin are fixed combinations (weights
    1, 1/2, 1/4) of the three sub-loops' phases and spins, so its bar takes
    the same combination of the sub-loops' sums of |segment phase| and spins:
      E_scal = max(tol, rel P_L),  E_ferm = max(1, cosh s_L) max(tol, rel (s_L + P_L)),
    rel = 2^-21 (FP32) or 2^-50 (FP64), tol = 1e-6 or 1e-12.
  * wln_extrapolate on identical level sums: 1e-12 relative against the
    oracle's extrapolation and group statistics.
  * Degenerate cases: zero flux gives exactly 0 at every level; ppl below 8
    or not a multiple of 4 is refused.
"""
import numpy as np
import pytest

import oracle
from oracle import stats as ost
from paper_1407_7486_gb300 import inputs as I
from paper_1407_7486_gb300 import wln

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

F32_REL = 2.0 ** -21
F64_REL = 2.0 ** -50


@pytest.fixture(scope="module")
def ctx():
    from paper_1407_7486_gb300 import build
    build.build()
    c = wln.Context(0)
    yield c
    c.close()


def _ensemble(ctx, seed, n_loops, ppl):
    y = oracle.gen_loops(seed, n_loops, ppl).astype(np.float32)
    return y, ctx.ensemble_from_host(y)


def _level_bars(y32, profile, rho, T, G, tol, rel):
    """Group and ensemble bars [n_points][G], [n_points] per level component."""
    y = y32.astype(np.float64)
    subs = [np.ascontiguousarray(y[:, :, 0::2]), np.ascontiguousarray(y[:, :, 1::4]),
            np.ascontiguousarray(y[:, :, 3::4])]
    lpg = y.shape[0] // G
    n = len(T) * len(rho)
    out = {c: (np.zeros((n, G)), np.zeros(n)) for c in range(6)}
    weights = [(0.5, 0.25, 0.25), (1.0, 0.0, 0.0), (0.0, 0.5, 0.5)]
    for b, t in enumerate(T):
        for a, r in enumerate(rho):
            ps = [oracle.phase_spin(s, profile, r, t) for s in subs]
            pa = [oracle.phase_abs(s, profile, r, t) for s in subs]
            p = b * len(rho) + a
            for L, wts in enumerate(weights):
                P = sum(w * x for w, x in zip(wts, pa))
                s = sum(w * x[1] for w, x in zip(wts, ps))
                with np.errstate(over="ignore", invalid="ignore"):
                    es = np.maximum(tol, rel * P)
                    ef = np.maximum(1.0, np.cosh(s)) * np.maximum(tol, rel * (np.abs(s) + P))
                for c, e in ((2 * L, es), (2 * L + 1, ef)):
                    out[c][0][p] = e.reshape(G, lpg).mean(axis=1)
                    out[c][1][p] = e.mean()
    return out


def _compare(gpu, ref, lpg, bars, what):
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(gpu)), f"{what}: non-finite entries differ"
    worst = {}
    with np.errstate(over="ignore", invalid="ignore"):
        dg = np.where(fin, gpu - ref, 0.0) / lpg
        de = np.abs(dg.mean(axis=1))
        for comp in range(6):
            bg, be = bars[comp]
            we = np.nan_to_num(de[:, comp] / be).max()
            wg = np.nan_to_num(np.abs(dg[:, :, comp]) / bg).max()
            worst[comp] = (round(float(we), 3), round(float(wg), 3))
            assert we <= 1.0, f"{what} comp {comp}: ensemble mean {we:.3g} x bar"
            assert wg <= 1.0, f"{what} comp {comp}: group mean {wg:.3g} x bar"
    print(what, worst)


LEVEL_CASES = [
    # (n_loops, ppl, G, profile, rho, T): several tiles (2 radii per lane,
    # 8 warps per CTA), ragged tails in radii and loops
    (96, 64, 3, I.Profile(0, F=10.0, lam=1.0), I.lin_grid(0.0, 5.0, 7), I.log_grid(0.01, 10.0, 5)),
    (72, 256, 8, I.Profile(0, F=100.0, lam=0.1), I.lin_grid(0.0, 5.0, 5), I.log_grid(0.01, 10.0, 3)),
    (64, 1024, 2, I.Profile(0, F=1.0, lam=1.0), I.lin_grid(0.0, 8.0, 3), I.log_grid(1e-3, 20.0, 6)),
    (64, 64, 4, I.Profile(1, B=1.0), np.array([0.0, 1.5]), I.log_grid(0.01, 10.0, 6)),
    (40, 8, 5, I.Profile(0, F=10.0, lam=0.5), I.lin_grid(0.0, 2.0, 6), I.log_grid(0.1, 4.0, 3)),
    (33, 16, 3, I.Profile(0, F=50.0, lam=1.0), I.lin_grid(0.0, 3.0, 3), I.log_grid(0.1, 4.0, 2)),
]


@pytest.mark.parametrize("case", range(len(LEVEL_CASES)))
@pytest.mark.parametrize("prec,tol,rel", [("fp64", 1e-12, F64_REL), ("fp32", 1e-6, F32_REL)])
def test_levels_match_oracle(ctx, case, prec, tol, rel):
    n_loops, ppl, G, prof, rho, T = LEVEL_CASES[case]
    y32, ens = _ensemble(ctx, 41 + case, n_loops, ppl)
    gpu = ctx.wilson_levels(ens, [prof], [rho], [T], G, prec=prec, where="host")
    ref = ost.level_sums(oracle, y32.astype(np.float64), prof, rho, T, G)
    _compare(gpu, ref, n_loops // G, _level_bars(y32, prof, rho, T, G, tol, rel),
             f"{prec} level case {case}")
    ens.free()


def test_levels_batch_of_profiles_and_device_output(ctx):
    y32, ens = _ensemble(ctx, 9, 128, 128)
    profs = [I.Profile(0, F=10.0, lam=1.0), I.Profile(1, B=2.0), I.Profile(0, F=1.0, lam=0.3)]
    rhos = [I.lin_grid(0, 4, 5), np.zeros(1), I.lin_grid(0, 2, 9)]
    Ts = [I.log_grid(0.01, 5, 4), I.log_grid(0.1, 2, 3), I.log_grid(0.05, 1, 2)]
    both = ctx.wilson_levels(ens, profs, rhos, Ts, 4, where="host")
    dev = ctx.wilson_levels(ens, profs, rhos, Ts, 4, where="device")
    assert np.array_equal(both, dev.cpu().numpy())
    p0 = 0
    for q in range(3):
        alone = ctx.wilson_levels(ens, [profs[q]], [rhos[q]], [Ts[q]], 4, where="host")
        n = len(rhos[q]) * len(Ts[q])
        assert np.array_equal(alone, both[p0:p0 + n])     # a point's sums do not depend on the batch
        p0 += n
    ens.free()


def test_levels_zero_flux_and_rules(ctx):
    _, ens = _ensemble(ctx, 5, 64, 64)
    for prec in ("fp64", "fp32", "fp32_naive"):
        S = ctx.wilson_levels(ens, [I.Profile(0, F=0.0, lam=1.0)], [I.lin_grid(0, 3, 5)],
                              [I.log_grid(0.1, 4, 3)], 4, prec=prec, where="host")
        assert np.all(S == 0.0), prec
    ens.free()
    _, small = _ensemble(ctx, 5, 32, 4)
    with pytest.raises(wln.WlnError):
        ctx.wilson_levels(small, [I.Profile(0, F=1.0, lam=1.0)], [np.zeros(1)], [np.ones(1)], 2)
    small.free()


def test_extrapolation_matches_oracle(ctx):
    n_loops, ppl, G = 256, 128, 8
    y32, ens = _ensemble(ctx, 77, n_loops, ppl)
    prof, rho, T = I.Profile(0, F=10.0, lam=1.0), I.lin_grid(0, 4, 6), I.log_grid(0.05, 8, 5)
    S = ctx.wilson_levels(ens, [prof], [rho], [T], G, prec="fp64", where="host")
    lpg = n_loops // G
    got = ctx.extrapolate(S, G, lpg, where="host")
    got_dev = ctx.extrapolate(torch.from_numpy(S).cuda(), G, lpg, where="device").cpu().numpy()
    assert np.array_equal(got, got_dev)
    E = ost.extrapolate(S)                      # [n_points][G][2] sums of W_inf - 1
    for x in range(2):
        for j, comp in enumerate((x, 2 + x, 4 + x)):
            m, _ = ost.mean_sem(S, lpg, comp)
            np.testing.assert_allclose(got[:, x, j], m, rtol=1e-12, atol=1e-15)
        m_inf, sem_inf = ost.mean_sem(E, lpg, x)
        np.testing.assert_allclose(got[:, x, 3], m_inf, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(got[:, x, 4], sem_inf, rtol=1e-10, atol=1e-15)
        np.testing.assert_allclose(got[:, x, 5], np.abs(got[:, x, 0] - m_inf), rtol=1e-10,
                                   atol=1e-15)
    ens.free()


def _nested_bars(y32, profile, rho, T, G, tol, rel):
    """Per-level bars for the nested levels: each level is a genuine loop
    (all, even, 0 mod 4 points), with its own sums of |segment phase| and spin."""
    y = y32.astype(np.float64)
    subs = [y, np.ascontiguousarray(y[:, :, 0::2]), np.ascontiguousarray(y[:, :, 0::4])]
    lpg = y.shape[0] // G
    n = len(T) * len(rho)
    out = {c: (np.zeros((n, G)), np.zeros(n)) for c in range(6)}
    for b, t in enumerate(T):
        for a, r in enumerate(rho):
            p = b * len(rho) + a
            for L, sub in enumerate(subs):
                _, s = oracle.phase_spin(sub, profile, r, t)
                P = oracle.phase_abs(sub, profile, r, t)
                with np.errstate(over="ignore", invalid="ignore"):
                    es = np.maximum(tol, rel * P)
                    ef = np.maximum(1.0, np.cosh(s)) * np.maximum(tol, rel * (np.abs(s) + P))
                for c, e in ((2 * L, es), (2 * L + 1, ef)):
                    out[c][0][p] = e.reshape(G, lpg).mean(axis=1)
                    out[c][1][p] = e.mean()
    return out


@pytest.mark.parametrize("case", range(len(LEVEL_CASES)))
@pytest.mark.parametrize("prec,tol,rel", [("fp64", 1e-12, F64_REL), ("fp32", 1e-6, F32_REL)])
def test_nested_levels_match_oracle(ctx, case, prec, tol, rel):
    n_loops, ppl, G, prof, rho, T = LEVEL_CASES[case]
    y32, ens = _ensemble(ctx, 141 + case, n_loops, ppl)
    gpu = ctx.wilson_levels(ens, [prof], [rho], [T], G, prec=prec, where="host", nested=True)
    ref = ost.nested_level_sums(oracle, y32.astype(np.float64), prof, rho, T, G)
    _compare(gpu, ref, n_loops // G, _nested_bars(y32, prof, rho, T, G, tol, rel),
             f"{prec} nested level case {case}")
    ens.free()


def test_nested_extrapolation_recovers_the_continuum(ctx):
    # constant field: the nested levels' parabola lands on b/sinh b and b coth b
    # within its group error, far closer than the finest level; the paper's
    # printed combination moves away from it (its levels are no hierarchy)
    import math
    n_loops, N, G, B = 32768, 32, 32, 1.0
    ens = ctx.gen_loops(3, n_loops, N)
    prof, rho, T = I.Profile(1, B=B), [np.zeros(1)], [np.array([1.0])]
    lpg = n_loops // G
    cont = [B / math.sinh(B) - 1.0, B / math.tanh(B) - 1.0]
    for nested in (True, False):
        L = ctx.wilson_levels(ens, [prof], rho, T, G, prec="fp64", where="host", nested=nested)
        X = ctx.extrapolate(L, G, lpg, where="host")[0]
        for x in (0, 1):
            m_N, m_inf, sem_inf = X[x, 0], X[x, 3], X[x, 4]
            if nested:
                assert abs(m_inf - cont[x]) < 5 * sem_inf, (x, m_inf, cont[x], sem_inf)
                assert abs(m_inf - cont[x]) < 0.2 * abs(m_N - cont[x])
            else:
                assert abs(m_inf - cont[x]) > abs(m_N - cont[x])
    ens.free()
