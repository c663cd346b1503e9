"""GPU parity of the per-loop values, the randomised grouping and the
correlation coefficients (Sec. "Correlations between Wilson Loops", Eq.
corrcoef; Sec. "Grouping Worldlines"), through the C ABI.

  * wln_wilson_loops: every loop's W - 1 against oracle.loop_values, element
    by element within the per-loop bar of the plain pass (FP32: max(1e-6,
    2^-21 P) scalar, max(1, cosh s) max(1e-6, 2^-21 (s + P)) spinor; FP64 the
    same with 1e-12 and 2^-50).
  * Contiguous group sums of the per-loop values equal wln_wilson_avg's up to
    summation order (FP64 path).
  * The shuffled order of every point equals the oracle's Fisher-Yates
    permutation bit for bit; shuffled group sums of seeded per-loop values
    equal the oracle's (same addition order: bitwise for the sums).
  * wln_corrcoef against oracle.stats.corrcoef_ref, 1e-12; and Fig. corr as a
    property: loops and fixed groups stay correlated across T, shuffled
    groups do not.
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


@pytest.mark.parametrize("prec,tol,rel", [("fp64", 1e-12, 2.0 ** -50), ("fp32", 1e-6, 2.0 ** -21)])
@pytest.mark.parametrize("case", range(3))
def test_loop_values_match_oracle(ctx, prec, tol, rel, case):
    n_loops, ppl, prof, rho, T = [
        (100, 256, I.Profile(0, F=10.0, lam=1.0), I.lin_grid(0, 4, 6), I.log_grid(0.01, 10, 5)),
        (37, 64, I.Profile(1, B=2.0), np.array([0.0, 1.0]), I.log_grid(0.05, 5, 4)),
        (64, 2048, I.Profile(0, F=50.0, lam=1.0), I.lin_grid(0, 8, 3), I.log_grid(1e-3, 20, 3)),
    ][case]
    y32, ens = _ensemble(ctx, 31 + case, n_loops, ppl)
    y = y32.astype(np.float64)
    got = ctx.wilson_loops(ens, [prof], [rho], [T], prec=prec, where="host")
    want = oracle.loop_values(y, prof, rho, T)
    for b, t in enumerate(T):
        for a, r in enumerate(rho):
            p = b * len(rho) + a
            ph, sp = oracle.phase_spin(y, prof, r, t)
            P = oracle.phase_abs(y, prof, r, t)
            with np.errstate(over="ignore", invalid="ignore"):
                es = np.maximum(tol, rel * P)
                ef = np.maximum(1.0, np.cosh(sp)) * np.maximum(tol, rel * (np.abs(sp) + P))
            fin = np.isfinite(want[p])
            assert np.array_equal(fin, np.isfinite(got[p]))
            d = np.where(fin, np.abs(got[p] - want[p]), 0.0)
            assert np.all(d[:, 0] <= es), (p, float((d[:, 0] / es).max()))
            assert np.all(d[:, 1] <= ef), (p, float((d[:, 1] / ef).max()))
    ens.free()


def test_contiguous_groups_of_loop_values_equal_group_sums(ctx):
    _, ens = _ensemble(ctx, 4, 320, 128)
    prof, rho, T = I.Profile(0, F=10.0, lam=1.0), I.lin_grid(0, 3, 5), I.log_grid(0.05, 5, 4)
    W = ctx.wilson_loops(ens, [prof], [rho], [T], prec="fp64")
    S, perm = ctx.group_sums_loops(W, 8, where="host")
    assert perm is None
    ref = ctx.wilson_avg(ens, [prof], [rho], [T], 8, prec="fp64", where="host")
    for c in (0, 1, 3, 4):
        scale = np.abs(ref[:, :, c]).max() + 1e-300
        assert np.abs(S[:, :, c] - ref[:, :, c]).max() <= 1e-13 * 40 * scale, c
    assert np.all(np.isnan(S[:, :, 2]))
    ens.free()


def test_shuffle_matches_oracle_bit_for_bit(ctx):
    rng = np.random.default_rng(9)
    n_points, n_loops, G = 7, 1000, 8          # 1000 loops: not a power of two
    W = rng.normal(size=(n_points, n_loops, 2))
    seed = 0x1234_5678_9ABC
    S, perm = ctx.group_sums_loops(W, G, shuffle=True, seed=seed, with_perm=True, where="host")
    want = np.stack([oracle.shuffle(seed, p, n_loops) for p in range(n_points)])
    assert np.array_equal(perm, want)
    ref = ost.group_sums_perm(W, G, want)
    assert np.array_equal(S[:, :, :2], ref)
    np.testing.assert_allclose(S[:, :, 3:], ost.group_sums_perm(W * W, G, want), rtol=1e-14)
    # device buffers give the same, and the totals are kept
    Sd, pd = ctx.group_sums_loops(torch.from_numpy(W).cuda(), G, shuffle=True, seed=seed,
                                  with_perm=True)
    assert np.array_equal(pd.cpu().numpy(), want) and np.array_equal(Sd.cpu().numpy(), S,
                                                                     equal_nan=True)
    np.testing.assert_allclose(S[:, :, :2].sum(axis=1), W.sum(axis=1), rtol=1e-12)


def test_corrcoef_matches_oracle(ctx):
    rng = np.random.default_rng(10)
    W = rng.normal(size=(12, 777, 2))
    W[5] = 2.0 * W[0] + 1.0
    for comp in (0, 1):
        got = ctx.corrcoef(W, 3, comp=comp, where="host")
        np.testing.assert_allclose(got, ost.corrcoef_ref(W[:, :, comp], 3), rtol=1e-12, atol=1e-14)
    assert ctx.corrcoef(W, 0, where="host")[5] == pytest.approx(1.0, abs=1e-14)
    S = rng.normal(size=(9, 32, 5))
    np.testing.assert_allclose(ctx.corrcoef(S, 2, comp=1, where="host"),
                               ost.corrcoef_ref(S[:, :, 1], 2), rtol=1e-12, atol=1e-14)


def test_fig_corr_shuffled_groups_decorrelate(ctx):
    # the paper's Fig. corr set-up: correlation of <W(T)> with <W(T = 3)> over
    # loops, over fixed groups and over groups drawn anew for every T
    n_loops, G = 4096, 64
    _, ens = _ensemble(ctx, 12, n_loops, 256)
    prof = I.Profile(1, B=1.0)
    T = np.array([1.0, 2.0, 2.5, 3.0, 3.5, 4.0, 6.0])
    W = ctx.wilson_loops(ens, [prof], [np.zeros(1)], [T], prec="fp32")
    ref = 3
    loops = ctx.corrcoef(W, ref, comp=1, where="host")
    S, _ = ctx.group_sums_loops(W, G)
    fixed = ctx.corrcoef(S, ref, comp=1, where="host")
    Ss, _ = ctx.group_sums_loops(W, G, shuffle=True, seed=77)
    shuffled = ctx.corrcoef(Ss, ref, comp=1, where="host")
    near = [2, 4]                                      # T = 2.5 and 3.5
    assert np.all(loops[near] > 0.5) and np.all(fixed[near] > 0.5)
    others = [i for i in range(len(T)) if i != ref]
    assert np.all(np.abs(shuffled[others]) < 4.5 / np.sqrt(G))
    ens.free()
