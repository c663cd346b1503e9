"""Parity at the full size of the benchmark's workloads for the rows beyond the
plain pass, in the launch configurations bench.py times (its defaults).

  * d-loops (`bench.py --dloops`): the paper ensemble's 10240 loops x 2048
    points drawn as d-loops (Eqs. yn2, ynk); 48 loops spread over the
    ensemble, regenerated by the oracle from their global index
    (counter-based Philox), double copy within 1e-13.
  * Discretisation levels and nested levels (`bench.py --levels [--nested]`):
    the paper workload (3 flux tubes, 24576 points, 32 groups) through
    wln_wilson_levels / wln_wilson_levels_nested; 24 seeded (profile, point,
    group) samples and, per tube, the point of largest spin (the smallest
    radius at the longest time) in two groups.  Each sampled group mean of
    every level component lies within its per-loop rounding bar (the R15 bar
    of the level tests, averaged over the group's loops), the oracle working
    on the same float points.
  * Per-loop values (`bench.py --correlation`): the bench's tube (F = 10), all
    8192 points x 10240 loops through wln_wilson_loops; 64 seeded (point,
    loop) samples and the largest-spin point's first loops against
    oracle.loop_values within the per-loop bar.
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

REL, TOL = 2.0 ** -21, 1e-6


@pytest.fixture(scope="module")
def ctx():
    from paper_1407_7486_gb300 import build
    build.build()
    stream = torch.cuda.Stream(0)
    c = wln.Context(0, stream)
    yield c
    c.close()


def _samples(rng, wl, n_random):
    """(profile, point index, group): seeded picks, then every tube's point of
    largest spin (first radius, last time) in its first and last group."""
    out = []
    for _ in range(n_random):
        q = int(rng.integers(len(wl.profiles)))
        out.append((q, int(rng.integers(len(wl.rho[q]) * len(wl.T[q]))),
                    int(rng.integers(wl.n_groups))))
    for q in range(len(wl.profiles)):
        p = (len(wl.T[q]) - 1) * len(wl.rho[q])
        out += [(q, p, 0), (q, p, wl.n_groups - 1)]
    return out


def _bar(subs, weights, prof, r, t):
    """Per-loop (scalar, spinor) bars of one level: the walks' sums of
    |segment phase| and spins combined with the level's weights."""
    ps = [oracle.phase_spin(s, prof, r, t) for s in subs]
    pa = [oracle.phase_abs(s, prof, r, t) for s in subs]
    P = sum(w * x for w, x in zip(weights, pa))
    s = sum(w * x[1] for w, x in zip(weights, ps))
    with np.errstate(over="ignore", invalid="ignore"):
        es = np.maximum(TOL, REL * P)
        ef = np.maximum(1.0, np.cosh(s)) * np.maximum(TOL, REL * (np.abs(s) + P))
    return es.mean(), ef.mean()


def test_dloops_full_size_sampled(ctx):
    wl = I.paper()
    ens = ctx.gen_dloops(wl.seed, wl.n_loops, wl.ppl, keep_fp64=True)
    _, f64 = ctx.loops_copy(ens, f32=False, f64=True)
    ens.free()
    picks = np.unique(np.concatenate([np.linspace(0, wl.n_loops - 1, 40).astype(int),
                                      np.random.default_rng(5).integers(0, wl.n_loops, 8)]))
    for l in picks:
        ref = oracle.gen_dloops(wl.seed, 1, wl.ppl, loop0=int(l))[0]
        assert np.abs(f64[l] - ref).max() < 1e-13, l


@pytest.mark.parametrize("nested", [False, True])
def test_levels_full_size_sampled(ctx, nested):
    wl = I.paper()
    lpg = wl.n_loops // wl.n_groups
    ens = ctx.gen_loops(wl.seed, wl.n_loops, wl.ppl)
    L = ctx.wilson_levels(ens, wl.profiles, wl.rho, wl.T, wl.n_groups, prec="fp32",
                          where="host", nested=nested)
    y32, _ = ctx.loops_copy(ens)
    ens.free()
    offs = np.cumsum([0] + [len(r) * len(t) for r, t in zip(wl.rho, wl.T)])
    if nested:
        weights = [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)]
    else:
        weights = [(0.5, 0.25, 0.25), (1.0, 0.0, 0.0), (0.0, 0.5, 0.5)]
    worst = 0.0
    n_checked = 0
    for q, p, g in _samples(np.random.default_rng(51 + nested), wl, 24):
        prof = wl.profiles[q]
        r, t = wl.rho[q][p % len(wl.rho[q])], wl.T[q][p // len(wl.rho[q])]
        y = y32[g * lpg:(g + 1) * lpg].astype(np.float64)
        if nested:
            subs = [y, np.ascontiguousarray(y[:, :, 0::2]), np.ascontiguousarray(y[:, :, 0::4])]
            ref = ost.nested_level_sums(oracle, y, prof, [r], [t], 1)[0, 0]
        else:
            subs = [np.ascontiguousarray(y[:, :, 0::2]), np.ascontiguousarray(y[:, :, 1::4]),
                    np.ascontiguousarray(y[:, :, 3::4])]
            ref = ost.level_sums(oracle, y, prof, [r], [t], 1)[0, 0]
        got = L[offs[q] + p, g]
        for lev, wts in enumerate(weights):
            bs, bf = _bar(subs, wts, prof, r, t)
            for c, b in ((2 * lev, bs), (2 * lev + 1, bf)):
                if not np.isfinite(ref[c]):
                    assert not np.isfinite(got[c]), (nested, q, p, g, c)
                    continue
                e = abs(got[c] - ref[c]) / lpg / b
                worst = max(worst, e)
                n_checked += 1
                assert e <= 1.0, (nested, q, p, g, c, e)
    print(f"nested={nested}: {n_checked} components, worst {worst:.3f} of the bar")
    assert n_checked >= 24 * 6


def test_loop_values_full_size_sampled(ctx):
    wl = I.paper()
    q = 1                                           # the bench's tube, F = 10
    prof, rho, T = wl.profiles[q], wl.rho[q], wl.T[q]
    n_points = len(rho) * len(T)
    ens = ctx.gen_loops(wl.seed, wl.n_loops, wl.ppl)
    W = torch.empty((n_points, wl.n_loops, 2), dtype=torch.float64, device="cuda:0")
    ctx.wilson_loops(ens, [prof], [rho], [T], prec="fp32", out=W)
    y32, _ = ctx.loops_copy(ens)
    ens.free()
    rng = np.random.default_rng(61)
    picks = [(int(rng.integers(n_points)), int(rng.integers(wl.n_loops))) for _ in range(64)]
    p_max = (len(T) - 1) * len(rho)                 # largest spin: first radius, last time
    picks += [(p_max, l) for l in range(8)]
    worst = 0.0
    for p, l in picks:
        r, t = rho[p % len(rho)], T[p // len(rho)]
        y = y32[l:l + 1].astype(np.float64)
        ref = oracle.loop_values(y, prof, [r], [t])[0, 0]
        got = W[p, l].cpu().numpy()
        ph, sp = oracle.phase_spin(y, prof, r, t)
        P = oracle.phase_abs(y, prof, r, t)[0]
        with np.errstate(over="ignore", invalid="ignore"):
            bs = max(TOL, REL * P)
            bf = max(1.0, np.cosh(sp[0])) * max(TOL, REL * (abs(sp[0]) + P))
        if not np.isfinite(ref[1]):
            assert not np.isfinite(got[1]), (p, l)
            continue
        es, ef = abs(got[0] - ref[0]) / bs, abs(got[1] - ref[1]) / bf
        worst = max(worst, es, ef)
        assert es <= 1.0 and ef <= 1.0, (p, l, es, ef)
    print(f"per-loop values: {len(picks)} samples, worst {worst:.3f} of the bar")
