"""Parity of the batch and server paths at the full size of their timed
workloads, in the launch configurations the benchmark uses.

  * Batched workload: its ensemble (16384 loops x 4096 points, seed 1, 32
    groups) and the first 6 of its 64 flux tubes (host seed 4: F log-uniform
    in [0.1, 100], lambda uniform in [0.2, 3], uneven grids of 8-256 radii x
    8-128 times), through wln_batch with CUDA-graph replay and the default
    tile shape (4 radii x 8 warps, 64-row chunks, 2 stages, the shape the
    autotuner picks on that workload).
  * Serving workload: its ensemble (32768 loops x 4096 points, 32 groups)
    and the first 2 requests of the seed-7 Poisson stream, through
    wln_server with the benchmark's arena (16 GiB) and step size (128 tile
    groups).

The oracle cannot redo these launches in test time, so it recomputes sampled
group means one by one on the same float loops: seeded (profile, point,
group) samples and, per tube, the point of largest spin (the smallest radius
at the longest time).  Each sampled group mean stays within the plain bar,
1e-6 for the scalar and 1e-6 of max(1, <cosh s>) for the spinor, wherever the
oracle's cosh s is finite in double (thin strong tubes reach spins beyond
710 at long times, where the spinor sum has no finite value to compare).
"""
import numpy as np
import pytest

import oracle
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
    stream = torch.cuda.Stream(0)
    c = wln.Context(0, stream)
    yield c
    c.close()


def _samples(rng, profiles, rhos, Ts, n_groups, n_random):
    """(profile, point index, group): seeded picks, then every tube's point of
    largest spin (rho first in the grid, T last) in two groups."""
    out = []
    for _ in range(n_random):
        q = int(rng.integers(len(profiles)))
        n = len(rhos[q]) * len(Ts[q])
        out.append((q, int(rng.integers(n)), int(rng.integers(n_groups))))
    for q in range(len(profiles)):
        p = (len(Ts[q]) - 1) * len(rhos[q])
        out += [(q, p, 0), (q, p, n_groups - 1)]
    return out


def _check_samples(y32, profiles, rhos, Ts, S, n_groups, samples, what):
    lpg = y32.shape[0] // n_groups
    offs = np.cumsum([0] + [len(r) * len(t) for r, t in zip(rhos, Ts)])
    n_finite = 0
    worst_s = worst_f = 0.0
    for q, p, g in samples:
        r, t = rhos[q][p % len(rhos[q])], Ts[q][p // len(rhos[q])]
        yg = y32[g * lpg:(g + 1) * lpg].astype(np.float64)
        ref = oracle.group_sums(yg, profiles[q], [r], [t], 1)[0, 0]
        got = S[offs[q] + p, g]
        _, sp = oracle.phase_spin(yg, profiles[q], r, t)
        with np.errstate(over="ignore"):
            cs = float(np.cosh(sp).sum())
        assert np.isfinite(ref[0]) and np.isfinite(got[0]), (what, q, p, g)
        e_s = abs(got[0] - ref[0]) / lpg
        worst_s = max(worst_s, e_s)
        assert e_s <= 1e-6, (what, "scalar", q, p, g, e_s)
        if np.isfinite(cs) and np.isfinite(ref[1]):
            e_f = abs(got[1] - ref[1]) / max(cs, lpg)
            worst_f = max(worst_f, e_f)
            assert e_f <= 1e-6, (what, "spinor", q, p, g, e_f)
            n_finite += 1
    print(f"{what}: {len(samples)} samples ({n_finite} with finite cosh sums), "
          f"scalar {worst_s:.2e}, spinor / <cosh s> {worst_f:.2e}")
    assert n_finite >= len(samples) // 2


def test_batched_workload_full_size_sampled(ctx):
    wl = I.batched()
    profs, rhos, Ts = wl.profiles[:6], wl.rho[:6], wl.T[:6]
    ens = ctx.gen_loops(wl.seed, wl.n_loops, wl.ppl)
    ctx.set_tuning(4, 8, 64, 2)
    try:
        b = wln.Batch(ctx, ens, profs, rhos, Ts, wl.n_groups, prec="fp32")
        b.run(graph=True)
        b.run(graph=True)
        S, _, _ = b.results()
        b.free()
    finally:
        ctx.set_tuning()
    y32, _ = ctx.loops_copy(ens)
    ens.free()
    samples = _samples(np.random.default_rng(41), profs, rhos, Ts, wl.n_groups, 24)
    _check_samples(y32, profs, rhos, Ts, S, wl.n_groups, samples, "batched")


def test_serving_workload_full_size_sampled(ctx):
    cfg = I.serving_ensemble()
    reqs = I.request_stream(2)
    ens = ctx.gen_loops(cfg["seed"], cfg["n_loops"], cfg["ppl"])
    sv = wln.Server(ctx, ens, cfg["n_groups"], prec="fp32", arena_bytes=16 << 30,
                    tile_groups_per_step=128)
    ids = [sv.submit(r.profile, r.rho, r.T) for r in reqs]
    res = {}
    for _ in range(100000):
        sv.step()
        for rid in ids:
            if rid not in res:
                state, out = sv.poll(rid)
                if state == sv.DONE:
                    res[rid] = out
                    sv.release(rid)
        if len(res) == len(ids):
            break
    assert len(res) == len(ids), "server did not finish"
    sv.free()
    y32, _ = ctx.loops_copy(ens)
    ens.free()
    rng = np.random.default_rng(43)
    for k, (r, rid) in enumerate(zip(reqs, ids)):
        samples = _samples(rng, [r.profile], [r.rho], [r.T], cfg["n_groups"], 12)
        _check_samples(y32, [r.profile], [r.rho], [r.T], res[rid][0], cfg["n_groups"], samples,
                       f"serving request {k}")
