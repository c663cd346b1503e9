"""GPU checks of the precision guard of the FP32-compensated group sums.

The spinor group mean of a strong tube is carried by its few loops of
largest spin, whose float rounding cosh(spin) magnifies (Sec. "Uncertainties
and the Fermion Problem").  The guard recomputes those loops in double-float.
  * The double-float walk against the oracle: with every recorded loop
    recomputed (guard mode "all") and every 32-loop block recorded (each holds
    a spin of at least 2, checked with the oracle), the spinor group means
    match the FP64 oracle within 1e-10 of max(1, <cosh spin>) -- a bound set
    by the double-float arithmetic (~2^-44 per term), not by float.
  * The guard leaves weak fields alone: for spins below 2 nothing is
    recorded, and the sums equal the unguarded ones bit for bit; it never
    changes the scalar components.
  * It is deterministic: repeated runs, a reusable batch (also replayed from a
    CUDA graph) and the server give the same bits as wln_wilson_avg.
  * Its statistics count the recomputed loops.
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
    c = wln.Context(0, torch.cuda.Stream(0))
    yield c
    c.set_precision_guard(True)
    c.close()


def _ens(ctx, seed, n_loops, ppl):
    y32 = oracle.gen_loops(seed, n_loops, ppl).astype(np.float32)
    return y32, ctx.ensemble_from_host(y32)


ALL_CASES = [
    # (n_loops, ppl, G, profile, rho, T): every block reaches spin 2
    (128, 512, 2, I.Profile(0, F=50.0, lam=1.0), np.array([0.0, 0.5]), np.array([1.0, 20.0])),
    (128, 256, 2, I.Profile(0, F=100.0, lam=0.1), np.array([0.0, 0.3]), np.array([1.0, 10.0])),
    (96, 1024, 3, I.Profile(0, F=100.0, lam=1.0), np.array([0.0, 1.0]), np.array([2.0, 10.0])),
]


@pytest.mark.parametrize("case", range(len(ALL_CASES)))
def test_double_float_walk_matches_oracle(ctx, case):
    n_loops, ppl, G, prof, rho, T = ALL_CASES[case]
    y32, ens = _ens(ctx, 31 + case, n_loops, ppl)
    y = y32.astype(np.float64)
    lpg = n_loops // G
    ref = oracle.group_sums(y, prof, rho, T, G)
    cosh = np.zeros((len(T) * len(rho), G))
    for b, t in enumerate(T):
        for a, r in enumerate(rho):
            _, sp = oracle.phase_spin(y, prof, r, t)
            assert np.all(np.abs(sp).reshape(-1, 32).max(axis=1) >= 2.0), "a block below 2"
            cosh[b * len(rho) + a] = np.cosh(sp).reshape(G, -1).sum(axis=1)
    ctx.set_precision_guard("all")
    try:
        ctx.precision_guard_stats(reset=True)
        S = ctx.wilson_avg(ens, [prof], [rho], [T], G, prec="fp32", where="host")
        st = ctx.precision_guard_stats()
    finally:
        ctx.set_precision_guard(True)
    assert st["escalated_loops"] == n_loops * len(rho) * len(T) and st["saturated"] == 0
    err = np.abs(S[:, :, 1] - ref[:, :, 1]) / np.maximum(cosh, lpg)
    print(f"case {case}: double-float spinor error {err.max():.2e} of max(1, <cosh s>)")
    assert err.max() <= 1e-10
    ens.free()


def test_weak_field_untouched_and_scalar_components_unchanged(ctx):
    y32, ens = _ens(ctx, 41, 640, 1024)
    args = ([I.Profile(0, F=1.0, lam=1.0)], [I.lin_grid(0, 4, 5)], [I.log_grid(0.01, 5, 4)], 2)
    ctx.set_precision_guard(False)
    off = ctx.wilson_avg(ens, *args, prec="fp32", where="host")
    ctx.set_precision_guard(True)
    ctx.precision_guard_stats(reset=True)
    on = ctx.wilson_avg(ens, *args, prec="fp32", where="host")
    assert np.array_equal(on, off)
    assert ctx.precision_guard_stats()["escalated_loops"] == 0
    strong = ([I.Profile(0, F=50.0, lam=1.0)], [np.array([0.0, 0.2])], [np.array([5.0, 20.0])], 2)
    ctx.set_precision_guard(False)
    off = ctx.wilson_avg(ens, *strong, prec="fp32", where="host")
    ctx.set_precision_guard(True)
    on = ctx.wilson_avg(ens, *strong, prec="fp32", where="host")
    for comp in (wln.C_SCAL, wln.C_SIN, wln.C_SCAL_SQ):
        assert np.array_equal(on[:, :, comp], off[:, :, comp])
    assert not np.array_equal(on[:, :, wln.C_FERM], off[:, :, wln.C_FERM])
    ens.free()


def test_guard_is_deterministic_in_every_path(ctx):
    y32, ens = _ens(ctx, 42, 640, 2048)
    prof, rho, T, G = I.Profile(0, F=50.0, lam=1.0), I.lin_grid(0, 2, 6), np.array([3.0, 20.0]), 2
    ctx.precision_guard_stats(reset=True)
    a = ctx.wilson_avg(ens, [prof], [rho], [T], G, prec="fp32", where="host")
    b = ctx.wilson_avg(ens, [prof], [rho], [T], G, prec="fp32", where="host")
    assert np.array_equal(a, b)
    st = ctx.precision_guard_stats()
    assert st["escalated_loops"] > 0 and st["overflows"] == 0
    bt = wln.Batch(ctx, ens, [prof], [rho], [T], G, prec="fp32")
    bt.run(graph=False)
    assert np.array_equal(bt.results()[0], a)
    bt.run(graph=True)
    bt.run(graph=True)
    assert np.array_equal(bt.results()[0], a)
    bt.free()
    sv = wln.Server(ctx, ens, G, arena_bytes=64 << 20, tile_groups_per_step=2)
    rid = sv.submit(prof, rho, T)
    for _ in range(1000):
        sv.step()
        state, res = sv.poll(rid)
        if state == sv.DONE:
            break
    assert state == sv.DONE
    ref = ctx.wilson_avg(ens, [prof], [rho], [T], G, prec="fp32", where="host")
    # the server's fixed decomposition (chain length) may differ from the
    # one-shot call's; its sums agree to double rounding of the group order
    lpg = 640 // G
    y = y32.astype(np.float64)
    cs = np.array([np.cosh(oracle.phase_spin(y, prof, r, t)[1]).reshape(G, -1).sum(axis=1)
                   for t in T for r in rho])
    assert np.all(np.abs(res[0][:, :, 1] - ref[:, :, 1]) <= 1e-12 * np.maximum(cs, lpg))
    sv.free()
    ens.free()


def _strong_grid():
    # 1024 loops of 256 points in 16 groups of 2 blocks, a strong tube on
    # 64 T x 80 rho where every block reaches spin 2: with every recorded loop
    # recomputed (mode "all"), a pass selects all 64 loops of every (point,
    # group), 5,242,880 in all.  That is above the 2^22 entries a call takes
    # up front, so the queue starts at 8 per (point, group), 655,360, and the
    # float pass's count has to regrow it
    return (I.Profile(0, F=50.0, lam=1.0), I.lin_grid(0.0, 1.0, 80), I.log_grid(2.0, 20.0, 64), 16)


def test_queue_grows_to_what_the_float_pass_selects(ctx):
    """A pass whose guard selects more loops than the queue first holds runs
    again with the queue sized to them: no selection is dropped, the
    double-float results match the oracle (on sampled points), and a batch
    does the same on its first run (its later graph replays give the same
    bits)."""
    prof, rho, T, G = _strong_grid()
    y32, ens = _ens(ctx, 43, 1024, 256)
    y = y32.astype(np.float64)
    lpg = 1024 // G
    ctx.set_precision_guard("all")
    try:
        ctx.precision_guard_stats(reset=True)
        S = ctx.wilson_avg(ens, [prof], [rho], [T], G, prec="fp32", where="host")
        st = ctx.precision_guard_stats(reset=True)
        bt = wln.Batch(ctx, ens, [prof], [rho], [T], G, prec="fp32")
        bt.run(graph=True)
        first = bt.results()[0]
        bt.run(graph=True)
        bt.run(graph=True)
        replay = bt.results()[0]
        st_b = ctx.precision_guard_stats(reset=True)
        bt.free()
    finally:
        ctx.set_precision_guard(True)
    n_sel = len(rho) * len(T) * G * 64
    assert st["overflows"] == 0 and st["escalated_loops"] == n_sel, st
    assert st_b["overflows"] == 0 and st_b["escalated_loops"] == 3 * n_sel, st_b
    assert np.array_equal(first, S) and np.array_equal(replay, S)
    rng = np.random.default_rng(44)
    worst = 0.0
    for p in rng.choice(len(rho) * len(T), 32, replace=False):
        r, t = rho[p % len(rho)], T[p // len(rho)]
        ref = oracle.group_sums(y, prof, [r], [t], G)[0]
        _, sp = oracle.phase_spin(y, prof, r, t)
        cosh = np.cosh(sp).reshape(G, -1).sum(axis=1)
        worst = max(worst, float((np.abs(S[p, :, 1] - ref[:, 1]) / np.maximum(cosh, lpg)).max()))
    assert worst <= 1e-10, worst
    ens.free()
