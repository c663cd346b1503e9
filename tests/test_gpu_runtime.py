"""GPU tests of the runtime around the Wilson kernel: reusable batches with
CUDA-graph replay, and the continuous-batching request server.

  * Batch and server group sums against the FP64 oracle on the same loops,
    at the parity bar of test_gpu_parity.py (every profile of a batch; every
    request of the server, alone and mixed).
  * A batch's group sums equal wln_wilson_avg's bitwise, its statistics and
    effective action equal wln_jackknife's and wln_effective_action's, and a
    graph replay reproduces a direct run bitwise.
  * A server request's results are the same, bitwise, whether it runs alone or
    mixed with other requests in the same launches (the accumulation order of
    a request's sums does not depend on the mix), and agree with
    wln_wilson_avg to 1e-12 of the group-mean scale.
  * Admission by arena memory: with a small arena requests wait and still
    complete; a request that can never fit is refused at submission;
    cancelled requests leave the others intact.
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


@pytest.fixture(scope="module")
def ctx():
    from paper_1407_7486_gb300 import build
    build.build()
    stream = torch.cuda.Stream(0)
    c = wln.Context(0, stream)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ens(ctx):
    e = ctx.gen_loops(5, 1024, 256)
    yield e
    e.free()


def _profiles():
    rng = np.random.default_rng(11)
    profs, rhos, Ts = [], [], []
    for _ in range(5):
        lam = float(rng.uniform(0.3, 2.0))
        profs.append(I.Profile(0, F=float(10 ** rng.uniform(-1, 2)), lam=lam))
        rhos.append(I.lin_grid(0.0, 5 * lam, int(rng.integers(3, 20))))
        Ts.append(I.log_grid(0.01, 10.0, int(rng.integers(2, 12))))
    profs.append(I.Profile(1, B=0.8))
    rhos.append(np.zeros(1))
    Ts.append(I.log_grid(0.05, 5.0, 7))
    return profs, rhos, Ts


def _oracle_check(ctx, ens, profs, rhos, Ts, G, S, what):
    y32, _ = ctx.loops_copy(ens)
    y = y32.astype(np.float64)
    lpg = ens.n_loops // G
    off = 0
    for q, (p, r, t) in enumerate(zip(profs, rhos, Ts)):
        n = len(r) * len(t)
        ref = oracle.group_sums(y, p, r, t, G)
        _compare(S[off:off + n], ref, lpg, _bars(y32, p, r, t, G, 1e-6, F32_REL),
                 what=f"{what} profile {q}")
        off += n
    assert off == S.shape[0]


def test_batch_matches_one_shot_calls_and_graph_replay(ctx, ens):
    profs, rhos, Ts = _profiles()
    G, lpg = 8, ens.n_loops // 8
    b = wln.Batch(ctx, ens, profs, rhos, Ts, G, prec="fp32")
    b.run(graph=False)
    S0, st0, g0 = b.results()
    _oracle_check(ctx, ens, profs, rhos, Ts, G, S0, "batch")
    ref = ctx.wilson_avg(ens, profs, rhos, Ts, G, prec="fp32", where="host")
    assert np.array_equal(S0, ref)
    js = ctx.jackknife(ref, G, lpg, 0, jk_var=False, where="host")
    jf = ctx.jackknife(ref, G, lpg, 1, jk_var=False, where="host")
    assert np.array_equal(st0[0], js["mean"]) and np.array_equal(st0[1], js["sem"])
    assert np.array_equal(st0[2], jf["mean"]) and np.array_equal(st0[3], jf["sem"])
    _, ms = ctx.effective_action(profs, rhos, Ts, ref, G, lpg, spinor=True, where="host")
    _, mss = ctx.effective_action(profs, rhos, Ts, ref, G, lpg, spinor=False, where="host")
    assert np.array_equal(g0[0], ms) and np.array_equal(g0[1], mss)
    n0 = ctx.launch_count
    for _ in range(3):
        b.run(graph=True)
    S1, st1, g1 = b.results()
    assert ctx.launch_count - n0 == 3 * b.kernels_per_run and b.kernels_per_run >= 5
    assert np.array_equal(S1, S0) and np.array_equal(st1, st0) and np.array_equal(g1, g0)
    b.free()


def _drain(sv, ids, max_steps=10000):
    out = {}
    for _ in range(max_steps):
        sv.step()
        for rid in ids:
            if rid in out:
                continue
            state, res = sv.poll(rid)
            if state == sv.DONE:
                out[rid] = res
                sv.release(rid)
        if len(out) == len(ids):
            return out
    raise AssertionError("server did not finish")


def test_server_results_are_the_same_alone_and_mixed(ctx, ens):
    profs, rhos, Ts = _profiles()
    G = 8
    sv = wln.Server(ctx, ens, G, arena_bytes=256 << 20, tile_groups_per_step=3)
    alone = {}
    for q in range(len(profs)):
        rid = sv.submit(profs[q], rhos[q], Ts[q])
        alone[q] = _drain(sv, [rid])[rid]
    ids = [sv.submit(profs[q], rhos[q], Ts[q]) for q in range(len(profs))]
    mixed = _drain(sv, ids)
    for q, rid in enumerate(ids):
        for a, m in zip(alone[q], mixed[rid]):
            assert np.array_equal(a, m), q
        _oracle_check(ctx, ens, [profs[q]], [rhos[q]], [Ts[q]], G, mixed[rid][0],
                      f"server request {q}")
        ref = ctx.wilson_avg(ens, [profs[q]], [rhos[q]], [Ts[q]], G, prec="fp32", where="host")
        lpg = ens.n_loops // G
        scale = np.maximum(1.0, np.abs(ref) / lpg)
        assert np.all(np.abs(mixed[rid][0] - ref) / lpg <= 1e-12 * scale)
    assert sv.info()["steps"] > 0
    sv.free()


def test_server_admission_and_cancellation(ctx, ens):
    G = 8
    prof = I.Profile(0, F=10.0, lam=1.0)
    rho, T = I.lin_grid(0, 5, 40), I.log_grid(0.01, 10, 20)     # 800 points
    sv = wln.Server(ctx, ens, G, arena_bytes=8 << 20, tile_groups_per_step=4)
    with pytest.raises(wln.WlnError):
        sv.submit(prof, I.lin_grid(0, 5, 256), I.log_grid(0.01, 10, 128))   # never fits 8 MiB
    small = [sv.submit(prof, rho[:10], T[:5]) for _ in range(6)]
    victim_q = sv.submit(prof, rho, T)
    victim_a = sv.submit(prof, rho[:12], T[:6])
    sv.cancel(victim_q)                                  # cancelled while queued
    a, q = sv.step()
    assert a + q >= 1
    sv.cancel(victim_a)                                  # cancelled while admitted or queued
    done = _drain(sv, small)
    assert len(done) == len(small)
    first = done[small[0]][0]
    for rid in small[1:]:
        assert np.array_equal(done[rid][0], first)       # identical requests, identical results
    assert sv.info()["queued"] == 0
    sv.free()
