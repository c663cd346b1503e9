"""GPU parity of the full effective action (wln_effective_action_full)
against the oracle's full_effective_action, through the C ABI.

Inputs are seeded synthetic group sums, and the oracle's own group sums of
oracle loops, never values made by the CUDA path.  Bar: 1e-12 relative
(the same double-precision arithmetic in a different summation order), for
the per-group action, the per-radius T integrals and the integrand with their
group means and standard errors, and the LCF columns.

Cases: mapped radii and times with the small-T part (Sec. "Renormalization",
Sec. "Computing an Effective Action"), linear radii with geometric times,
mixed kinds in one batch, constant fields, single-node axes; grids that do
not follow their kind are refused.
"""
import math

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

M = ost.GRID_MAPPED


@pytest.fixture(scope="module")
def ctx():
    from paper_1407_7486_gb300 import build
    build.build()
    c = wln.Context(0)
    yield c
    c.close()


def _batch():
    profs = [I.Profile(0, F=2 * math.pi * 10.0, lam=1.0), I.Profile(0, F=3.0, lam=0.4),
             I.Profile(1, B=0.7), I.Profile(0, F=20.0, lam=2.0)]
    rhos = [ost.mapped_nodes(17, 1.5, 0.0), I.lin_grid(0.0, 2.0, 9), np.zeros(1),
            ost.mapped_nodes(1, 2.0, 0.0)]
    Ts = [ost.mapped_nodes(24, 1.0, 0.02), I.log_grid(0.02, 8.0, 12),
          ost.mapped_nodes(9, 3.0, 0.05), ost.mapped_nodes(1, 1.0, 0.1)]
    quads = [(M, M, 1.5, 1.0, True), (ost.GRID_LINEAR, ost.GRID_LOG, 0.0, 0.0, True),
             (ost.GRID_LINEAR, M, 0.0, 3.0, False), (M, M, 2.0, 1.0, True)]
    return profs, rhos, Ts, quads


def _check(got, S, lpg, profs, rhos, Ts, quads, spinor):
    off = roff = 0
    for q, (p, r, t, qd) in enumerate(zip(profs, rhos, Ts, quads)):
        n = len(r) * len(t)
        ref = ost.full_effective_action(S[off:off + n], lpg, p, r, t, qd[0], qd[1],
                                        rho_scale=qd[2], T_scale=qd[3], small_T=qd[4],
                                        spinor=spinor)
        kw = dict(rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(got["gamma_groups"][q], ref["gamma"], **kw)
        G = ref["gamma"].size
        g_mean = ref["gamma"].mean()
        g_sem = math.sqrt(((ref["gamma"] - g_mean) ** 2).sum() / (G * (G - 1)))
        np.testing.assert_allclose(got["gamma"][q], [g_mean, g_sem, ref["gamma_lcf"]], **kw)
        D = got["density"][roff:roff + len(r)]
        np.testing.assert_allclose(D[:, 0], ref["D"].mean(axis=1), **kw)
        np.testing.assert_allclose(D[:, 1], ref["D"].std(axis=1, ddof=1) / math.sqrt(G),
                                   rtol=1e-10, atol=1e-300)
        np.testing.assert_allclose(D[:, 2], ref["D_lcf"], **kw)
        In = got["integrand"][off:off + n].reshape(len(t), len(r), 3)
        np.testing.assert_allclose(In[:, :, 0], ref["I"].mean(axis=2), **kw)
        np.testing.assert_allclose(In[:, :, 1], ref["I"].std(axis=2, ddof=1) / math.sqrt(G),
                                   rtol=1e-10, atol=1e-300)
        np.testing.assert_allclose(In[:, :, 2], ref["I_lcf"], **kw)
        off += n
        roff += len(r)


@pytest.mark.parametrize("spinor", [True, False])
def test_full_action_on_synthetic_sums(ctx, spinor):
    profs, rhos, Ts, quads = _batch()
    G, lpg = 8, 16
    n = sum(len(a) * len(b) for a, b in zip(rhos, Ts))
    S = np.random.default_rng(5).normal(size=(n, G, 5))
    Q = [wln.Quad(*qd) for qd in quads]
    got = ctx.effective_action_full(profs, rhos, Ts, S, G, lpg, quad=Q, spinor=spinor,
                                    where="host")
    _check(got, S, lpg, profs, rhos, Ts, quads, spinor)
    dev = ctx.effective_action_full(profs, rhos, Ts, torch.from_numpy(S).cuda(), G, lpg,
                                    quad=Q, spinor=spinor, where="device")
    for k in got:
        assert np.array_equal(got[k], dev[k].cpu().numpy()), k


def test_full_action_on_oracle_loop_sums(ctx):
    # realistic sums: the oracle's group sums of oracle loops (flux tube, mapped grids)
    prof = I.Profile(0, F=2 * math.pi * 10.0, lam=1.0)
    rho, T = ost.mapped_nodes(9, 1.5, 0.0), ost.mapped_nodes(12, 1.0, 0.02)
    G, n_loops = 4, 64
    y = oracle.gen_loops(3, n_loops, 128)
    S = oracle.group_sums(y, prof, rho, T, G)
    qd = (M, M, 1.5, 1.0, True)
    for spinor in (True, False):
        got = ctx.effective_action_full([prof], [rho], [T], S, G, n_loops // G,
                                        quad=[wln.Quad(*qd)], spinor=spinor, where="host")
        _check(got, S, n_loops // G, [prof], [rho], [T], [qd], spinor)


def test_default_quadrature_matches_effective_action(ctx):
    profs = [I.Profile(0, F=10.0, lam=1.0), I.Profile(1, B=0.5)]
    rhos, Ts = [I.lin_grid(0, 5, 16), I.lin_grid(0, 1, 3)], [I.log_grid(0.01, 10, 16),
                                                              I.log_grid(0.1, 1, 5)]
    G, lpg = 8, 20
    n = sum(len(a) * len(b) for a, b in zip(rhos, Ts))
    S = np.random.default_rng(2).normal(size=(n, G, 5))
    gg, ms = ctx.effective_action(profs, rhos, Ts, S, G, lpg, where="host")
    full = ctx.effective_action_full(profs, rhos, Ts, S, G, lpg, quad=None, where="host")
    np.testing.assert_allclose(full["gamma_groups"], gg, rtol=1e-12)
    np.testing.assert_allclose(full["gamma"][:, :2], ms, rtol=1e-10)


def test_full_action_rejects_grids_off_their_kind(ctx):
    prof = I.Profile(0, F=10.0, lam=1.0)
    rho, T = I.lin_grid(0, 2, 5), I.log_grid(0.02, 8.0, 6)
    S = np.zeros((30, 4, 5))
    with pytest.raises(wln.WlnError):     # geometric times declared as mapped
        ctx.effective_action_full([prof], [rho], [T], S, 4, 4,
                                  quad=[wln.Quad(ost.GRID_LINEAR, M, 0.0, 1.0)], where="host")
    with pytest.raises(wln.WlnError):     # mapped grid without a scale
        ctx.effective_action_full([prof], [rho], [ost.mapped_nodes(6, 1.0, 0.02)], S, 4, 4,
                                  quad=[wln.Quad(ost.GRID_LINEAR, M, 0.0, 0.0)], where="host")
    with pytest.raises(wln.WlnError):     # linear radii declared as mapped
        ctx.effective_action_full([prof], [rho], [T], S, 4, 4,
                                  quad=[wln.Quad(M, ost.GRID_LOG, 1.0, 0.0)], where="host")


@pytest.mark.parametrize("spinor", [True, False])
def test_wide_tube_agrees_with_lcf_within_statistics(ctx, spinor):
    # Sec. "Verification and Validation", Fig. vsrhocm: for a tube much wider
    # than the Compton wavelength (lambda = 10, calF = 10) the worldline action
    # density agrees with the LCF approximation within the statistics.  Mapped
    # grids as in Sec. "Computing an Effective Action", small-T part below a = 1.
    prof = I.Profile(0, F=2 * math.pi * 10.0, lam=10.0)
    n_loops, G = 10240, 32
    ens = ctx.gen_loops(1, n_loops, 2048)
    rho, T = wln.mapped_grid(48, 10.0, 0.0), wln.mapped_grid(64, 2.0, 1.0)
    S = ctx.wilson_avg(ens, [prof], [rho], [T], G, prec="fp32")
    r = ctx.effective_action_full([prof], [rho], [T], S, G, n_loops // G,
                                  quad=[wln.Quad(M, M, 10.0, 2.0, True)], spinor=spinor,
                                  where="host")
    D = r["density"]
    z = (D[:, 0] - D[:, 2]) / D[:, 1]
    assert np.all(np.isfinite(z)) and np.all(np.abs(z) < 4.0), np.abs(z).max()
    g = r["gamma"][0]
    assert abs(g[0] - g[2]) < 4.0 * g[1]
    # the LCF sign is the physical one: spinor action density negative, scalar positive
    assert (D[0, 2] < 0) == spinor
    ens.free()
