"""GPU parity of the CUDA path against the FP64 CPU oracle, through the C ABI.

Tolerances:
  * Philox words: bit-exact.
  * Loops: the double copy within 1e-13 absolute (coordinates are O(1));
    float copies identical except where the double value sits on a float
    rounding boundary (at most one unit in the last place).
  * Group means of W - 1, FP64 path: |d<W>| <= 1e-12 * scale.
  * Group means of W - 1, FP32 compensated path: |d<W>| <= 1e-6 * scale.
    scale = 1 for the scalar loop and the imaginary part, and
    max(1, mean over the group of cosh(spin)) for the spinor loop (the
    fermion factor grows like cosh, Sec. "Uncertainties and the Fermion
    Problem").
  * Statistics and quadrature on identical group sums: 1e-12 relative.
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


def _ensemble_from_oracle(ctx, seed, n_loops, ppl):
    y = oracle.gen_loops(seed, n_loops, ppl).astype(np.float32)
    return y, ctx.ensemble_from_host(y)


# Relative precision of a phase or spin summed from float segment terms: each
# term passes through about eight roundings (geometry, closed forms, the
# arctangent, the products), so a loop's phase and spin carry up to ~8 ulps
# (2^-21) of the sum of their terms' magnitudes, P = sum_k |phase_k| and s,
# and W an error of about 2^-21 P (scalar) and cosh(s) 2^-21 (s + P)
# (spinor).  Where that exceeds the 1e-6 bar (phases or spins of tens of
# radians) it is the bar.  The FP64 path uses 2^-50.
F32_REL = 2.0 ** -21
F64_REL = 2.0 ** -50


def _bars(y32, profile, rho, T, G, tol, rel):
    """Per-loop error bars from the oracle's phases and spins, averaged over each
    group and over the ensemble (worst case: no credit for cancellation):
      E_scal = max(tol, rel P),  P = sum over segments of |segment phase|
      E_ferm = max(1, cosh s) max(tol, rel (s + P))
    and, for the (W-1)^2 diagnostics, 2 |w| E + E^2.  Returns
    {comp: (group bars [n_points][G], ensemble bars [n_points])}."""
    y = y32.astype(np.float64)
    lpg = y.shape[0] // G
    n = len(T) * len(rho)
    out = {c: (np.zeros((n, G)), np.zeros(n)) for c in range(5)}
    for b, t in enumerate(T):
        for a, r in enumerate(rho):
            ph, sp = oracle.phase_spin(y, profile, r, t)
            pa = oracle.phase_abs(y, profile, r, t)          # sum of |segment phases|
            with np.errstate(over="ignore", invalid="ignore"):
                ch = np.cosh(sp)
                es = np.maximum(tol, rel * pa)
                ef = np.maximum(1.0, ch) * np.maximum(tol, rel * (sp + pa))
                ws = np.cos(ph) - 1.0
                wf = np.cos(ph) * ch - 1.0
                per = {0: es, 1: ef, 2: es, 3: 2 * np.abs(ws) * es + es ** 2,
                       4: 2 * np.abs(wf) * ef + ef ** 2}
            p = b * len(rho) + a
            for c, e in per.items():
                out[c][0][p] = e.reshape(G, lpg).mean(axis=1)
                out[c][1][p] = e.mean()
    return out


def _compare(gpu, ref, lpg, bars, what=""):
    """Every group mean and the ensemble mean <W> within their bars.  Squares can
    exceed the double range for huge spins (cosh(s) > 1e154); both sides must
    then agree on which entries are infinite."""
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(gpu)), f"{what}: non-finite entries differ"
    worst = {}
    with np.errstate(over="ignore", invalid="ignore"):
        dg = np.where(fin, gpu - ref, 0.0) / lpg              # group-mean differences
        de = np.abs(dg.mean(axis=1))                          # ensemble-mean differences
        for comp in range(5):
            bg, be = bars[comp]
            worst_e = np.nan_to_num(de[:, comp] / be).max()
            worst_g = np.nan_to_num(np.abs(dg[:, :, comp]) / bg).max()
            worst[comp] = (worst_e, worst_g)
            assert worst_e <= 1.0, f"{what} comp {comp}: ensemble mean {worst_e:.3g} x bar"
            assert worst_g <= 1.0, f"{what} comp {comp}: group mean {worst_g:.3g} x bar"
    print(what, {k: (round(float(a), 3), round(float(b), 3)) for k, (a, b) in worst.items()})


def test_philox_stream_bit_exact(ctx):
    for seed, loop0 in ((1, 0), (0xDEADBEEFCAFE, 12345)):
        got = ctx.philox_stream(seed, loop0, 37, 129)
        want = oracle.philox_stream(seed, 37, 129, loop0=loop0)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("n_loops,ppl", [(40, 4), (96, 64), (33, 512), (64, 2048), (32, 16384)])
def test_generated_loops_match_oracle(ctx, n_loops, ppl):
    ens = ctx.gen_loops(7, n_loops, ppl, keep_fp64=True)
    f32, f64 = ctx.loops_copy(ens, f32=True, f64=True)
    ref = oracle.gen_loops(7, n_loops, ppl)
    assert np.abs(f64 - ref).max() < 1e-13
    ref32 = ref.astype(np.float32)
    diff = f32 != ref32
    assert diff.mean() < 1e-4
    if diff.any():
        ulp = np.spacing(np.abs(ref32[diff]))
        assert np.all(np.abs(f32[diff] - ref32[diff]) <= ulp)
    ens.free()


@pytest.mark.parametrize("gen", ["increments", "dloops"])
def test_generation_across_scratch_slices(ctx, gen):
    """Ensembles whose raw increments (Gaussians) exceed one 1 GiB slice of
    scratch are generated slice by slice: at ppl = 16384 a slice holds 120
    blocks of 32 loops for the increments (3840 loops) and 128 for d-loops
    (4096).  Loops on both sides of every slice boundary, and the last
    (partial) block, match the oracle regenerated from their global index."""
    n_loops, ppl, loop0 = 8200, 16384, 7
    draw = ctx.gen_loops if gen == "increments" else ctx.gen_dloops
    ref_of = oracle.gen_loops if gen == "increments" else oracle.gen_dloops
    slice_loops = 3840 if gen == "increments" else 4096
    ens = draw(11, n_loops, ppl, keep_fp64=True, loop0=loop0)
    _, f64 = ctx.loops_copy(ens, f32=False, f64=True)
    ens.free()
    picks = []
    for b in (slice_loops, 2 * slice_loops):
        picks += [b - 2, b - 1, b, b + 1]
    picks += [0, n_loops - 1]
    for l in picks:
        ref = ref_of(11, 1, ppl, loop0=loop0 + l)[0]
        assert np.abs(f64[l] - ref).max() < 1e-13, (gen, l)


def test_freed_ensemble_memory_is_reused_cleanly():
    """A context keeps freed ensembles' device memory for the next ensemble of
    the same shape: ensembles drawn into reused memory (with and without the
    double copy, the d-loop generator too) equal the oracle's, and ensembles
    of other shapes still come out right beside them."""
    c = wln.Context(0)
    try:
        for _ in range(2):
            for seed in (3, 4, 5):
                ens = c.gen_loops(seed, 96, 256, keep_fp64=True)
                f32, f64 = c.loops_copy(ens, f32=True, f64=True)
                ref = oracle.gen_loops(seed, 96, 256)
                assert np.abs(f64 - ref).max() < 1e-13
                assert np.all(np.abs(f32 - ref.astype(np.float32)) <=
                              np.spacing(np.abs(ref.astype(np.float32))))
                ens.free()
            a = c.gen_loops(6, 64, 128)          # float only: another shape
            b = c.gen_dloops(7, 96, 256)         # the float shape of the freed ones
            fa, _ = c.loops_copy(a)
            fb, _ = c.loops_copy(b)
            assert np.all(np.abs(fa - oracle.gen_loops(6, 64, 128).astype(np.float32)) <= 1e-6)
            assert np.all(np.abs(fb - oracle.gen_dloops(7, 96, 256).astype(np.float32)) <= 1e-6)
            a.free()
            b.free()
    finally:
        c.close()


@pytest.mark.parametrize("n_loops,ppl", [(40, 4), (96, 64), (33, 512), (32, 16384)])
def test_generated_dloops_match_oracle(ctx, n_loops, ppl):
    ens = ctx.gen_dloops(8, n_loops, ppl, keep_fp64=True, loop0=5)
    f32, f64 = ctx.loops_copy(ens, f32=True, f64=True)
    ref = oracle.gen_dloops(8, n_loops, ppl, loop0=5)
    assert np.abs(f64 - ref).max() < 1e-13
    ref32 = ref.astype(np.float32)
    diff = f32 != ref32
    assert diff.mean() < 1e-4
    if diff.any():
        ulp = np.spacing(np.abs(ref32[diff]))
        assert np.all(np.abs(f32[diff] - ref32[diff]) <= ulp)
    ens.free()


CASES = [
    # (n_loops, ppl, G, profile, rho, T)
    (96, 64, 3, I.Profile(0, F=10.0, lam=1.0), I.lin_grid(0.0, 5.0, 7), I.log_grid(0.01, 10.0, 5)),
    (96, 128, 4, I.Profile(0, F=50.0, lam=1.0), I.lin_grid(0.0, 8.0, 9), I.log_grid(1e-3, 20.0, 4)),
    (72, 256, 8, I.Profile(0, F=100.0, lam=0.1), I.lin_grid(0.0, 5.0, 5), I.log_grid(0.01, 10.0, 3)),
    (64, 256, 2, I.Profile(0, F=1.0, lam=1.0), I.lin_grid(0.0, 8.0, 3), I.log_grid(1e-3, 20.0, 6)),
    (64, 64, 4, I.Profile(1, B=1.0), np.zeros(1), I.log_grid(0.01, 10.0, 6)),
    (64, 64, 4, I.Profile(1, B=5.0), np.array([0.0, 2.0]), I.log_grid(0.01, 10.0, 3)),
    (32, 16384, 2, I.Profile(0, F=1.0, lam=1.0), I.lin_grid(0.0, 5.0, 4), I.log_grid(0.01, 10.0, 2)),
    (40, 8, 5, I.Profile(0, F=10.0, lam=0.5), I.lin_grid(0.0, 2.0, 6), I.log_grid(0.1, 4.0, 3)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_wilson_group_sums_match_oracle(ctx, case, prec, tol):
    n_loops, ppl, G, prof, rho, T = CASES[case]
    y32, ens = _ensemble_from_oracle(ctx, 11 + case, n_loops, ppl)
    gpu = ctx.wilson_avg(ens, [prof], [rho], [T], G, prec=prec, where="host")
    ref = oracle.group_sums(y32.astype(np.float64), prof, rho, T, G)
    bars = _bars(y32, prof, rho, T, G, tol, F32_REL if prec == "fp32" else F64_REL)
    _compare(gpu, ref, n_loops // G, bars, what=f"{prec} case {case}")
    ens.free()


def test_zero_flux_is_exactly_one(ctx):
    y32, ens = _ensemble_from_oracle(ctx, 5, 64, 64)
    for prec in ("fp64", "fp32", "fp32_naive"):
        S = ctx.wilson_avg(ens, [I.Profile(0, F=0.0, lam=1.0)], [I.lin_grid(0, 3, 5)],
                           [I.log_grid(0.1, 4, 3)], 4, prec=prec, where="host")
        assert np.all(S == 0.0), prec


def test_batch_equals_single_profile_calls_bitwise(ctx):
    y32, ens = _ensemble_from_oracle(ctx, 6, 64, 64)
    profs = [I.Profile(0, F=3.0, lam=0.5), I.Profile(1, B=0.7), I.Profile(0, F=30.0, lam=2.0)]
    rhos = [I.lin_grid(0, 2, 5), np.zeros(1), I.lin_grid(0, 9, 11)]
    Ts = [I.log_grid(0.01, 1, 3), I.log_grid(0.1, 5, 7), I.log_grid(1, 2, 2)]
    for prec in ("fp32", "fp64"):
        batch = ctx.wilson_avg(ens, profs, rhos, Ts, 4, prec=prec, where="host")
        parts, off = [], 0
        for p, r, t in zip(profs, rhos, Ts):
            single = ctx.wilson_avg(ens, [p], [r], [t], 4, prec=prec, where="host")
            n = len(r) * len(t)
            assert np.array_equal(batch[off:off + n], single), prec
            off += n


def test_repeated_runs_are_bitwise_identical(ctx):
    ens = ctx.gen_loops(3, 256, 256)
    args = ([I.Profile(0, F=10.0, lam=1.0)], [I.lin_grid(0, 5, 16)], [I.log_grid(0.01, 10, 16)], 8)
    a = ctx.wilson_avg(ens, *args, prec="fp32", where="host")
    b = ctx.wilson_avg(ens, *args, prec="fp32", where="host")
    assert np.array_equal(a, b)


def test_device_and_host_outputs_agree(ctx):
    ens = ctx.gen_loops(4, 64, 128)
    args = ([I.Profile(0, F=10.0, lam=1.0)], [I.lin_grid(0, 5, 6)], [I.log_grid(0.01, 10, 4)], 2)
    h = ctx.wilson_avg(ens, *args, prec="fp32", where="host")
    d = ctx.wilson_avg(ens, *args, prec="fp32", where="device")
    torch.cuda.synchronize()
    assert np.array_equal(h, d.cpu().numpy())


def test_statistics_match_oracle(ctx):
    rng = np.random.default_rng(1)
    n_points, G, lpg = 300, 16, 10
    S = rng.normal(size=(n_points, G, 5)) * 3.0
    r = ctx.jackknife(S, G, lpg, 1, jk_var=True, cov=True, where="host")
    m, e = ost.mean_sem(S, lpg, 1)
    assert np.allclose(r["mean"], m, rtol=1e-13, atol=0)
    assert np.allclose(r["sem"], e, rtol=1e-12, atol=0)
    assert np.allclose(r["jk_var"], ost.jackknife_var(S, lpg, 1), rtol=1e-12)
    assert np.allclose(r["cov"], ost.covariance(S, lpg, 1), rtol=1e-12, atol=1e-16)
    ls = ctx.loop_sem(S, G, G * lpg, 0, 3, where="host")
    assert np.allclose(ls, ost.loop_sem(S, G * lpg, 0, 3), rtol=1e-10, equal_nan=True)
    # device inputs and outputs
    Sd = torch.from_numpy(S).cuda()
    rd = ctx.jackknife(Sd, G, lpg, 1, cov=True)
    torch.cuda.synchronize()
    assert np.allclose(rd["cov"].cpu().numpy(), r["cov"], rtol=1e-14, atol=0)


@pytest.mark.parametrize("n_points", [1, 63, 64, 65, 300])
def test_packed_covariance_is_the_upper_triangle(ctx, n_points):
    """wln_jackknife_packed: the upper triangle of the full covariance, row by
    row, bit for bit (tile edges at 64 points, a ragged last tile), from host
    and device inputs into host and device outputs; mean, SEM and jackknife
    variance as the full call's."""
    rng = np.random.default_rng(n_points)
    G, lpg = 16, 10
    S = rng.normal(size=(n_points, G, 5)) * 3.0
    full = ctx.jackknife(S, G, lpg, 1, jk_var=True, cov=True, where="host")
    pk = ctx.jackknife(S, G, lpg, 1, jk_var=True, cov="packed", where="host")
    iu = np.triu_indices(n_points)
    assert pk["cov"].shape == (n_points * (n_points + 1) // 2,)
    assert np.array_equal(pk["cov"], full["cov"][iu])
    for k in ("mean", "sem", "jk_var"):
        assert np.array_equal(pk[k], full[k])
    assert np.allclose(pk["cov"], ost.covariance(S, lpg, 1)[iu], rtol=1e-12, atol=1e-16)
    Sd = torch.from_numpy(S).cuda()
    pd = ctx.jackknife(Sd, G, lpg, 1, cov="packed")
    torch.cuda.synchronize()
    assert np.array_equal(pd["cov"].cpu().numpy(), pk["cov"])


@pytest.mark.parametrize("spinor", [True, False])
def test_effective_action_matches_oracle(ctx, spinor):
    profs = [I.Profile(0, F=10.0, lam=1.0), I.Profile(0, F=2.0, lam=0.5), I.Profile(1, B=0.5)]
    rhos = [I.lin_grid(0, 5, 16), I.lin_grid(0, 2.5, 7), I.lin_grid(0, 1, 2)]
    Ts = [I.log_grid(0.01, 10, 16), I.log_grid(0.02, 5, 9), I.log_grid(0.1, 1, 1)]
    G, lpg = 8, 20
    n = sum(len(a) * len(b) for a, b in zip(rhos, Ts))
    rng = np.random.default_rng(2)
    S = rng.normal(size=(n, G, 5))
    gg, ms = ctx.effective_action(profs, rhos, Ts, S, G, lpg, spinor=spinor, where="host")
    off = 0
    for q, (p, r, t) in enumerate(zip(profs, rhos, Ts)):
        m = len(r) * len(t)
        ref = ost.effective_action_groups(S[off:off + m], lpg, p, r, t, spinor=spinor)
        assert np.allclose(gg[q], ref, rtol=1e-12, atol=1e-300)
        assert ms[q, 0] == pytest.approx(ref.mean(), rel=1e-12, abs=1e-300)
        off += m


def test_invalid_arguments_raise(ctx):
    with pytest.raises(wln.WlnError):
        ctx.gen_loops(1, 10, 100)                         # ppl not a power of two
    ens = ctx.gen_loops(1, 64, 64)
    with pytest.raises(wln.WlnError):
        ctx.wilson_avg(ens, [I.Profile(0, F=1.0, lam=1.0)], [[0.0]], [[1.0]], 5)   # 5 does not divide 64
    with pytest.raises(wln.WlnError):
        ctx.wilson_avg(ens, [I.Profile(0, F=1.0, lam=0.0)], [[0.0]], [[1.0]], 4)   # lambda = 0
    with pytest.raises(wln.WlnError):
        ctx.wilson_avg(ens, [I.Profile(0, F=1.0, lam=1.0)], [[0.0]], [[-1.0]], 4)  # T < 0
    xy = np.zeros((32, 2, 8), np.float32)
    with pytest.raises(wln.WlnError):
        ctx.ensemble_from_host(xy)                        # zero-length segments
    # the context is still usable
    ctx.wilson_avg(ens, [I.Profile(0, F=1.0, lam=1.0)], [[0.0]], [[1.0]], 4, where="host")


# Every launch shape the library instantiates for the float paths, as the
# autotuner (and wln_set_tuning) can select them: (radii per lane, warps per
# CTA) x float4 rows per staged chunk x chunks in flight.
SHAPES = [(P, w, r, st) for (P, w) in ((2, 8), (4, 4), (4, 8), (8, 8))
          for r in (16, 32, 64) for st in (2, 3, 4)]


def _float_cosh_overflows(y32, prof, rho, T, G):
    """[n_points][G]: whether some loop of the group has a spin whose float
    cosh overflows (|spin| > 88.7)."""
    y = y32.astype(np.float64)
    out = np.zeros((len(T) * len(rho), G), bool)
    for b, t in enumerate(T):
        for a, r in enumerate(rho):
            _, sp = oracle.phase_spin(y, prof, r, t)
            out[b * len(rho) + a] = (np.abs(sp) > 88.0).reshape(G, -1).any(axis=1)
    return out


def _naive_rel(ppl):
    # The naive flavour sums ppl/8 partials of 8 terms without compensation
    # (worst case (ppl/8) float ulps, 2^-24 each, of the summed magnitudes) on
    # top of the per-term rounding of the compensated bar.
    return F32_REL + (ppl / 8) * 2.0 ** -24


@pytest.mark.parametrize("case", [0, 1, 2])
def test_every_launch_shape_matches_oracle(ctx, case):
    """All 36 float shapes (with the low-angle forms on) against the oracle at
    the parity bar, FP32 compensated; FP32 naive on the four (radii, warps)
    shapes.  Warps per CTA, rows per chunk and stages change how the work is
    scheduled, not the arithmetic of a radius, so at fixed radii per lane the
    sums are also bitwise equal across them."""
    n_loops, ppl, G, prof, rho, T = CASES[case]
    y32, ens = _ensemble_from_oracle(ctx, 11 + case, n_loops, ppl)
    ref = oracle.group_sums(y32.astype(np.float64), prof, rho, T, G)
    bars = _bars(y32, prof, rho, T, G, 1e-6, F32_REL)
    nbars = _bars(y32, prof, rho, T, G, 1e-6, _naive_rel(ppl))
    ctx.set_low_angle(2)
    by_P = {}
    try:
        for P, w, r, st in SHAPES:
            ctx.set_tuning(P, w, r, st, 0)
            gpu = ctx.wilson_avg(ens, [prof], [rho], [T], G, prec="fp32", where="host")
            _compare(gpu, ref, n_loops // G, bars, what=f"case {case} shape {(P, w, r, st)}")
            if P in by_P:
                assert np.array_equal(gpu, by_P[P]), (P, w, r, st)
            else:
                by_P[P] = gpu
            if r == 32 and st == 3:
                nv = ctx.wilson_avg(ens, [prof], [rho], [T], G, prec="fp32_naive", where="host")
                # the naive flavour's float cosh overflows past a spin of ~88.7:
                # there (and only there) its spinor sums may be infinite
                over = _float_cosh_overflows(y32, prof, rho, T, G)
                bad = ~np.isfinite(nv).all(axis=2)
                assert not np.any(bad & ~over), f"naive case {case}: non-finite below overflow"
                nv = np.where(over[:, :, None], ref, nv)
                _compare(nv, ref, n_loops // G, nbars, what=f"naive case {case} shape {(P, w)}")
    finally:
        ctx.set_tuning()
    ens.free()
