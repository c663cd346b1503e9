"""Parity at the full size of the timed workload, in the launch configuration
the benchmark uses.

The paper workload (10240 loops x 2048 points, flux tubes F = 1, 10, 50 with
lambda = 1, 64 T in [1e-3, 20] x 128 rho in [0, 8], 32 groups) goes through
the same wln_gen_loops and wln_wilson_avg calls as bench.py.  The oracle cannot
redo all 24576 points x 32 groups in test time, so it recomputes sampled
outputs one by one:

  * loops: 48 loops spread over the ensemble regenerated by the oracle from
    their global index (counter-based Philox), double copy within 1e-13;
  * FP32 group sums: 48 seeded (profile, point, group) samples plus the
    corners (largest flux at the smallest radius and longest time, where the
    spin is largest; smallest flux at the largest radius and shortest time),
    each group mean within its R15 bar (max(1e-6, 2^-21 P) scalar,
    max(1, cosh s) max(1e-6, 2^-21 (s + P)) spinor, averaged over the
    group's loops), the oracle working on the same float points; the same
    samples and 24 more from the strongest spins (F = 50, the 8 longest
    times, the 16 smallest radii), where the precision guard works, within
    the plain bar: 1e-6 scalar, 1e-6 max(1, <cosh s>) spinor;
  * FP64 group sums on the benchmark's FP64 subset (one tube, every 8th
    radius, every 4th time), sampled the same way with 1e-12 and 2^-50;
  * properties that hold at any size, on every output: the group means of
    W_scal - 1 = -2 sin^2(phase/2) are finite and lie in [-2, 0], and the
    imaginary part <sin(phase)> vanishes within 8 group standard errors
    (reflection y -> -y maps the loop law to itself and flips the phase).
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
def full():
    from paper_1407_7486_gb300 import build
    build.build()
    stream = torch.cuda.Stream(0)
    ctx = wln.Context(0, stream)
    wl = I.paper()
    with torch.cuda.stream(stream):
        ens = ctx.gen_loops(wl.seed, wl.n_loops, wl.ppl, keep_fp64=True)
        S = ctx.wilson_avg(ens, wl.profiles, wl.rho, wl.T, wl.n_groups, prec="fp32", where="host")
        y32, y64 = ctx.loops_copy(ens, f32=True, f64=True)
    yield ctx, wl, ens, S, y32, y64
    ens.free()
    ctx.close()


def _group_bar(y, prof, rho, T, tol, rel):
    """Mean over the group's loops of the per-loop bars (scalar, spinor)."""
    ph, sp = oracle.phase_spin(y, prof, rho, T)
    P = oracle.phase_abs(y, prof, rho, T)
    with np.errstate(over="ignore", invalid="ignore"):
        es = np.maximum(tol, rel * P)
        ef = np.maximum(1.0, np.cosh(sp)) * np.maximum(tol, rel * (np.abs(sp) + P))
    return es.mean(), ef.mean()


def _check_samples(S, y32, wl, samples, tol, rel, q_sub=None):
    lpg = wl.n_loops // wl.n_groups
    worst = 0.0
    for q, p, g in samples:
        prof = wl.profiles[q] if q_sub is None else q_sub[0]
        rho = wl.rho[q] if q_sub is None else q_sub[1]
        T = wl.T[q] if q_sub is None else q_sub[2]
        base = sum(len(wl.rho[k]) * len(wl.T[k]) for k in range(q)) if q_sub is None else 0
        r, t = rho[p % len(rho)], T[p // len(rho)]
        yg = y32[g * lpg:(g + 1) * lpg].astype(np.float64)
        ref = oracle.group_sums(yg, prof, [r], [t], 1)[0, 0]
        got = S[base + p, g]
        es, ef = _group_bar(yg, prof, r, t, tol, rel)
        for c, bar in ((0, es), (1, ef)):
            if not np.isfinite(ref[c]):
                assert not np.isfinite(got[c]) or np.isnan(ref[c]), (q, p, g, c)
                continue
            err = abs(got[c] - ref[c]) / lpg
            worst = max(worst, err / bar)
            assert err <= bar, (q, p, g, c, err, bar)
    return worst


def test_full_size_loops_match_oracle(full):
    _, wl, _, _, y32, y64 = full
    idx = np.linspace(0, wl.n_loops - 1, 48).astype(int)
    for l in idx:
        want = oracle.gen_loops(wl.seed, 1, wl.ppl, loop0=int(l))[0]
        assert np.abs(y64[l] - want).max() < 1e-13, l
        assert np.mean(y32[l] != want.astype(np.float32)) < 1e-3, l


def test_full_size_fp32_group_sums_sampled(full):
    _, wl, _, S, y32, _ = full
    rng = np.random.default_rng(2024)
    samples = []
    for q in range(len(wl.profiles)):
        n = len(wl.rho[q]) * len(wl.T[q])
        for _ in range(16):
            samples.append((q, int(rng.integers(n)), int(rng.integers(wl.n_groups))))
    last = len(wl.profiles) - 1
    n_rho = len(wl.rho[last])
    samples.append((last, (len(wl.T[last]) - 1) * n_rho + 0, 0))          # F = 50, rho = 0, T = 20
    samples.append((0, n_rho - 1, wl.n_groups - 1))                        # F = 1, rho = 8, T = 1e-3
    worst = _check_samples(S, y32, wl, samples, 1e-6, 2.0 ** -21)
    print("worst sample / bar", worst)
    n_T = len(wl.T[last])
    for _ in range(24):
        it = n_T - 1 - int(rng.integers(8))
        samples.append((last, it * n_rho + int(rng.integers(16)), int(rng.integers(wl.n_groups))))
    lpg = wl.n_loops // wl.n_groups
    worst_s = worst_f = 0.0
    for q, p, g in samples:
        base = sum(len(wl.rho[k]) * len(wl.T[k]) for k in range(q))
        r, t = wl.rho[q][p % len(wl.rho[q])], wl.T[q][p // len(wl.rho[q])]
        yg = y32[g * lpg:(g + 1) * lpg].astype(np.float64)
        ref = oracle.group_sums(yg, wl.profiles[q], [r], [t], 1)[0, 0]
        cosh = np.cosh(oracle.phase_spin(yg, wl.profiles[q], r, t)[1]).sum()
        es = abs(S[base + p, g, 0] - ref[0]) / lpg
        ef = abs(S[base + p, g, 1] - ref[1]) / max(cosh, lpg)
        worst_s, worst_f = max(worst_s, es), max(worst_f, ef)
        assert es <= 1e-6 and ef <= 1e-6, (q, p, g, es, ef)
    print(f"plain bar: scalar {worst_s:.2e}, spinor / <cosh s> {worst_f:.2e}")


def test_full_size_properties_on_every_output(full):
    _, wl, _, S, _, _ = full
    lpg = wl.n_loops // wl.n_groups
    assert S.shape == (wl.n_points, wl.n_groups, wln.WLN_K)
    m_scal = S[:, :, 0] / lpg
    assert np.all(np.isfinite(m_scal))
    assert np.all(m_scal <= 1e-12) and np.all(m_scal >= -2.0 - 1e-12)
    # the imaginary part averages out: |mean sin| within 8 group standard errors
    ms = S[:, :, 2] / lpg
    sem = ms.std(axis=1, ddof=1) / np.sqrt(wl.n_groups)
    assert np.all(np.abs(ms.mean(axis=1)) <= 8 * sem + 1e-12)


def test_full_size_fp64_subset_sampled(full):
    ctx, wl, ens, _, y32, _ = full
    q = 1
    sub = (wl.profiles[q], wl.rho[q][::8], wl.T[q][::4])
    S = ctx.wilson_avg(ens, [sub[0]], [sub[1]], [sub[2]], wl.n_groups, prec="fp64", where="host")
    rng = np.random.default_rng(7)
    n = len(sub[1]) * len(sub[2])
    samples = [(q, int(rng.integers(n)), int(rng.integers(wl.n_groups))) for _ in range(12)]
    worst = _check_samples(S, y32, wl, samples, 1e-12, 2.0 ** -50, q_sub=sub)
    print("fp64 worst sample / bar", worst)
