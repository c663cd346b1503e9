"""Precision and discretisation sweep, through the
C ABI: 8192 loops at ppl = 256, 1024, 4096 and 16384; flux tubes F in {1, 100}
x lambda in {0.1, 1} and constant fields B in {0.1, 1, 5} at rho = 0; FP32
naive, FP32 compensated and FP64 side by side.  Each result is compared with
the FP64 oracle on two groups (512 loops) at a 2 x 2 sub-grid of every profile,
and the errors are printed per precision.  The FP64 and FP32-compensated
paths must meet their parity bars (tests/test_gpu_parity.py); the naive float
path is reported, not bounded.  The constant-field spinor average of all
8192 loops matches the exact finite-N result and, where the discretisation
bias is below the error bar, eBT coth(eBT) (Sec. "Renormalization"), within
five group standard errors.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import stats as ost
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


def _exact_scalar(b, N):
    k = np.arange(1, N)
    return float(np.prod((1.0 + (b / (N * np.tan(np.pi * k / N))) ** 2) ** -0.5))


@pytest.mark.parametrize("ppl", [256, 1024, 4096, 16384])
def test_sweep_precisions_against_oracle(ctx, ppl):
    wl = I.sweep(ppl)
    G = wl.n_groups
    lpg = wl.n_loops // G
    ens = ctx.gen_loops(wl.seed, wl.n_loops, ppl)
    y32, _ = ctx.loops_copy(ens)
    ysub = y32[:2 * lpg]                                  # groups 0 and 1
    report = {}
    for prof, rho, T in zip(wl.profiles, wl.rho, wl.T):
        r_s, t_s = rho[[0, len(rho) // 2]] if len(rho) > 1 else rho, T[[2, len(T) - 3]]
        ref = oracle.group_sums(ysub.astype(np.float64), prof, r_s, t_s, 2)
        for prec, tol, rel in (("fp64", 1e-12, F64_REL), ("fp32", 1e-6, F32_REL),
                               ("fp32_naive", None, None)):
            S = ctx.wilson_avg(ens, [prof], [r_s], [t_s], G, prec=prec, where="host")[:, :2]
            with np.errstate(invalid="ignore", over="ignore"):
                d = np.nan_to_num(np.abs(S - ref) / lpg)
            key = (prof.kind, prof.F, prof.lam, prof.B, prec)
            report[key] = (float(d[:, :, 0].max()), float(d[:, :, 1].max()))
            if tol is not None:
                bars = _bars(ysub, prof, r_s, t_s, 2, tol, rel)
                _compare(S, ref, lpg, bars, what=f"ppl={ppl} {key}")
    for key, (es, ef) in report.items():
        print(f"ppl={ppl} kind={key[0]} F={key[1]} lam={key[2]} B={key[3]} {key[4]:>10s}: "
              f"max |d<W_scal>| {es:.2e}  max |d<W_ferm>| {ef:.2e}")
    ens.free()


def test_constant_field_matches_exact_results(ctx):
    N, n_loops, G = 16384, 8192, 32
    ens = ctx.gen_loops(1, n_loops, N)
    Ts = I.log_grid(0.01, 10.0, 16)
    checked = 0
    for B in (0.1, 1.0, 5.0):
        S = ctx.wilson_avg(ens, [I.Profile(1, B=B)], [np.zeros(1)], [Ts], G, where="host")
        ms, es = ost.mean_sem(S, n_loops // G, 0)
        mf, ef = ost.mean_sem(S, n_loops // G, 1)
        for i, t in enumerate(Ts):
            b = B * t
            if b > 12:      # the spinor average is dominated by a handful of loops
                continue
            ex = _exact_scalar(b, N)
            assert abs(1 + ms[i] - ex) < 5 * es[i] + 1e-12, (B, t)
            assert abs(1 + mf[i] - math.cosh(b) * ex) < 5 * ef[i] + 1e-12, (B, t)
            cont = b / math.tanh(b)
            bias = abs(math.cosh(b) * ex - cont)
            if bias < ef[i]:
                assert abs(1 + mf[i] - cont) < 5 * ef[i] + 1e-12, (B, t)
                checked += 1
    assert checked >= 10
    ens.free()
