"""The paper's own validation experiments, run through the GPU path.

  * Sec. "Grouping Worldlines", Fig. uncinmean: at B T = 6 single loops do
    not estimate the mean -- W_scal = cos(phase) spreads over [-1, 1] like an
    arcsine law (excess kurtosis near -1.5) -- while the means of groups of
    100 loops are close to Gaussian, which is what makes the group standard
    error a sensible error bar.
  * Sec. "Uncertainties and the Fermion Problem", Fig. smallT: in a constant
    field the worldline integrand e^{-T}/T^3 (<W> - 1 - (BT)^2/3) follows the
    exact result (here the exact finite-N average, so the discretisation
    bias of the N-point loops is not mistaken for noise) within its group
    errors, and those errors are amplified as T -> 0.
"""
import math

import numpy as np
import pytest

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


def _moments(x):
    x = np.asarray(x, np.float64)
    d = x - x.mean()
    s2 = (d * d).mean()
    return (d ** 3).mean() / s2 ** 1.5, (d ** 4).mean() / s2 ** 2 - 3.0


def test_group_means_are_gaussian_where_single_loops_are_not(ctx):
    n_loops, lpg = 20000, 100
    ens = ctx.gen_loops(5, n_loops, 256)
    W = ctx.wilson_loops(ens, [I.Profile(1, B=6.0)], [np.zeros(1)], [np.ones(1)], prec="fp32")
    S, _ = ctx.group_sums_loops(W, n_loops // lpg, where="host")
    w = W.cpu().numpy()[0, :, 0] + 1.0                      # W_scal of every loop
    g = S[0, :, 0] / lpg + 1.0                              # group means
    skew_w, kurt_w = _moments(w)
    skew_g, kurt_g = _moments(g)
    assert kurt_w < -1.0                                    # platykurtic, far from normal
    # 200 group means: standard errors of skewness and excess kurtosis ~0.17, ~0.35
    assert abs(skew_g) < 0.6 and abs(kurt_g) < 1.2, (skew_g, kurt_g)
    ens.free()


def _exact_scal(b, N):
    k = np.arange(1, N)
    return float(np.prod((1.0 + (b / (N * np.tan(np.pi * k / N))) ** 2) ** -0.5))


def test_small_T_integrand_follows_exact_result_with_amplified_errors(ctx):
    n_loops, N, G, B = 10240, 1024, 32, 1.0
    ens = ctx.gen_loops(2, n_loops, N)
    prof = I.Profile(1, B=B)
    T = I.log_grid(0.02, 2.0, 9)
    rho = np.zeros(1)
    S = ctx.wilson_avg(ens, [prof], [rho], [T], G, prec="fp32")
    r = ctx.effective_action_full([prof], [rho], [T], S, G, n_loops // G, spinor=True,
                                  where="host")
    Iw = r["integrand"]                # [T][mean, SEM, LCF] of the integrand (one radius)
    for j, t in enumerate(T):
        b = B * t
        exact_N = math.exp(-t) / t ** 3 * (math.cosh(b) * _exact_scal(b, N) - 1.0 - b * b / 3.0)
        assert abs(Iw[j, 0] - exact_N) < 4.0 * Iw[j, 1], (t, Iw[j], exact_N)
    # the amplification of the uncertainties towards small T
    assert Iw[0, 1] > 30.0 * Iw[-1, 1]
    assert np.all(np.diff(Iw[:, 1]) < 0)
    ens.free()
