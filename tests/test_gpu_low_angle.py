"""The low-angle form of theta changes no bit.

Where every segment of a 32-loop block subtends at most pi/4 at the field
axis, the float walks skip the arctangent's range fold and octant unfolding.
On the grids below the smallest proper times certainly qualify (2 sqrt(T)
|d|max ~ 0.02 against 0.9 lambda; |d|max ~ 0.3 for 512-point loops) and
T = 50 at the axis certainly does not (~4), so a pass mixes both forms; its
results must equal, bit for bit, those of the same pass with the low form
switched off (wln_set_low_angle), in every mode and float precision.
"""
import numpy as np
import pytest

from paper_1407_7486_gb300 import inputs as I
from paper_1407_7486_gb300 import wln

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def setup():
    from paper_1407_7486_gb300 import build
    build.build()
    c = wln.Context(0)
    ens = c.gen_loops(12, 333, 512)          # ragged last block
    yield c, ens
    ens.free()
    c.set_low_angle(True)
    c.close()


PROFS = [I.Profile(0, F=10.0, lam=1.0), I.Profile(0, F=50.0, lam=0.3), I.Profile(1, B=2.0)]
RHOS = [I.lin_grid(0.0, 8.0, 23), I.lin_grid(0.0, 3.0, 9), np.zeros(1)]
TS = [I.log_grid(1e-3, 50.0, 13), I.log_grid(1e-3, 20.0, 7), I.log_grid(0.01, 5.0, 4)]


@pytest.mark.parametrize("prec", ["fp32", "fp32_naive"])
@pytest.mark.parametrize("mode", ["sums", "levels", "nested", "loops"])
def test_low_angle_form_is_bitwise_neutral(setup, prec, mode):
    ctx, ens = setup

    def run():
        if mode == "sums":
            return ctx.wilson_avg(ens, PROFS, RHOS, TS, 9, prec=prec, where="host")
        if mode in ("levels", "nested"):
            return ctx.wilson_levels(ens, PROFS, RHOS, TS, 9, prec=prec, where="host",
                                     nested=mode == "nested")
        return ctx.wilson_loops(ens, PROFS, RHOS, TS, prec=prec, where="host")

    ctx.set_low_angle(True)
    a = run()
    ctx.set_low_angle(False)
    b = run()
    ctx.set_low_angle(True)
    assert np.isfinite(a).any()
    assert np.array_equal(a, b, equal_nan=True)


def test_low_angle_switch_rejects_other_values(setup):
    ctx, _ = setup
    from paper_1407_7486_gb300.wln import load
    assert load().wln_set_low_angle(ctx.handle, 2) != 0
