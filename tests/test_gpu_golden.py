"""The Wilson pass, both precisions, against the stored oracle case of
tests/golden/oracle_small_case.txt (a value written by the oracle alone), with
the per-loop error bars of the parity tests.  The loops are the oracle's,
rounded to float32 as the GPU stores them."""
import importlib.util
import os

import numpy as np
import pytest

from paper_1407_7486_gb300 import inputs as I
from paper_1407_7486_gb300 import wln
from test_gpu_parity import F32_REL, F64_REL, _bars, _compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _case():
    spec = importlib.util.spec_from_file_location(
        "make_oracle_small_case", os.path.join(GOLDEN, "make_oracle_small_case.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def ctx():
    from paper_1407_7486_gb300 import build
    build.build()
    c = wln.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("prec,tol,rel", [("fp64", 1e-12, F64_REL), ("fp32", 1e-6, F32_REL)])
def test_gpu_matches_stored_oracle_case(ctx, prec, tol, rel):
    m = _case()
    stored = np.loadtxt(os.path.join(GOLDEN, "oracle_small_case.txt"))
    rho, T = np.array(m.RHO), np.array(m.T)
    ref = stored[:, 2:].reshape(len(rho) * len(T), m.G, 5)
    prof = I.Profile(m.PROFILE["kind"], F=m.PROFILE["F"], lam=m.PROFILE["lam"])
    y32 = m.loops().astype(np.float32)
    ens = ctx.ensemble_from_host(y32)
    gpu = ctx.wilson_avg(ens, [prof], [rho], [T], m.G, prec=prec, where="host")
    _compare(gpu, ref, m.N_LOOPS // m.G, _bars(y32, prof, rho, T, m.G, tol, rel),
             what=f"{prec} stored case")
    ens.free()
