"""The C ABI driven from plain C (tests/c_api_example.c, no Python or
PyTorch in the process): its printed group statistics equal, bit for bit,
those of the same calls made through the Python binding."""
import subprocess

import numpy as np
import pytest

from paper_1407_7486_gb300 import inputs as I
from paper_1407_7486_gb300 import wln

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def test_c_program_matches_python_binding(tmp_path):
    from test_abi import _build_c_example
    exe = _build_c_example(tmp_path)
    out = subprocess.run([exe, "0"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    rows = np.array([[float(v) for v in line.split()] for line in out.stdout.strip().splitlines()])
    assert rows.shape == (12, 6)
    ctx = wln.Context(0)
    ens = ctx.gen_loops(1, 1024, 256)
    prof = I.Profile(I.PROFILE_FLUX_TUBE, F=10.0, lam=1.0)
    rho, T = np.array([0.0, 1.0, 2.0, 3.0]), np.array([0.1, 1.0, 10.0])
    S = ctx.wilson_avg(ens, [prof], [rho], [T], 8, prec="fp32", where="host")
    st = ctx.jackknife(S, 8, 128, 1, jk_var=False, where="host")
    assert np.array_equal(rows[:, 1], np.tile(rho, 3)) and np.array_equal(rows[:, 2], np.repeat(T, 4))
    assert np.array_equal(rows[:, 3], st["mean"])
    assert np.array_equal(rows[:, 4], st["sem"])
    assert np.array_equal(rows[:, 5], S[:, 0, 0])
    ens.free()
    ctx.close()
