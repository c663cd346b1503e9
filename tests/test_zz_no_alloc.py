"""wln_wilson_avg_noalloc: the group sums computed without any allocation.

Callers that cannot allocate device memory (their framework's allocator owns
the device memory, or they must avoid cudaMalloc's implicit synchronisation)
use this entry point; its working memory is a fixed array inside the
library.  These checks call it through the C ABI twice in a row, on
different problems, and compare each result with wln_wilson_avg at the
FP32 parity bar of the other tests (1e-6 on a group mean of W - 1).  The
file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_1407_7486_gb300 import inputs as I
from paper_1407_7486_gb300 import wln

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

TOL = 1e-6   # FP32 bar on a group mean of W - 1 (see test_gpu_parity.py)


@pytest.fixture(scope="module")
def ctx():
    from paper_1407_7486_gb300 import build
    build.build()
    c = wln.Context(0)
    yield c
    c.close()


def _check(a, b, lpg):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    b = b.cpu().numpy() if hasattr(b, "cpu") else b
    scale = np.maximum(1.0, np.abs(b) / lpg)
    assert np.all(np.abs(a - b) / lpg <= TOL * scale)


def test_noalloc_matches_wilson_avg_twice_in_a_row(ctx):
    ens = ctx.gen_loops(21, 640, 256)
    first = ([I.Profile(0, F=10.0, lam=1.0)], [I.lin_grid(0, 5, 13)], [I.log_grid(0.01, 10, 9)], 8)
    second = ([I.Profile(0, F=50.0, lam=0.7), I.Profile(1, B=0.5)],
              [I.lin_grid(0, 3, 6), np.zeros(1)], [I.log_grid(0.1, 5, 4), I.log_grid(0.1, 2, 3)], 5)
    for args, where in ((first, "device"), (second, "host")):
        lpg = ens.n_loops // args[3]
        ref = ctx.wilson_avg(ens, *args, prec="fp32", where=where)
        got = ctx.wilson_avg_noalloc(ens, *args, prec="fp32", where=where)
        torch.cuda.synchronize()
        _check(got, ref, lpg)
    # and the first problem again, after the array held the second one
    ref = ctx.wilson_avg(ens, *first, prec="fp32", where="host")
    got = ctx.wilson_avg_noalloc(ens, *first, prec="fp32", where="host")
    _check(got, ref, ens.n_loops // first[3])
    ens.free()


def test_noalloc_rejects_problems_beyond_its_array(ctx):
    ens = ctx.gen_loops(22, 10240, 64)
    big = ([I.Profile(0, F=10.0, lam=1.0)], [I.lin_grid(0, 8, 512)], [I.log_grid(1e-3, 20, 512)], 32)
    with pytest.raises(wln.WlnError) as e:
        ctx.wilson_avg_noalloc(ens, *big, prec="fp32")
    assert "MiB" in str(e.value)
    ens.free()
