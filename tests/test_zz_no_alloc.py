"""wln_wilson_avg_noalloc: the group sums computed without any allocation.

Callers that cannot allocate device memory (their framework's allocator owns
the device memory, or they must avoid cudaMalloc's implicit synchronisation)
use this entry point; its working memory is a fixed array inside the
library.  These checks call it through the C ABI:
  * twice in a row, on different problems, and again on the first one after
    the array held the second: each result equals wln_wilson_avg bit for bit
    (the same kernels and the same work decomposition);
  * on a fresh context, before any other Wilson call: the device's free
    memory does not change across the call;
  * after a bounded device wait has run out (the self-test wait): the next
    calls return WLN_OK, so a timeout does not stick to the context;
  * with a problem beyond the array: a clear error naming the size.
The file is collected last so that a run stopping at the first failure has
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

FIRST = ([I.Profile(0, F=10.0, lam=1.0)], [I.lin_grid(0, 5, 13)], [I.log_grid(0.01, 10, 9)], 8)
SECOND = ([I.Profile(0, F=50.0, lam=0.7), I.Profile(1, B=0.5)],
          [I.lin_grid(0, 3, 6), np.zeros(1)], [I.log_grid(0.1, 5, 4), I.log_grid(0.1, 2, 3)], 5)


@pytest.fixture(scope="module")
def ctx():
    from paper_1407_7486_gb300 import build
    build.build()
    c = wln.Context(0)
    yield c
    c.close()


def _np(a):
    return a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)


def test_noalloc_matches_wilson_avg_twice_in_a_row(ctx):
    ens = ctx.gen_loops(21, 640, 256)
    for args, where in ((FIRST, "device"), (SECOND, "host")):
        ref = ctx.wilson_avg(ens, *args, prec="fp32", where=where)
        got = ctx.wilson_avg_noalloc(ens, *args, prec="fp32", where=where)
        torch.cuda.synchronize()
        assert np.array_equal(_np(got), _np(ref))
    # and the first problem again, after the array held the second one
    ref = ctx.wilson_avg(ens, *FIRST, prec="fp64", where="host")
    got = ctx.wilson_avg_noalloc(ens, *FIRST, prec="fp64", where="host")
    assert np.array_equal(got, ref)
    ens.free()


def test_noalloc_allocates_nothing(ctx):
    ens = ctx.gen_loops(23, 320, 128)
    ctx.wilson_avg_noalloc(ens, *FIRST, prec="fp32", where="host")   # array looked up
    fresh = wln.Context(0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    a = fresh.wilson_avg_noalloc(ens, *SECOND, prec="fp32", where="host")
    b = fresh.wilson_avg_noalloc(ens, *FIRST, prec="fp32", where="host")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory moved by {free0 - free1} bytes"
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(b))
    fresh.close()
    ens.free()


def test_noalloc_after_a_timed_out_wait(ctx):
    ens = ctx.gen_loops(24, 320, 128)
    assert ctx.selftest_wait(20) == wln.WLN_ETIMEOUT
    ref = ctx.wilson_avg(ens, *FIRST, prec="fp32", where="host")
    for _ in range(2):
        got = ctx.wilson_avg_noalloc(ens, *FIRST, prec="fp32", where="host")
        assert np.array_equal(got, ref)
    ens.free()


def test_noalloc_rejects_problems_beyond_its_array(ctx):
    ens = ctx.gen_loops(22, 10240, 64)
    big = ([I.Profile(0, F=10.0, lam=1.0)], [I.lin_grid(0, 8, 512)], [I.log_grid(1e-3, 20, 512)], 32)
    with pytest.raises(wln.WlnError) as e:
        ctx.wilson_avg_noalloc(ens, *big, prec="fp32")
    assert "MiB" in str(e.value)
    ens.free()


def test_noalloc_reports_a_full_guard_queue(ctx):
    # The fixed array cannot grow the precision guard's queue.  With every
    # recorded loop recomputed (guard mode "all"), a strong tube on 16 x 16
    # points selects 64 loops per (point, group), 131072 in all, twice the
    # 65536 entries the queue holds: the call returns WLN_ENOMEM instead of
    # leaving loops in float silently, the flag is cleared, and the next call
    # (guard in its normal mode) matches wln_wilson_avg.
    prof = I.Profile(0, F=50.0, lam=1.0)
    args = ([prof], [I.lin_grid(0.0, 1.0, 16)], [I.log_grid(2.0, 20.0, 16)], 8)
    ens = ctx.gen_loops(25, 1024, 256)
    ctx.set_precision_guard("all")
    try:
        with pytest.raises(wln.WlnError) as e:
            ctx.wilson_avg_noalloc(ens, *args, prec="fp32", where="host")
        assert e.value.status == wln.WLN_ENOMEM and "queue" in str(e.value)
    finally:
        ctx.set_precision_guard(True)
    ref = ctx.wilson_avg(ens, *args, prec="fp32", where="host")
    got = ctx.wilson_avg_noalloc(ens, *args, prec="fp32", where="host")
    assert np.array_equal(got, ref)
    ens.free()
