"""GPU checks of failure detection and of the sharded ensemble.

  * The bounded device wait runs out as designed: a kernel waits on a barrier
    nothing completes, the call returns WLN_ETIMEOUT within its limit, and the
    context keeps working afterwards (no fault, no hang).
  * Loops loop0.. generated on their own equal the same loops of the whole
    ensemble bitwise (counter-based Philox), so ranks can hold disjoint group
    slices; the group sums of a slice equal the matching groups of the whole
    ensemble when the work decomposition matches.
"""
import time

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


def test_bounded_wait_times_out_and_context_survives(ctx):
    t0 = time.perf_counter()
    st = ctx.selftest_wait(50)
    dt = time.perf_counter() - t0
    assert st == 4                                        # WLN_ETIMEOUT
    assert dt < 5.0
    ctx.synchronize()                                     # flag was cleared
    ens = ctx.gen_loops(1, 64, 64)
    S = ctx.wilson_avg(ens, [I.Profile(0, F=1.0, lam=1.0)], [[0.5]], [[1.0]], 2, where="host")
    assert np.all(np.isfinite(S))


def test_loop_slices_equal_whole_ensemble(ctx):
    whole = ctx.gen_loops(3, 256, 128)
    a, _ = ctx.loops_copy(whole)
    for loop0, n in ((0, 64), (64, 96), (160, 96)):
        part = ctx.gen_loops(3, n, 128, loop0=loop0)
        b, _ = ctx.loops_copy(part)
        assert np.array_equal(b, a[loop0:loop0 + n])
        part.free()
    # group sums of the second half equal groups 4..7 of the whole ensemble
    ctx.set_tuning(chain_blocks=1)            # same decomposition on both sides
    args = ([I.Profile(0, F=10.0, lam=1.0)], [I.lin_grid(0, 5, 6)], [I.log_grid(0.01, 10, 5)])
    S_whole = ctx.wilson_avg(whole, *args, 8, where="host")
    half = ctx.gen_loops(3, 128, 128, loop0=128)
    S_half = ctx.wilson_avg(half, *args, 4, where="host")
    ctx.set_tuning()
    assert np.array_equal(S_half, S_whole[:, 4:])
    half.free(); whole.free()
