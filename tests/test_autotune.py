"""CPU checks of the autotuner's search (paper_1407_7486_gb300/autotune.py).

The GPU timing is replaced by an injected timer, and the context by a stand-in
that records the tuning calls, so the search logic runs without a GPU:
  * every candidate is timed once, with its own shape set on the context;
  * the fastest candidate (highest segment rate) is chosen and left set;
  * the cache key names the GPU, the points per loop and the precision, and a
    second call with the cache returns the stored choice without timing;
  * FP64 keeps its fixed shape and times nothing.
The shapes themselves are compared with the oracle on the GPU
(test_gpu_parity.py, test_every_launch_shape_matches_oracle).
"""
import json

import numpy as np
import pytest

from paper_1407_7486_gb300 import autotune
from paper_1407_7486_gb300 import inputs as I


class FakeCtx:
    def __init__(self):
        self.calls = []
        self.current = None

    def set_tuning(self, P=0, warps=0, rows=0, stages=0, chain=0):
        self.current = (P, warps, rows, stages)
        self.calls.append(self.current)


class FakeEns:
    n_loops, ppl = 1024, 256


def _workload():
    return ([I.Profile(0, F=10.0, lam=1.0)], [I.lin_grid(0, 5, 16)], [I.log_grid(0.01, 10, 16)])


def test_search_picks_the_fastest_and_caches(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    ctx = FakeCtx()
    cands = autotune.candidates()
    assert len(cands) == len(set(cands)) == 4 * 3 * 3
    rng = np.random.default_rng(3)
    cost = {c: float(rng.uniform(1.0, 2.0)) for c in cands}
    fastest = (4, 4, 32, 3)
    cost[fastest] = 0.5
    timed = []

    def timer():
        timed.append(ctx.current)
        return cost[ctx.current]

    out = autotune.tune(ctx, FakeEns(), *_workload(), 8, timer=timer, device_name="GPU-X")
    assert sorted(timed) == sorted(cands)                     # each candidate timed once
    assert (out["P"], out["warps"], out["rows"], out["stages"]) == fastest
    assert ctx.current == fastest and out["source"] == "measured"
    assert min(c["ms"] for c in out["candidates"]) == 0.5
    data = json.load(open(autotune.CACHE))
    assert list(data) == ["GPU-X|ppl=256|fp32"]
    # cached: no timing, same choice
    ctx2 = FakeCtx()
    hit = autotune.tune(ctx2, FakeEns(), *_workload(), 8, timer=lambda: pytest.fail("timed"),
                        device_name="GPU-X")
    assert hit["source"] == "cache" and ctx2.current == fastest
    # another GPU or points per loop is another key
    assert autotune._key("GPU-Y", 256, "fp32") not in data
    assert autotune._key("GPU-X", 512, "fp32") not in data


def test_fp64_keeps_its_fixed_shape(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    ctx = FakeCtx()
    out = autotune.tune(ctx, FakeEns(), *_workload(), 8, prec="fp64",
                        timer=lambda: pytest.fail("timed"), device_name="GPU-X")
    assert out["source"] == "fixed for fp64" and ctx.calls == [(0, 0, 0, 0)]


def test_probe_is_a_prefix_of_the_points():
    profs = [I.Profile(0, F=1.0, lam=1.0)] * 3
    rho = [I.lin_grid(0, 5, 10)] * 3
    T = [I.log_grid(0.01, 10, 20)] * 3
    P, R, TT, n = autotune._probe(profs, rho, T, 1024, 256, 1e9, 1e-3)
    assert n == sum(len(r) * len(t) for r, t in zip(R, TT)) and n >= 256
    for t in TT:
        assert np.array_equal(t, T[0][:len(t)])
