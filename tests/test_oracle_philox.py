"""Pins of the oracle's Philox against independent implementations.

The loop ensemble is drawn from Philox-4x32-10 (Salmon et al., SC'11) with
counter (j, loop, 0, 0) and key (seed_lo, seed_hi).  The oracle writes the
round once for both word widths, so:
  * the 64-bit instance is checked against numpy's own Philox-4x64-10
    bit generator, which pins the round structure, key schedule and word
    permutation;
  * the 32-bit instance is checked against Triton's Philox-4x32-10, run by
    Triton's CPU interpreter, which pins the 32-bit multipliers, Weyl
    constants and the (counter, key) convention used for the loops.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle


def test_philox4x64_matches_numpy_bitgenerator():
    rng = np.random.default_rng(2024)
    for _ in range(20):
        key = rng.integers(0, 2**64, size=2, dtype=np.uint64)
        ctr = rng.integers(0, 2**63, size=4, dtype=np.uint64)
        # numpy's Philox advances the counter by one before each block of four.
        bg = np.random.Philox(counter=ctr, key=key)
        got = bg.random_raw(8).astype(np.uint64)
        c1 = ctr.copy(); c1[0] += np.uint64(1)
        c2 = ctr.copy(); c2[0] += np.uint64(2)
        want = np.concatenate([oracle.philox4x64(c1, key), oracle.philox4x64(c2, key)])
        assert np.array_equal(got, want)


def test_philox_zero_rounds_is_identity_and_rounds_mix():
    ctr = np.array([1, 2, 3, 4], np.uint32)
    key = np.array([5, 6], np.uint32)
    assert np.array_equal(oracle.philox4x32(ctr, key, rounds=0), ctr)
    a = oracle.philox4x32(ctr, key)
    b = oracle.philox4x32(ctr + np.array([1, 0, 0, 0], np.uint32), key)
    # one flipped counter bit changes about half of the 128 output bits
    flips = sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b))
    assert 40 < flips < 88


def test_stream_layout_is_counter_j_loop():
    s = oracle.philox_stream(seed=0xABCDEF0123, n_loops=3, n_calls=5, loop0=7)
    key = np.array([0xABCDEF0123 & 0xFFFFFFFF, 0xABCDEF0123 >> 32], np.uint32)
    for l in range(3):
        for j in range(5):
            assert np.array_equal(s[l, j], oracle.philox4x32(np.array([j, 7 + l, 0, 0], np.uint32), key))


_TRITON_PROBE = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    import triton
    import triton.language as tl

    @triton.jit
    def stream(out_ptr, seed, c0_ptr, c1_ptr, n, BLOCK: tl.constexpr):
        i = tl.arange(0, BLOCK)
        m = i < n
        c0 = tl.load(c0_ptr + i, mask=m)
        c1 = tl.load(c1_ptr + i, mask=m)
        z = c0 * 0
        a, b, c, d = tl.philox(seed, c0, c1, z, z)
        tl.store(out_ptr + 4 * i + 0, a, mask=m)
        tl.store(out_ptr + 4 * i + 1, b, mask=m)
        tl.store(out_ptr + 4 * i + 2, c, mask=m)
        tl.store(out_ptr + 4 * i + 3, d, mask=m)

    seed = int(sys.argv[1])
    j = np.array([int(v) for v in sys.argv[2].split(",")], np.uint32)
    loop = np.array([int(v) for v in sys.argv[3].split(",")], np.uint32)
    n = len(j)
    out = torch.zeros(4 * 64, dtype=torch.int32)
    stream[(1,)](out, seed, torch.from_numpy(j.view(np.int32)), torch.from_numpy(loop.view(np.int32)),
                 n, BLOCK=64)
    print(",".join(str(int(v)) for v in out.numpy().view(np.uint32)[: 4 * n]))
""")


def test_philox4x32_matches_triton_interpreter(tmp_path):
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    probe = tmp_path / "probe.py"
    probe.write_text(_TRITON_PROBE)
    rng = np.random.default_rng(7)
    seed = 0x9E3779B97F4A7C15 >> 1
    j = rng.integers(0, 2**32, size=40, dtype=np.uint64)
    loop = rng.integers(0, 2**32, size=40, dtype=np.uint64)
    j[:4] = [0, 1, 2, 2**32 - 1]
    loop[:4] = [0, 0, 1, 2**31]
    env = dict(os.environ, TRITON_INTERPRET="1")
    res = subprocess.run([sys.executable, str(probe), str(seed), ",".join(map(str, j)),
                          ",".join(map(str, loop))], capture_output=True, text=True, env=env,
                         timeout=600)
    if res.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + res.stderr[-300:])
    got = np.array([int(v) for v in res.stdout.strip().split(",")], np.uint64).reshape(-1, 4)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    for i in range(len(j)):
        want = oracle.philox4x32(np.array([j[i], loop[i], 0, 0], np.uint32), key)
        assert np.array_equal(got[i], want.astype(np.uint64)), i
