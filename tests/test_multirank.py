"""Multi-rank path on CPU (gloo, world size 2): each rank computes the group
sums of its own groups from its own loops (the oracle stands in for the GPU,
as a rank's arithmetic is the same whatever the rank), the sums are
all-gathered, and the result equals the single-process computation bitwise;
the jackknife of the gathered sums equals the single-process jackknife."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from oracle import stats as ost
from paper_1407_7486_gb300 import inputs as I
from paper_1407_7486_gb300.shard import gather_group_sums, shard

N_LOOPS, PPL, G, SEED = 64, 32, 8, 9
PROF = I.Profile(0, F=10.0, lam=1.0)
RHO, T = I.lin_grid(0, 4, 5), I.log_grid(0.05, 5, 4)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sh = shard(N_LOOPS, G, world, rank)
    y = oracle.gen_loops(SEED, sh.n_loops, PPL, loop0=sh.loop0, threads=1)
    local = oracle.group_sums(y.astype(np.float32).astype(np.float64), PROF, RHO, T,
                              sh.n_groups, threads=1)
    full = gather_group_sums(torch.from_numpy(local), world)
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), full.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_shard_layout():
    s = [shard(10240, 32, 4, r) for r in range(4)]
    assert [x.loop0 for x in s] == [0, 2560, 5120, 7680]
    assert all(x.n_loops == 2560 and x.n_groups == 8 for x in s)
    with pytest.raises(ValueError):
        shard(100, 10, 3, 0)


def test_two_ranks_gather_equals_one_process(tmp_path):
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    gathered = np.load(tmp_path / "gathered.npy")
    y = oracle.gen_loops(SEED, N_LOOPS, PPL).astype(np.float32).astype(np.float64)
    single = oracle.group_sums(y, PROF, RHO, T, G)
    assert np.array_equal(gathered, single)
    lpg = N_LOOPS // G
    for comp in (0, 1):
        a = ost.mean_sem(gathered, lpg, comp)
        b = ost.mean_sem(single, lpg, comp)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
