"""Host logic of the multi-process path, on the CPU.

The realizations of one field are independent chains keyed by their index
(Sec. 2.1), so ranks that each run a disjoint index range and add their
per-site sums must reproduce what one process gets for all indices. Here two
gloo ranks play the two GPUs, with the oracle running each rank's share; the
collectives (temperature broadcast, accumulator all-reduce, max of the
times, sum of the work) are the ones bench.py and replicas.fill_shared_field
use on the GPU.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2212_01317_gb300 import replicas, synth

LB, R = 4, 5


def problem():
    z, m = synth.small_problem(12, 10, 0.4, seed=3)
    return np.where(m != 0, np.nan, z).astype(np.float32), m


def test_partition_covers_every_index_once():
    for R_ in (0, 1, 7, 100, 101):
        for world in (1, 2, 3, 8):
            assert (replicas.check_partition(R_, world) == 1).all()
            sizes = [replicas.shard_realizations(R_, world, r)[1] for r in range(world)]
            assert max(sizes) - min(sizes) <= 1 and sum(sizes) == R_
    with pytest.raises(ValueError):
        replicas.shard_realizations(4, 2, 2)


def test_rank_seeds():
    f = {replicas.rank_seed(11, r, "fields") for r in range(8)}
    assert len(f) == 8 and len({s for _, s in f}) == 8
    assert {replicas.rank_seed(11, r, "realizations") for r in range(8)} == {(11, 0)}


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        values, m = problem()
        H, W = m.shape
        nblk = ((H + LB - 1) // LB) * ((W + LB - 1) // LB)
        T = torch.zeros(nblk, dtype=torch.float32)
        if rank == 0:
            T[:] = torch.from_numpy(oracle.gapfill(values, m, LB, 0, seed=9, n_bisect=8).T)
        replicas.broadcast_temperatures(T, 0)
        first, count = replicas.shard_realizations(R, world, rank)
        res = oracle.gapfill(values, m, LB, count, seed=9, T_blk=T.numpy().astype(np.float64),
                             r0=first)
        acc = torch.from_numpy(np.where(m != 0, res.mean_phi * count, 0.0))
        total = replicas.allreduce_accumulator(acc, count)
        tmax = replicas.max_over_ranks(10.0 + rank)
        work = replicas.sum_over_ranks(res.gap_updates)
        np.savez(os.path.join(out, f"rank{rank}.npz"), acc=acc.numpy(), total=total, tmax=tmax,
                 work=work, T=T.numpy(), first=first, count=count)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_one_process(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(world)]
    values, m = problem()
    T = r[0]["T"].astype(np.float64)
    np.testing.assert_array_equal(r[0]["T"], r[1]["T"])            # broadcast reached rank 1
    assert [int(x["count"]) for x in r] == [3, 2] and int(r[1]["first"]) == 3
    one = oracle.gapfill(values, m, LB, R, seed=9, T_blk=T)
    for x in r:                                                    # every rank holds the sum
        assert int(x["total"]) == R
        assert float(x["tmax"]) == 11.0
        assert int(x["work"]) == one.gap_updates
        gap = m != 0
        np.testing.assert_allclose(x["acc"][gap] / R, one.mean_phi[gap], rtol=0, atol=1e-12)
        assert (x["acc"][~gap] == 0).all()
