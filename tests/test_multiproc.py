"""Multi-rank path of the bench on CPU: two gloo ranks, world size 2.

Shots are independent (Sec. 7: every noise realisation is decoded on its own),
so ranks shard the shot range and exchange nothing but two scalars for
reporting.  Each rank decodes its shard (with the CPU oracle standing in for
the GPU library); the union of the shards must equal one single-process
decode of all shots, and the reported time must be the max over ranks.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench

L, P, PER_RANK, WORLD = 12, 0.06, 6, 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        import oracle
        shot0, n = bench.shard(rank, PER_RANK)
        N = oracle.sample_errors(L, n, P, seed=0, shot0=shot0)
        C, steps, flags = oracle.decode_batch(N, max_steps=300, shot0=shot0)
        # per-rank "time": the rank index + 1, so the max is known
        tmax = bench.reduce_time_max(float(rank + 1), dist, "cpu")
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), C=C, steps=steps, flags=flags,
                 shot0=shot0, tmax=tmax)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_shots(tmp_path, oracle_mod):
    port = _free_port()
    mp.start_processes(_rank_main, args=(port, str(tmp_path)), nprocs=WORLD, join=True,
                       start_method="spawn")
    parts = [np.load(tmp_path / f"r{r}.npz") for r in range(WORLD)]
    assert [int(p["shot0"]) for p in parts] == [0, PER_RANK]
    assert all(float(p["tmax"]) == float(WORLD) for p in parts)
    N = oracle_mod.sample_errors(L, WORLD * PER_RANK, P, seed=0)
    C, steps, flags = oracle_mod.decode_batch(N, max_steps=300)
    np.testing.assert_array_equal(np.concatenate([p["C"] for p in parts]), C)
    np.testing.assert_array_equal(np.concatenate([p["steps"] for p in parts]), steps)
    np.testing.assert_array_equal(np.concatenate([p["flags"] for p in parts]), flags)


def test_shard_ranges_tile_the_job():
    seen = []
    for r in range(4):
        s0, n = bench.shard(r, 25)
        seen.extend(range(s0, s0 + n))
    assert seen == list(range(100))
    assert bench.reduce_time_max(3.5) == 3.5


def test_executed_site_updates_leave_out_exhausted_shots():
    # shots that ran out of the budget report it as their step count but may
    # have been stopped early in a periodic orbit: their steps are not counted
    steps = np.array([10, 4096, 7, 4096])
    flags = np.array([0, 2, 1, 2])
    assert bench.executed_site_updates(steps, flags, 8) == (10 + 7) * 64
    assert bench.executed_site_updates(steps, flags, np.array([8, 16, 4, 32])) == 10 * 64 + 7 * 16
