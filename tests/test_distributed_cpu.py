"""Multi-rank path on CPU: two gloo ranks shard a rollout batch, each computes its
systems' parameter-gradient contributions (with the oracle, as a stand-in for the
per-rank GPU kernels), and the rank-ordered sum must equal the single-process
total bitwise on every rank; the shard ranges tile the batch; the slowest-rank
time is the max over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2107_05395_gb300.distributed import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import synth
    from oracle import rollout
    from paper_2107_05395_gb300.distributed import max_over_ranks, shard, sum_in_rank_order

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N, M, T = 12, 9, 5
    x0 = synth.rhs_uniform(seed=1, N=N, M=M)
    y = synth.rhs_uniform(seed=2, N=N, M=M)
    start, count = shard(M, rank, world)
    prob = rollout.diffusion_problem(N, 0.5)
    _, _, dp = rollout.adjoint(prob, x0[:, start:start + count], y[:, start:start + count], T, M_total=M)
    mine = torch.tensor([float(np.sum(dp))], dtype=torch.float64)
    total = sum_in_rank_order(mine)
    slowest = max_over_ranks(float(rank + 1))
    out[rank] = (float(total.item()), slowest, start, count)
    dist.destroy_process_group()


def test_shard_ranges_tile_the_batch():
    for M in (0, 1, 7, 65536, 1 << 20):
        for world in (1, 2, 3, 8):
            ranges = [shard(M, r, world) for r in range(world)]
            assert ranges[0][0] == 0
            for (s0, c0), (s1, _) in zip(ranges, ranges[1:]):
                assert s0 + c0 == s1
            assert sum(c for _, c in ranges) == M
            assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1
    with pytest.raises(ValueError):
        shard(10, 2, 2)


def test_two_gloo_ranks_sum_the_parameter_gradient_in_rank_order():
    import synth
    from oracle import rollout

    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    N, M, T = 12, 9, 5
    parts = []
    for r in range(world):
        s, c = shard(M, r, world)
        _, _, dp = rollout.adjoint(rollout.diffusion_problem(N, 0.5),
                                   synth.rhs_uniform(seed=1, N=N, M=M)[:, s:s + c],
                                   synth.rhs_uniform(seed=2, N=N, M=M)[:, s:s + c], T, M_total=M)
        parts.append(float(np.sum(dp)))
    expect = parts[0] + parts[1]
    totals = {out[r][0] for r in range(world)}
    assert totals == {expect}, (totals, expect)
    assert all(out[r][1] == float(world) for r in range(world))
    _, _, dp_all = rollout.adjoint(rollout.diffusion_problem(N, 0.5), synth.rhs_uniform(seed=1, N=N, M=M),
                                   synth.rhs_uniform(seed=2, N=N, M=M), T)
    assert abs(expect - float(np.sum(dp_all))) <= 1e-14 * abs(expect)
