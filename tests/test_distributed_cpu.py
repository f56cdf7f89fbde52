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


def _ell_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import synth
    from oracle import matrices, steppers
    from paper_2107_05395_gb300.distributed import batch_mean_in_rank_order, shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N, M, steps = 24, 11, 6
    C = synth.rhs_uniform(seed=3, N=N, M=M, lo=-0.5, hi=0.5)
    start, count = shard(M, rank, world)
    A = steppers.SharedPentaPeriodic(*matrices.ch_matrix_periodic(N, 0.05 * 0.5))
    Cl = C[:, start:start + count]
    ell = []
    for _ in range(steps):
        Cl = steppers.ch_step_periodic(A, Cl, 0.05)
        ell.append(steppers.coarsening_length(Cl))
    series = batch_mean_in_rank_order(torch.tensor(ell, dtype=torch.float64), count, M)
    out[rank] = series.numpy().tolist()
    dist.destroy_process_group()


def test_two_gloo_ranks_average_the_coarsening_length():
    import synth
    from oracle import matrices, steppers

    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_ell_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert out[0] == out[1]  # the same bits on every rank
    N, M, steps = 24, 11, 6
    C = synth.rhs_uniform(seed=3, N=N, M=M, lo=-0.5, hi=0.5)
    A = steppers.SharedPentaPeriodic(*matrices.ch_matrix_periodic(N, 0.05 * 0.5))
    ref = []
    for _ in range(steps):
        C = steppers.ch_step_periodic(A, C, 0.05)
        ref.append(steppers.coarsening_length(C))
    assert np.max(np.abs(np.array(out[0]) - np.array(ref)) / np.array(ref)) <= 1e-14
