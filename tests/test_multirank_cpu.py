"""The N > 1 host path of bench.py on CPU: two gloo ranks (no GPU).

Each rank maps its own problem (same shapes, different seeds: independent
problems, weak scaling, no collective on the data path); the only
collectives are the timing barrier and the max over ranks of the step time.
"""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    import lfgen
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        specs = bench.rank_specs(lfgen.config_specs("tiny"), rank)
        H = lfgen.generate(specs[0])
        step_ms = 2.0 + rank          # rank 1 is the slower one
        t = bench._max_over_ranks(step_ms, world)
        bench._barrier(world)
        val = bench.aggregate_gbs(2 * H.numel() * 4, t, world)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as fh:
            fh.write(f"{t} {val} {specs[0].seed} {float(H.sum())} {H.numel()}\n")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    rows = [open(tmp_path / f"r{r}.txt").read().split() for r in range(world)]
    t0, v0, seed0, sum0, n0 = rows[0]
    t1, v1, seed1, sum1, n1 = rows[1]
    assert float(t0) == float(t1) == 3.0          # both see the slowest rank's time
    assert float(v0) == float(v1)
    nbytes = 2 * int(n0) * 4
    assert abs(float(v0) - world * nbytes / 3e-3 / 1e9) < 1e-9
    assert int(n0) == int(n1)                     # same shapes ...
    assert seed0 != seed1 and sum0 != sum1        # ... independent problems


def _strong_worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import lfgen
    import paper_2003_09133_gb300 as lf
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        s = lfgen.config_specs("highres")[0]
        plan = lf.Plan(s.Nx, s.Ny, list(s.Ks), list(s.Kt), torch.float32)
        z0, z1 = plan.partition(world, rank)
        part = plan.depth_offset(z1) - plan.depth_offset(z0)
        sub = plan.sub_plan(z0, z1) if z1 > z0 else None
        t = torch.tensor([float(part)], dtype=torch.float64)
        dist.all_reduce(t)                      # the ranks' parts add up to the array
        with open(os.path.join(out_dir, f"s{rank}.txt"), "w") as fh:
            fh.write(f"{z0} {z1} {part} {sub.elems if sub else 0} {int(t.item())} {plan.elems}\n")
    finally:
        dist.destroy_process_group()


def test_strong_scaling_partition_two_gloo_ranks(tmp_path):
    """--scaling strong: the ranks split the depths of one array with
    lfbp_plan_partition; the parts are contiguous, cover every depth once,
    hold about equal shares, and their sub-plans are the matching slices."""
    world = 3
    port = _free_port()
    mp.start_processes(_strong_worker, args=(world, port, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    rows = [[int(x) for x in open(tmp_path / f"s{r}.txt").read().split()] for r in range(world)]
    assert rows[0][0] == 0 and rows[-1][1] == 41
    for a, b in zip(rows, rows[1:]):
        assert a[1] == b[0]
    total = rows[0][5]
    for z0, z1, part, sub_elems, summed, elems in rows:
        assert sub_elems == part and summed == total == elems
        assert abs(part - total / world) < 0.1 * total     # about a third each
