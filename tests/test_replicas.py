"""The multi-GPU path is replicas only (one independent system per rank, no
collective on the data path): the host logic that seeds the replicas and
takes the slowest replica's time, run as two gloo ranks on the CPU."""
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


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    import gsrgen

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        base = gsrgen.workloads()["c2"].cfg
        cfg = bench.replica_cfg(gsrgen, base, rank, world)
        slowest = bench.max_over_ranks(torch, dist, 10.0 + rank, world, torch.device("cpu"))
        out[rank] = (cfg.seed, cfg.n_stars, cfg.ncols(), slowest)
    finally:
        dist.destroy_process_group()


def test_two_replicas_on_gloo():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    import gsrgen

    base = gsrgen.workloads()["c2"].cfg
    seeds = {res[r][0] for r in range(world)}
    assert seeds == {base.seed, base.seed + 1000}  # every rank its own system
    assert {res[r][1] for r in range(world)} == {base.n_stars}  # of the same shape
    assert {res[r][2] for r in range(world)} == {base.ncols()}
    assert all(res[r][3] == 11.0 for r in range(world))  # the slowest replica's time, on every rank


def test_single_rank_keeps_the_workload():
    sys.path.insert(0, ROOT)
    import bench
    import gsrgen

    base = gsrgen.workloads()["c2"].cfg
    assert bench.replica_cfg(gsrgen, base, 0, 1) is base
    assert bench.max_over_ranks(torch, dist, 3.5, 1, torch.device("cpu")) == 3.5
