"""The N-rank launch path of bench.py on CPU (gloo, world size 2): every rank
gets its own chain of the same shape (weak scaling, no data-path
collective), and the timing every rank reports is the slowest rank's."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        chain = bench.workload(rank)
        ms = bench.max_over_ranks(100.0 + 7.0 * rank, dist, torch.device("cpu"))
        out[rank] = (chain.seed, sorted(chain.body_sizes), ms, len(bench.subset_sizes(chain, 3)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_weak_scaling_host_path():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] != res[1][0]                      # independent chains (seed 2310 + rank)
    assert res[0][1] == res[1][1]                      # same shape: same work per rank
    assert res[0][3] == res[1][3] == 40 + 780 + 9880   # same CI problem count per rank
    assert res[0][2] == res[1][2] == pytest.approx(107.0)   # every rank reports the slowest rank's time


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(3.5, None, torch.device("cpu")) == 3.5
