"""Multi-rank logic of bench.py on CPU (gloo, world size 2): every rank solves its own geometry (weak scaling,
no collective on the data path); the job's time is the slowest rank's, its work the sum over ranks."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2106_06149_gb300.synth import WORKLOADS, make_problem
    # each rank draws its own geometry exactly as bench.py does (seed offset per rank)
    _, pk, _ = WORKLOADS[0]
    p = make_problem(**{**pk, "seed": pk["seed"] + 1000 * rank})
    ms = 10.0 * (rank + 1)
    units = float(p.n_occ * (rank + 2))
    tot_ms, tot_units = bench.reduce_over_ranks(ms, units, world, "cpu")
    out[rank] = (tot_ms, tot_units, float(p.B.sum()))
    dist.destroy_process_group()


def test_weak_scaling_reduction_two_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 20.0                  # max over ranks
    assert out[0][1] == out[1][1] == 10.0 * 2 + 10.0 * 3   # sum of the ranks' work (n_occ = 10)
    assert out[0][2] != out[1][2]                           # independent geometries
