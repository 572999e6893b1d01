"""Replica parallelism (the only multi-GPU form the method admits: epochs are
independent and the time recursion is sequential) with world size 2 over gloo
on CPU: each rank solves its own epoch, no data-path collective; the job's
time is the maximum over ranks and its throughput the sum of all ranks' time
steps divided by that time, as bench.py computes it under torchrun."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import kf_oracle as ko
from paper_1107_4192_gb300 import synth
from tests.helpers import oracle_dense


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = synth.random_walk_problem(24, 5, 6, seed=100 + rank)   # each rank its own epoch
    F, Q, H, R, P0 = oracle_dense(prob)
    dist.barrier()
    import time
    t0 = time.perf_counter()
    res = ko.kf_fis(F, Q, H, R, prob.Y, prob.x0, P0)
    elapsed = torch.tensor([time.perf_counter() - t0 + 0.01 * rank], dtype=torch.float64)
    dist.barrier()
    dist.all_reduce(elapsed, op=dist.ReduceOp.MAX)
    out[rank] = (float(elapsed.item()), res["x_smooth"].copy())
    dist.destroy_process_group()


def test_two_replicas_over_gloo():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    t_max = [out[r][0] for r in range(world)]
    assert t_max[0] == t_max[1]                     # every rank sees the job's time
    T = 6
    value = world * T / t_max[0]                    # whole-job timesteps/s, weak scaling
    assert value > 0
    for r in range(world):                          # replicas equal single-process solves
        prob = synth.random_walk_problem(24, 5, 6, seed=100 + r)
        F, Q, H, R, P0 = oracle_dense(prob)
        ref = ko.kf_fis(F, Q, H, R, prob.Y, prob.x0, P0)
        assert np.array_equal(out[r][1], ref["x_smooth"])
