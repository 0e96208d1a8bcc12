"""CPU checks of the multi-rank host logic (paper_2509_25110_gb300.shard) with
two gloo ranks: every rank draws its own sources, the timed region's time is
the maximum over ranks, and the rate counts all ranks' spectra."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2509_25110_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = shard.rank_params(8, rank)
        shard.barrier()
        ms = shard.max_over_ranks(10.0 + 5.0 * rank)
        out[rank] = (ms, shard.job_rate(world, 8, 100, ms), float(p.r_s[0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    (ms0, r0, rs0), (ms1, r1, rs1) = out[0], out[1]
    assert ms0 == ms1 == 15.0                       # the slowest rank's time
    assert r0 == r1 == pytest.approx(2 * 8 * 100 / 15e-3)
    assert rs0 != rs1                               # different sources per rank
    assert rs0 == float(synth.model_params(8, seed=0).r_s[0])  # rank 0 = the single-GPU batch


def test_single_process_without_group():
    assert shard.max_over_ranks(3.5) == 3.5
    assert shard.job_rate(1, 256, 10, 2.0) == pytest.approx(256 * 10 / 2e-3)
    a, b = shard.rank_params(4, 0), shard.rank_params(4, 1)
    assert not np.allclose(a.tau_star, b.tau_star)
