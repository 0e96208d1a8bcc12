"""CPU checks of the multi-rank host logic (paper_2509_25110_gb300.shard) with
two gloo ranks: every rank draws its own sources, the timed region's time is
the maximum over ranks, and the rate counts all ranks' spectra.  And the
other way the path shards: over k.  Eq. (1) is a sum over k nodes, so ranks
that each sum their share of the k nodes (with the full grid's weights) and
add the partial C_l reproduce the single-rank C_l of the FP64 oracle."""
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


def _kworker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        k = synth.log_grid(1e-4, 0.3, 40)
        tau = synth.uniform_grid(200.0, 14000.0, 120)
        p = synth.model_params(3, seed=5)
        S, P = synth.sources(k, tau, p), synth.primordial(k, p)
        delta, _ = oracle.los_cl(k, tau, 14000.0, 2, 200, S, P, want_cl=False)
        wk = oracle.lnk_weights(k)
        mine = np.array_split(np.arange(k.size), world)[rank]  # this rank's k nodes
        part = oracle.cl_from_delta(k[mine], delta[:, mine], P[:, mine], wk=wk[mine])
        t = torch.as_tensor(part)
        dist.all_reduce(t)
        out[rank] = t.numpy()
    finally:
        dist.destroy_process_group()


def test_k_split_over_two_gloo_ranks_matches_the_oracle():
    import oracle
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_kworker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    k = synth.log_grid(1e-4, 0.3, 40)
    tau = synth.uniform_grid(200.0, 14000.0, 120)
    p = synth.model_params(3, seed=5)
    _, ref = oracle.los_cl(k, tau, 14000.0, 2, 200, synth.sources(k, tau, p), synth.primordial(k, p))
    for r in range(world):
        np.testing.assert_allclose(out[r], ref, rtol=1e-12, atol=0)


def test_single_process_without_group():
    assert shard.max_over_ranks(3.5) == 3.5
    assert shard.job_rate(1, 256, 10, 2.0) == pytest.approx(256 * 10 / 2e-3)
    a, b = shard.rank_params(4, 0), shard.rank_params(4, 1)
    assert not np.allclose(a.tau_star, b.tau_star)
