"""Multi-GPU host logic on CPU: two gloo ranks run independent replicas of the
workload (no collective on the data path) and combine timings as bench.py does:
max over ranks, aggregate units / max time."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    wl = bench.make_workload("ea_pm_L4_chi16", rank)
    my_time = 1.0 + rank          # a stand-in for the rank's measured time
    units = wl.n_chains           # chains advanced by one sweep on this rank
    t = torch.tensor([my_time])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)])
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    checksum = torch.tensor([float(np.sum(wl.couplings.astype(np.int64) % 9973))])
    gathered = [torch.zeros(1) for _ in range(world)]
    dist.all_gather(gathered, checksum)
    out[rank] = (float(t.item()), float(u.item()), [float(g.item()) for g in gathered])
    dist.destroy_process_group()


def test_two_rank_replicas_aggregate():
    port = 29600 + os.getpid() % 200
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    t0, u0, sums0 = out[0]
    t1, u1, _ = out[1]
    assert t0 == t1 == 2.0                  # max over ranks
    assert u0 == u1 == 4.0                  # 2 chains per rank
    assert sums0[0] != sums0[1]             # each rank draws its own disorder (independent replicas)


def test_tau_from_series_pooled_ar1():
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(1)
    phi, T, pairs = 0.6, 400, 64
    x = np.zeros((T, pairs))
    for t in range(1, T):
        x[t] = phi * x[t - 1] + rng.standard_normal(pairs)
    tau, W = bench.tau_from_series(x)
    assert abs(tau - (1 + phi) / (2 * (1 - phi))) < 0.3
