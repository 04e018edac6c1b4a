"""The multi-rank path on CPU processes (gloo, world size 2).

Ranks own disjoint shards of the canonical quartets (bra/ket pair key mod
nranks); the only exchange is a sum of the natom x 3 fp64 gradients.  Here
each rank evaluates its shard with the oracle, the shards are summed with a
gloo all-reduce, and the result must equal the unsharded gradient.  The same
processes exercise bench.py's whole-job aggregation (max time, summed units).
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    import oracle
    from paper_2407_16586_gb300 import synth

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = synth.molecule(3, 1, 2)
        g, _, nq = oracle.grad2e(s, tau=1e-12, rank=rank, nranks=world, nthreads=1)
        t = torch.from_numpy(g.copy())
        dist.all_reduce(t)
        ms, units = bench.aggregate_over_ranks(dist, 10.0 * (rank + 1), nq, torch.device("cpu"))
        out[rank] = (t.numpy().copy(), nq, ms, units)
    finally:
        dist.destroy_process_group()


def test_two_rank_shard_sum():
    import oracle
    from paper_2407_16586_gb300 import synth

    oracle.build()
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    s = synth.molecule(3, 1, 2)
    g_all, _, nq_all = oracle.grad2e(s, tau=1e-12, nthreads=1)
    for r in range(world):
        g, nq, ms, units = res[r]
        assert np.abs(g - g_all).max() <= 1e-13 * max(1.0, np.abs(g_all).max())
        assert ms == 20.0                       # max over ranks
        assert units == float(nq_all)           # shards partition the quartets
    assert res[0][1] + res[1][1] == nq_all
    assert res[0][1] > 0 and res[1][1] > 0


def _leaving_worker(rank, world, port, out):
    import datetime
    import time

    import torch
    import torch.distributed as dist
    import oracle
    from paper_2407_16586_gb300 import synth

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    s = synth.molecule(3, 1, 2)
    g, _, _ = oracle.grad2e(s, tau=1e-12, rank=rank, nranks=world, nthreads=1)
    if rank == 1:
        # this rank fails between steps: it leaves without joining the sum
        out[rank] = "left"
        os._exit(3)
    t0 = time.time()
    try:
        dist.all_reduce(torch.from_numpy(g.copy()))
        out[rank] = "completed"
    except Exception as e:  # the survivor's collective ends with an error
        out[rank] = ("error", type(e).__name__, time.time() - t0)
    os._exit(0)


def test_rank_that_leaves_ends_the_others_sum_with_an_error():
    """Failure detection on the host: a rank that exits between steps never
    joins the gradient sum; the surviving rank's all-reduce ends with an
    error within the process group's timeout instead of hanging."""
    import oracle

    oracle.build()
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_leaving_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        for p in procs:
            if p.is_alive():
                p.kill()
        res = dict(out)
        codes = [p.exitcode for p in procs]
    assert res.get(1) == "left" and codes[1] == 3
    assert codes[0] == 0
    assert isinstance(res.get(0), tuple) and res[0][0] == "error", res.get(0)
    assert res[0][2] < 60.0
