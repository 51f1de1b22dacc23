"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks each run an
independent replica (no data-path collective), and the whole-job throughput
is all ranks' node updates over the slowest rank's time (max over ranks)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import time

    import bench
    import oracle
    from paper_1603_08221_gb300 import workloads

    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env() == (rank, world, rank)
    p = workloads.preset("heli_argon_320x16", N=6, N_x=24)
    o = oracle.Oracle(p)
    o.init()
    dist.barrier()
    t0 = time.perf_counter()
    o.step(50 + 25 * rank)  # unequal work: the slow rank sets the time
    elapsed = time.perf_counter() - t0
    units = o.N * (o.N_x - 2) * (50 + 25 * rank)
    t = torch.tensor([elapsed], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units], dtype=torch.float64)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    cl = torch.tensor([o.separation()["CL"]], dtype=torch.float64)
    gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, cl)
    if rank == 0:
        val, tmax = bench.aggregate([float(t)], [float(u)])
        out.put((val, tmax, float(u), [float(g) for g in gathered], elapsed))
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_aggregation():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    val, tmax, units, cls, t0 = out.get(timeout=10)
    assert units == 6 * 22 * (50 + 75)
    assert tmax >= t0 > 0
    assert val == pytest.approx(units / tmax)
    # replicas of different lengths give different (finite) states
    assert all(c == c for c in cls) and cls[0] != cls[1]


def test_aggregate_is_units_over_slowest_rank():
    import bench
    v, t = bench.aggregate([1.0, 2.0, 1.5], [10.0, 10.0, 10.0])
    assert t == 2.0 and v == 15.0
