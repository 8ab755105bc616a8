"""The multi-rank path of bench.py (one independent instance per rank, max-over-ranks
timing, whole-job throughput) on two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1407_7220_gb300 import datagen
    ms = [12.5, 20.0][rank]                       # the slower rank sets the job time
    mx = bench.dist_max(ms)
    # replicas: each rank solves its own seeded instance of the same recipe
    X, yb, _ = datagen.make("maxaff", N=64, n=10, seed=datagen.default_seed("maxaff") + rank)
    v = bench.job_value(64 * 63, 10, mx, world)
    q.put((rank, mx, v, float(X.sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_and_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][1] == out[1][1] == 20.0              # max over ranks
    assert out[0][2] == pytest.approx(2 * 64 * 63 * 10 / 0.020)
    assert out[0][3] != out[1][3]                      # distinct instances per rank


def _solver_worker(rank, world, port, q):
    # each rank runs the P-APG iterations of its own seeded instance (the FP64 oracle stands in for
    # the GPU solve on the CPU), times them, and the job takes the slowest rank's time
    import time
    import numpy as np
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import oracle as O
    from paper_1407_7220_gb300 import datagen
    N, K = 48, 15
    X, yb, _ = datagen.make("maxaff", N=N, n=10, seed=datagen.default_seed("maxaff") + rank)
    t0 = time.perf_counter()
    o = O.Solver(X, yb, gamma=1e-2)
    o.iterate(K)
    ms = 1e3 * (time.perf_counter() - t0)
    mx = bench.dist_max(ms)
    v = bench.job_value(N * (N - 1), K, mx, world)
    fits = [None] * world
    dist.all_gather_object(fits, np.asarray(o.y_hat).tolist())
    if rank == 0:
        q.put((mx, v, fits))
    q.put(("ms", rank, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_solve_their_own_instances():
    import numpy as np
    from oracle import oracle as O
    from paper_1407_7220_gb300 import datagen
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_solver_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(3)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    mine = {g[1]: g[2] for g in got if g[0] == "ms"}
    mx, v, fits = next(g for g in got if g[0] != "ms")
    assert mx == max(mine.values())                                     # the slowest rank's time
    assert v == 2 * 48 * 47 * 15 / (mx / 1e3)                            # units of all ranks over it
    for r in range(2):                                                   # each rank's own instance
        X, yb, _ = datagen.make("maxaff", N=48, n=10, seed=datagen.default_seed("maxaff") + r)
        o = O.Solver(X, yb, gamma=1e-2)
        o.iterate(15)
        assert np.array_equal(np.asarray(fits[r]), np.asarray(o.y_hat))
    assert not np.array_equal(np.asarray(fits[0]), np.asarray(fits[1]))
