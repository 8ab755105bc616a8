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
