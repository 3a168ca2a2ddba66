"""The multi-rank path of bench.py on CPU: two gloo ranks (world size 2) run
the barrier and the max-over-ranks timing reduction, and the reference arm
runs on rank 0 only.  Every rank of a GPU run is an independent replica, so
no other collective exists."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    w, r, local = bench.dist_setup()
    bench.barrier(w)
    m = bench.max_over_ranks(w, 1.5 * (rank + 1))
    total = bench.aggregate_throughput(w, steps=10, pairs=1e6, ms_max=m)
    q.put((rank, w, m, total, dist.get_backend()))
    dist.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, m, total, backend in out:
        assert w == 2 and backend == "gloo"
        assert m == 3.0                                   # max over ranks
        assert total == pytest.approx(2 * 10 * 1e6 / 3e-3)  # whole-job throughput


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup = 2, 1
    assert bench.run_reference(A, 2, 1) is None
    res = bench.run_reference(A, 2, 0)
    assert res["impl"] == "reference" and res["value"] > 0 and res["n_gpus"] == 2
    assert res["e2e"]["h2d_bytes_per_step"] == 0 and res["cpu_baseline"]["kind"] == "oracle"
