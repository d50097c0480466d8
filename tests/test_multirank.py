"""The N > 1 path of bench.py on CPU: world_size 2 over gloo.

Ranks are independent replicas (each its own suspension, or its own shard of
the ensemble), so the only cross-rank step is the final reduction: the
slowest rank's time per step and the sum of the units all ranks processed.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, local = bench.dist_setup()
        # rank r: 1.5 + r ms per step, 1000 * (r + 1) pairs
        ms, units = bench.aggregate(1.5 + r, 1000 * (r + 1), w, "cpu")
        q.put((r, w, local, ms, units, bench.rank_seed(r), bench.ensemble_shard(10, w, r)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_max_time_and_sum_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, ws, local, ms, units, seed, shard) in enumerate(out):
        assert (rank, ws, local) == (r, 2, r)
        assert ms == pytest.approx(2.5)           # the slower rank
        assert units == pytest.approx(3000.0)     # both ranks' pairs
    # replicas: different workloads per rank, the ensemble split without overlap
    assert out[0][5] != out[1][5]
    assert sorted(out[0][6] + out[1][6]) == list(range(10)) and not set(out[0][6]) & set(out[1][6])


def test_one_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(3.0, 7.0, 1, "cpu") == (3.0, 7.0)
    assert bench.ensemble_shard(5, 1, 0) == [0, 1, 2, 3, 4]
