"""Multi-rank path: two gloo ranks on the CPU (world size 2), each tracing its own path-id range
with the oracle, combine their tallies with the sharding helpers that bench.py uses on GPUs; the
result must be the single-process job over the union of the ranges, and the step time the slower
rank's. (The data path has no collective: paths are keyed by id.)"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene():
    import scenegen as sg
    return sg.cfg2_cornell_box(width=16, height=16, grid=16, n_paths=1)


def _worker(rank, world, port, n, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1706_03024_gb300 import shard
        first, count = shard.path_range(n, rank)
        r = oracle.render(_scene(), n_paths=count, path_offset=first, n_threads=1)
        job = shard.combine_tallies(r, count)
        slowest = shard.reduce_scalar(10.0 * (rank + 1), "max")
        total = shard.reduce_scalar(count, "sum")
        if rank == 0:
            out_q.put((job, slowest, total))
    finally:
        dist.destroy_process_group()


def test_path_range_partitions_the_ids():
    from paper_1706_03024_gb300 import shard
    ranges = [shard.path_range(1000, r) for r in range(4)]
    assert ranges == [(0, 1000), (1000, 1000), (2000, 1000), (3000, 1000)]
    with pytest.raises(ValueError):
        shard.path_range(-1, 0)


def test_combine_without_process_group_is_identity():
    from paper_1706_03024_gb300 import shard
    t = {"face": np.arange(6.0), "film": None, "counters": {"paths": 5}}
    out = shard.combine_tallies(t, 5)
    assert np.array_equal(out["face"], t["face"]) and out["film"] is None
    assert out["counters"] == {"paths": 5}
    assert shard.reduce_scalar(3.5, "max") == 3.5


def test_two_gloo_ranks_reproduce_the_whole_job():
    import multiprocessing as mp

    import oracle

    oracle.build()
    n = 1500
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        job, slowest, total = q.get(timeout=180)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    assert slowest == 20.0 and total == 2 * n
    whole = oracle.render(_scene(), n_paths=2 * n, path_offset=0, n_threads=1)
    for key in ("face", "absorbed", "emitted", "film"):
        np.testing.assert_allclose(job[key], whole[key], rtol=1e-12, atol=1e-15, err_msg=key)
    assert job["counters"] == whole["counters"]


def _worker_with_failure(rank, world, port, out_q):
    """Rank 1 fails on the host before the reduction (it exits without joining the collective);
    rank 0 must learn of it as an error from its collective within the group's timeout, not hang."""
    import datetime
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    from paper_1706_03024_gb300 import shard
    if rank == 1:
        os._exit(3)   # the failing rank leaves between steps, nothing in flight
    try:
        shard.reduce_scalar(1.0, "sum")
        out_q.put("no error")
    except Exception as e:   # gloo reports the lost peer (closed connection or timeout)
        out_q.put("error: " + type(e).__name__)


def test_a_failed_rank_is_reported_to_the_others():
    import multiprocessing as mp
    import time

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_with_failure, args=(r, 2, port, q)) for r in range(2)]
    t0 = time.time()
    for p in procs:
        p.start()
    try:
        msg = q.get(timeout=120)
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    assert msg.startswith("error"), msg
    assert time.time() - t0 < 110
    assert procs[1].exitcode == 3
