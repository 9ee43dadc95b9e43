"""The multi-process timing path of bench.py (barrier + max over ranks) with two gloo ranks
on the CPU.  The benchmark shards nothing on the data path: each rank renders its own
replica; only the timing reduction crosses ranks.  A rank that leaves before the barrier makes
the other fail with an error, not wait."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_init()
    bench.barrier(w)
    m = bench.dist_max(10.0 + rank, w)
    q.put((r, w, m))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_max_and_barrier():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(k, 2, port, q)) for k in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 11.0), (1, 2, 11.0)]


def _worker_leaves(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import time

    import bench
    w, r, local = bench.dist_init(timeout_s=10)
    if rank == 1:
        os._exit(3)  # a rank that dies between steps, before the barrier
    t0 = time.time()
    try:
        bench.barrier(w)
        bench.dist_max(1.0, w)
        q.put(("no error", time.time() - t0))
    except Exception as e:  # noqa: BLE001 -- the failure is the point
        q.put((type(e).__name__, time.time() - t0))


def test_a_rank_that_leaves_fails_the_other_within_the_timeout():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker_leaves, args=(k, 2, port, q)) for k in range(2)]
    for p in ps:
        p.start()
    what, waited = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
    assert what != "no error" and waited < 60
    assert ps[1].exitcode == 3
