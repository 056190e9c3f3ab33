"""The benchmark's multi-rank aggregation on CPU ranks (gloo, world size 2):
a barrier, the max over ranks of the step time and the sum of the work, as
bench.py computes them when launched by torchrun with one replica per GPU."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    r, w, lr = bench.dist_env()
    bench.dist_init(w, "gloo")
    bench.barrier(w)
    mx = bench.reduce_scalar(100.0 + 7 * r, w, "max", "cpu")
    sm = bench.reduce_scalar(1000 * (r + 1), w, "sum", "cpu")
    bench.barrier(w)
    q.put((r, w, lr, mx, sm))
    dist.destroy_process_group()


def test_rank_aggregation_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert all(x[3] == 107.0 for x in res)   # slowest rank's time
    assert all(x[4] == 3000.0 for x in res)  # work of both replicas


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_scalar(3.5, 1, "max", "cpu") == 3.5
    bench.barrier(1)
