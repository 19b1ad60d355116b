"""The multi-rank path of bench.py on CPU: two gloo ranks, each reporting its
own time; both must see the slowest rank's times (no GPU)."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    dist.barrier()
    got = bench.slowest_rank(dist, "cpu", 10.0 + 5.0 * rank, 100.0 - rank)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got))


def test_slowest_rank_gloo_world_size_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == (15.0, 100.0)


def test_slowest_rank_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank(None, "cpu", 3.0, 4.0) == (3.0, 4.0)
