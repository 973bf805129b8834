"""Multi-GPU path of bench.py (independent replicas): the max-over-ranks step time and the
whole-job value, checked with two gloo ranks on the CPU."""
import os
import socket
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 2.0 if rank == 0 else 5.0           # rank 1 is the slow one
    out = bench.aggregate_ranks(ms, 1000, dist, device="cpu")
    q.put((rank, out))
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
    for r in (0, 1):
        ms, value = res[r]
        assert ms == 5.0
        assert abs(value - 2 * 1000 / 5e-3) < 1e-6


def test_aggregate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(4.0, 100) == (4.0, 100 / 4e-3)
