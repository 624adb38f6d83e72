"""Several GPUs run independent replicas (queries partition with no exchange):
the bench times every rank between barriers and reports all ranks' queries
over the slowest rank's time. The rank aggregation is checked here with two
gloo processes on the CPU."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    slow = bench.max_over_ranks(10.0 + 7.5 * rank, dist, "cpu")      # ms of work on this rank
    dist.barrier()
    out.put((rank, slow, bench.replica_throughput(1000, world, slow / 1e3)))
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_throughput_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, value in res:
        assert slow == 17.5                       # the slower rank's time, on every rank
        assert abs(value - 2 * 1000 / 0.0175) < 1e-6
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
