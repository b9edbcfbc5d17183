"""The multi-rank path of the benchmark (independent replicas, no collective on the data path):
two gloo ranks on the CPU agree on the slowest rank's time and on the whole-job throughput."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.replica_throughput(100.0 + 50.0 * rank, 10, world, "cpu")))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        total_ms, value = out[r]
        assert total_ms == 150.0
        assert abs(value - 2 * 10 / 0.150) < 1e-9


def test_single_rank_is_plain_throughput():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(200.0, 10, 1) == (200.0, 50.0)
