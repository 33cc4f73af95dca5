"""The N > 1 path of bench.py: one independent replica of the workload per
rank (no data-path collective), and the whole-job figure formed from all
ranks: the cells of every rank's counted steps over the slowest rank's time.
Checked on a world-size-2 gloo process group on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r counted 100 (r + 1) cell-steps in 10 + r ms
        q.put((rank, bench.replica_throughput(100.0 * (rank + 1), 10.0 + rank, dist, "cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_single_process_figure_is_the_local_one():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(500.0, 20.0, None) == (500.0 / 0.02, 500.0, 20.0)


def test_two_gloo_ranks_sum_cells_over_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        value, cells, ms = results[rank]
        assert cells == 300.0 and ms == 11.0
        assert value == pytest.approx(300.0 / 0.011)
