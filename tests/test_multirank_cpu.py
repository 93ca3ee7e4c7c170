"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks (127.0.0.1)
reduce their times to the slowest rank's and count every rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t = bench.max_over_ranks(1.5 + rank, ws, "cpu")  # rank 1 is the slow one
    v = bench.job_throughput(ws, 10, 320, t)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, v))


def test_two_gloo_ranks_take_the_slowest_time_and_all_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 2.5
        assert v == pytest.approx(2 * 10 * 320 / 2.5)


def test_single_rank_passes_through():
    import bench
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.job_throughput(1, 300, 320, 0.1) == pytest.approx(960000.0)
