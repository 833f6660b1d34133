"""The multi-rank path of bench.py on CPU: two gloo ranks reduce their timings
to the maximum and report the whole job's rate (weak scaling, every rank its
own boxes, no collective on the data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [3.0, 5.0][rank]
        m = bench.max_over_ranks(ms, dist, device="cpu")
        out.put((rank, m, bench.whole_job_mlups(1000, 10, world, m / 1e3)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [5.0, 5.0]
    # 2 ranks x 1000 nodes x 10 steps in 5 ms
    assert all(abs(r[2] - 2 * 1000 * 10 / 5e-3 / 1e6) < 1e-9 for r in res)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
