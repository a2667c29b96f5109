"""Multi-rank logic of bench.py on CPU (gloo, world size 2): the timing is
the maximum over ranks, the whole-job rate counts every rank's frames
against the slowest rank's time, and the ranks render different frames."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = [2.0, 3.5][rank]
    t_max = bench.reduce_max(t_local, dist, "cpu")
    rate = bench.whole_job_rate(10, world, t_max)
    frames = [bench.frame_index(rank, i, 60) for i in range(10)]
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t_max, rate, frames))


def test_two_rank_timing_and_frames():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, rate, frames in res:
        assert t_max == 3.5                      # the slowest rank's time on every rank
        assert rate == pytest.approx(2 * 10 / 3.5)
    assert not set(res[0][3]) & set(res[1][3])   # disjoint frames


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(1.25, None, "cpu") == 1.25
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0
