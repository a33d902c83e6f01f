"""The benchmark's multi-process path on the CPU: two ranks over gloo.

bench.py runs one process per GPU, each an independent replica of the
lattice; the process group carries only the timing barrier and the
max-reduce of the timed interval, and the whole-job throughput is every
rank's work over the slowest rank's time.  Here two CPU processes join a
gloo group on 127.0.0.1 and exercise exactly that host logic.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist, r, ws, local = bench.dist_setup(None, backend="gloo")
    assert (r, ws, local) == (rank, world, rank)
    bench.barrier(dist)
    ms = bench.max_over_ranks(dist, 10.0 + 5.0 * rank, device="cpu")  # rank 1 is slower
    value = bench.job_throughput(1_000_000, 100, ws, ms)
    out.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slower rank's 15 ms; the job did 2 x 1e8 updates in it
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == pytest.approx(2 * 1e6 * 100 / 15e-3 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    # rank 1 returns before building or running anything
    assert bench.run_reference(None) is None
