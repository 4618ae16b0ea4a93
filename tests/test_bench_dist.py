"""Host logic of bench.py for N > 1 ranks, on the CPU with two gloo ranks: the environment
is read as torchrun sets it, the timing is the maximum over ranks, the value counts every
rank's configurations, and the reference arm does its work on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as tdist
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    r, w, loc = bench.dist_env()
    tdist.init_process_group("gloo", rank=r, world_size=w)
    ms = 100.0 + 50.0 * r  # rank 1 is the slow one
    mx = bench.max_over_ranks(ms, w, "cpu")
    val = bench.whole_job_value(4096, 10, w, mx)

    class A:
        steps, warmup = 1, 3
    ref = bench.run_reference(A(), r, w, loc) if r != 0 else "skipped"
    tdist.barrier()
    tdist.destroy_process_group()
    q.put((r, w, loc, mx, val, ref))


def test_two_gloo_ranks():
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
    for r, (rank, world, local, mx, val, ref) in enumerate(res):
        assert (rank, world, local) == (r, 2, r)
        assert mx == 150.0                       # the slowest rank's time
        assert val == pytest.approx(2 * 4096 * 10 / 0.150)
    assert res[1][5] is None                     # reference arm: no work off rank 0


def test_single_rank_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_value(4096, 2, 1, 1000.0) == pytest.approx(8192.0)
