"""Host logic of bench.py for N > 1 ranks, on the CPU with two gloo ranks: the environment
is read as torchrun sets it, the timing is the maximum over ranks, the value counts every
rank's configurations, and the reference arm does its work on rank 0 only; and the reference
arm's JSON line (one bounded step of the FP64 oracle) carries the keys of the contract."""
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


def test_reference_arm_line(tmp_path):
    """`bench.py --impl reference` (the FP64 oracle on the host cores, one bounded step) prints
    one JSON line with the arm's metric, unit and workload, its own cpu_baseline and an e2e
    block without host-device copies."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=900, cwd=str(tmp_path))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["value"] > 0 and d["steps"] == 1
    assert d["config"]["workload"] == bench.WORKLOAD and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
