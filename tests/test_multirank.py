"""The replica path of bench.py on two gloo ranks (CPU only).

bench.py runs one independent replica per GPU: the step is not sharded, so the
ranks exchange nothing on the data path. The only collectives are the barriers
around the timed region and one MAX all-reduce of its duration. These tests run
those host-side pieces as world-size-2 gloo ranks: the job's time is the
slowest rank's, the value counts the sites of every rank, and the reference arm
runs on rank 0 alone."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench

    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tdist.barrier()
        t = bench.max_over_ranks(times[rank], True, "cpu")
        tdist.barrier()
        q.put((rank, t))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [12.5, 17.25]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert results == [(0, 17.25), (1, 17.25)]


def test_job_value_counts_every_replica():
    import bench

    # 2 ranks x 30,000 sites x 40 steps in 40 x 5 ms
    assert bench.job_value(2, 30000, 40, 40 * 5.0) == pytest.approx(2 * 30000 / 5e-3)
    assert bench.max_over_ranks(3.5, False, "cpu") == 3.5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench

    called = []
    monkeypatch.setattr(bench, "run_reference", lambda args: called.append(args))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    bench.main()
    assert called == [] and capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    bench.main()
    assert len(called) == 1
