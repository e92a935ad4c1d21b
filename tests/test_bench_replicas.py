"""Host logic of bench.py's multi-rank replica path, on CPU with two gloo ranks: the
slowest rank's time is what every rank reports, and the whole-job throughput counts
the points of all replicas."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(times[rank], world, torch.device("cpu"))
        value = bench.replica_throughput(world, 10, 4096 * 4096, ms)
        out.put((rank, ms, value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_throughput_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [12.5, 20.0]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    for rank, ms, value in got:
        assert ms == 20.0
        assert value == pytest.approx(2 * 10 * 4096 * 4096 / 0.020)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1, None) == 3.25
    assert bench.replica_throughput(1, 4, 100, 2.0) == pytest.approx(4 * 100 / 0.002)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.main(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"])
    assert capsys.readouterr().out == ""


def test_bench_rejects_bad_arguments():
    """bench.py refuses fewer than 3 warm-up steps and unknown extra lines, before any
    GPU work; the default runs every extra line."""
    sys.path.insert(0, ROOT)
    import bench
    for argv in (["--warmup", "2"], ["--extra", "poisson_star1024,nope"]):
        with pytest.raises(SystemExit) as e:
            bench.main(argv)
        assert e.value.code == 2
    assert set(bench.EXTRA_LINES) == {"poisson_star1024", "poisson_kite_d10",
                                      "ff_interior_kite2048", "ff_solve_kite2048",
                                      "ff_scaling", "stars8_batched"}
