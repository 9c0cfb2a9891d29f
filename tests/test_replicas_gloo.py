"""The multi-GPU form of bench.py is independent replicas (one solve per rank, no
collective in the data path): what ranks share is the timing rule - every rank waits at a
barrier, the job's time is the slowest rank's, and the value is the whole job's columns in
that time.  Checked here with two gloo ranks on the CPU; the reference arm's rule that only
rank 0 runs is checked in-process."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, dist, "cpu")
    value = bench.whole_job_value(world, 16 * 5, ms)
    out.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(out.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [150.0, 150.0]           # the slowest rank's time on both
    assert all(abs(r[2] - 2 * 80 / 0.150) < 1e-9 for r in res)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_value(1, 16, 2000.0) == 8.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "run_cpu_sample", lambda *a, **k: called.append(1))
    class A:
        method, steps, warmup, gpus = "cocr_rq", 1, 0, 2
    assert bench.run_reference(A()) is None
    assert not called
