"""Multi-process path of the benchmark on CPU (gloo, world size 2): the
solve shards as independent replicas, so the only collective is the
max-over-ranks of the step time, and the whole-job value counts every
rank's chain."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, ms_by_rank, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(ms_by_rank[rank])
    out[rank] = (ms, bench.replica_throughput(world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_value_gloo_world2():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, [2.5, 3.75], out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    import bench
    for r in range(2):
        ms, value = res[r]
        assert ms == pytest.approx(3.75)                         # the slowest rank sets the time
        assert value == pytest.approx(2 * bench.EVALS_4096 / 3.75e-3)


def test_single_process_is_local_value():
    import bench
    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.replica_throughput(1, 1.0) == pytest.approx(bench.EVALS_4096 / 1e-3)


def test_reference_arm_non_zero_rank_does_no_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 0
    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""
