"""The benchmark's multi-rank logic (replicas: every rank runs the same workload, the
slowest rank's time counts, rank 0 reports; the reference arm runs on rank 0 only), on CPU
with world-size-2 gloo process groups."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")   # rank 1 is the slow one
        val = bench.job_gpx_s(world, 1_000_000, ms)

        class A:   # arguments of the reference arm
            workload, steps, warmup = "noiseblur512", 1, 0
        ref = bench.run_reference(A, rank, world)
        out[rank] = (ms, val, ref is None)
        torch.distributed.barrier()
    finally:
        torch.distributed.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_rank0_reports():
    mp = torch.multiprocessing.get_context("spawn")
    with mp.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [mp.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert abs(res[0][1] - 2 * 1_000_000 / 15e-3 / 1e9) < 1e-12
    assert res[0][2] is False and res[1][2] is True   # only rank 0 runs the reference arm


def test_single_rank_is_a_no_op():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_gpx_s(1, 2_000_000_000, 100.0) == 20.0
