"""The benchmark's multi-rank logic on CPU: two gloo ranks.

Each rank computes its own reference vertices (weak scaling, no data-path
collective); the per-rank timings meet in one max-reduction, and the job time
per volume divides the slowest rank's time by the volumes all ranks processed.
Under torchrun the reference arm runs on rank 0 alone; other ranks exit 0
without output."""
import io
import contextlib
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    refs = bench.rank_references(1000, 8, rank)
    timings = [10.0 + rank, 5.0 - rank, 7.5]
    mx = bench.max_over_ranks(timings, world, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, refs)
    q.put((rank, refs, mx, bench.job_ms_per_volume(mx[0], 4, world), gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, refs0, mx0, per0, g0), (r1, refs1, mx1, per1, g1) = res
    assert refs0 != refs1                      # every rank has its own references
    assert g0 == g1 == [refs0, refs1]
    assert mx0 == mx1 == [11.0, 5.0, 7.5]      # element-wise maximum over ranks
    assert per0 == per1 == pytest.approx(11.0 / (4 * world))


def test_single_rank_helpers():
    assert bench.max_over_ranks([3.0, 1.0], 1, "cpu") == [3.0, 1.0]
    assert bench.job_ms_per_volume(12.0, 3, 1) == 4.0
    assert bench.rank_references(50, 5, 0) == bench.rank_references(50, 5, 0)


def test_reference_arm_other_ranks_exit_silently(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        rc = bench.run_reference(None, None)
    assert rc == 0 and out.getvalue() == ""
