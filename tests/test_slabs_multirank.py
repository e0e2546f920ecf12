"""The z-slab split of the benchmark's multi-GPU mode, on CPU ranks (gloo).

Each rank holds one contiguous z-slab of the tiny ensemble.  Per reference, the
rank whose slab holds the reference vertex reads its member column and
broadcasts it (the split's one exchange); every rank computes the volumes of its
own slab against that column, here with the oracle's per-pair functions (the
per-slab GPU kernels have their own parity tests: tests/test_gpu_slabs.py).
The gathered slab volumes must be bit-equal to the single-process volumes."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, refs, q):
    import oracle
    import synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    f = synth.generate(synth.TINY)
    M, Z, Y, X = f.shape
    plane = X * Y
    bounds = bench.slab_bounds(Z, world)
    z0, z1 = bounds[rank]
    slab = np.ascontiguousarray(f[:, z0:z1]).reshape(M, -1)  # this rank's data only
    exchanged = []

    def column_of(v_local):
        return torch.from_numpy(slab[:, v_local].copy())

    def broadcast(col, owner):
        t = col if col is not None else torch.empty(M, dtype=torch.float32)
        dist.broadcast(t, src=owner)
        exchanged.append(t.numel())
        return t

    def compute(col):
        x = col.numpy()
        r = np.array([oracle.pearson(x, slab[:, v]) for v in range(slab.shape[1])])
        mi = np.array([oracle.ksg_pair(x, slab[:, v], 4)[0] for v in range(slab.shape[1])])
        return r, mi

    out = []
    for ref in refs:
        r, mi = bench.slab_step(ref, plane, bounds, rank, column_of, broadcast, compute)
        gathered = [None] * world
        dist.all_gather_object(gathered, (r, mi))
        out.append(gathered)
    q.put((rank, out, exchanged))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_split_gloo(world):
    import oracle
    import synth

    f = synth.generate(synth.TINY)
    M, Z, Y, X = f.shape
    refs = [synth.vertex_index(*synth.TINY_REF, synth.TINY),  # z = 2
            synth.vertex_index(3, 5, 0, synth.TINY), synth.vertex_index(15, 15, 3, synth.TINY)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, refs, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, out, exchanged in res:
        assert exchanged == [M] * len(refs)  # one M-float column per reference
    for i, ref in enumerate(refs):
        gathered = res[0][1][i]
        r = np.concatenate([g[0] for g in gathered])
        mi = np.concatenate([g[1] for g in gathered])
        np.testing.assert_array_equal(r, oracle.pearson_volume(f, f, ref))
        np.testing.assert_array_equal(mi, oracle.ksg_volume(f, f, ref, 4))


def test_slab_bounds_and_owner():
    assert bench.slab_bounds(20, 1) == [(0, 20)]
    assert bench.slab_bounds(20, 8) == [(0, 3), (3, 6), (6, 9), (9, 12), (12, 14), (14, 16),
                                        (16, 18), (18, 20)]
    assert bench.slab_bounds(2, 3) == [(0, 1), (1, 2), (2, 2)]  # an empty slab
    for Z, world in ((20, 8), (4, 3), (7, 7), (5, 2)):
        b = bench.slab_bounds(Z, world)
        assert b[0][0] == 0 and b[-1][1] == Z
        assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
        assert max(z1 - z0 for z0, z1 in b) - min(z1 - z0 for z0, z1 in b) <= 1
    plane = 6
    b = bench.slab_bounds(5, 2)  # (0, 3), (3, 5)
    assert [bench.slab_owner(v, plane, b) for v in (0, 17, 18, 29)] == [0, 0, 1, 1]
    with pytest.raises(ValueError):
        bench.slab_owner(30, plane, b)
