"""Parity at the paper's scale (1000 members, 250 x 352 x 20 grid, 7.04 GB), in
the launch configuration the benchmark times (full-volume calls), checked on
seeded vertex samples that the CPU oracle computes one by one."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def csens(ndf_mod, ctx):
    f = synth.generate(synth.CSENS)
    M, Z, Y, X = f.shape
    fid = ndf_mod.ndf_load_ensemble(ctx, f, M, Z, Y, X)
    yield f, fid
    ndf_mod.ndf_free_ensemble(ctx, fid)


REF = (131, 200, 9)  # (x, y, z)


def test_csens_pearson_sampled(ndf_mod, ctx, csens):
    f, fid = csens
    N = synth.CSENS.N
    r = synth.vertex_index(*REF, synth.CSENS)
    out = torch.empty(N, dtype=torch.float32, device="cuda")
    ndf_mod.ndf_pearson(ctx, fid, fid, r, out)
    ndf_mod.ndf_synchronize(ctx)
    verts = np.concatenate([synth.sample_vertices(synth.CSENS, 8192, seed=5),
                            [0, r, N - 1]]).astype(np.int64)
    ref = oracle.pearson_volume(f, f, r, verts=verts)
    got = out.cpu().numpy()[verts]
    assert np.abs(got - ref).max() <= 1e-5
    assert np.isfinite(out.cpu().numpy()).all()


@pytest.mark.parametrize("algorithm", ["pruned", "brute", "block"])
def test_csens_ksg_sampled(ndf_mod, ctx, csens, algorithm):
    f, fid = csens
    N = synth.CSENS.N
    M = synth.CSENS.M
    r = synth.vertex_index(*REF, synth.CSENS)
    out = torch.empty(N, dtype=torch.float32, device="cuda")
    code = {"pruned": ndf_mod.NDF_KSG_PRUNED, "brute": ndf_mod.NDF_KSG_BRUTE,
            "block": ndf_mod.NDF_KSG_BLOCK}[algorithm]
    ndf_mod.ndf_set_ksg_algorithm(ctx, code)
    ndf_mod.ndf_mi_ksg(ctx, fid, fid, r, 8, out)
    ndf_mod.ndf_synchronize(ctx)
    vol = out.cpu().numpy()
    assert np.isfinite(vol).all()
    verts = np.concatenate([synth.sample_vertices(synth.CSENS, 4096, seed=6),
                            [0, r, N - 1]]).astype(np.int64)
    ref = oracle.ksg_volume(f, f, r, 8, verts=verts)
    got = vol[verts].astype(np.float64)
    bad = np.abs(got - ref) > 1e-6 * np.abs(ref) + 1e-9
    assert not bad.any(), (verts[bad][:5], got[bad][:5], ref[bad][:5])
    # per-member eps / counts bit-exact on a smaller sample
    f2 = f.reshape(M, N)
    for v in synth.sample_vertices(synth.CSENS, 64, seed=7):
        eps = np.empty(M, np.float32)
        nx = np.empty(M, np.int32)
        ny = np.empty(M, np.int32)
        mi = np.empty(1, np.float64)
        ndf_mod.ndf_ksg_debug_pair(ctx, fid, fid, r, int(v), 8, eps, nx, ny, mi)
        o = oracle.ksg_pair(f2[:, r], f2[:, v], 8)
        np.testing.assert_array_equal(eps, o[1])
        np.testing.assert_array_equal(nx, o[2])
        np.testing.assert_array_equal(ny, o[3])
    ndf_mod.ndf_set_ksg_algorithm(ctx, ndf_mod.NDF_KSG_BLOCK)  # the default


def test_csens_ksg2_sampled(ndf_mod, ctx, csens):
    """KSG algorithm 2 on the full-size ensemble (the default, pruned search)
    against the oracle on sampled vertices; per-member extents and counts
    bit-exact on a smaller sample."""
    f, fid = csens
    N = synth.CSENS.N
    M = synth.CSENS.M
    r = synth.vertex_index(*REF, synth.CSENS)
    out = torch.empty(N, dtype=torch.float32, device="cuda")
    ndf_mod.ndf_mi_ksg2(ctx, fid, fid, r, 8, out)
    ndf_mod.ndf_synchronize(ctx)
    vol = out.cpu().numpy()
    assert np.isfinite(vol).all()
    verts = np.concatenate([synth.sample_vertices(synth.CSENS, 2048, seed=16),
                            [0, r, N - 1]]).astype(np.int64)
    ref = oracle.ksg2_volume(f, f, r, 8, verts=verts)
    got = vol[verts].astype(np.float64)
    bad = np.abs(got - ref) > 1e-6 * np.abs(ref) + 1e-9
    assert not bad.any(), (verts[bad][:5], got[bad][:5], ref[bad][:5])
    f2 = f.reshape(M, N)
    for v in synth.sample_vertices(synth.CSENS, 16, seed=17):
        ex, ey = np.empty(M, np.float32), np.empty(M, np.float32)
        nx, ny = np.empty(M, np.int32), np.empty(M, np.int32)
        mi = np.empty(1, np.float64)
        ndf_mod.ndf_ksg2_debug_pair(ctx, fid, fid, r, int(v), 8, ex, ey, nx, ny, mi)
        o = oracle.ksg2_pair(f2[:, r], f2[:, v], 8)
        np.testing.assert_array_equal(ex, o[1])
        np.testing.assert_array_equal(ey, o[2])
        np.testing.assert_array_equal(nx, o[3])
        np.testing.assert_array_equal(ny, o[4])


def test_csens_ksg_batch_sampled(ndf_mod, ctx, csens):
    """Four references in one batched launch against the oracle on sampled vertices."""
    f, fid = csens
    N = synth.CSENS.N
    refs = [int(v) for v in synth.sample_vertices(synth.CSENS, 4, seed=8)]
    out = torch.empty((4, N), dtype=torch.float32, device="cuda")
    ndf_mod.ndf_mi_ksg_batch(ctx, fid, fid, refs, 8, out)
    ndf_mod.ndf_synchronize(ctx)
    vol = out.cpu().numpy()
    verts = synth.sample_vertices(synth.CSENS, 512, seed=9)
    for i, r in enumerate(refs):
        ref = oracle.ksg_volume(f, f, r, 8, verts=verts)
        got = vol[i][verts].astype(np.float64)
        assert (np.abs(got - ref) <= 1e-6 * np.abs(ref) + 1e-9).all()
