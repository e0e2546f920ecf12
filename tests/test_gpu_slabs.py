"""Volumes of a grid split into z-slabs (one GPU, slabs computed in turn): the
reference column read from the slab that holds it (ndf_field_column) and the
slab volumes against it (ndf_pearson_column, ndf_mi_ksg_column), concatenated,
are bit-equal to the whole-grid calls, for every exact search; and they match
the oracle."""
import numpy as np
import pytest
import torch

import bench
import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("recipe,world", [
    (synth.TINY, 2),
    (synth.scaled(synth.CSENS, M=1000, Z=5, Y=9, X=11), 3),
], ids=["tiny_2_slabs", "m1000_11x9x5_3_slabs"])
def test_slab_volumes_bit_equal(ndf_mod, ctx, recipe, world):
    ndf = ndf_mod
    f = synth.generate(recipe)
    M, Z, Y, X = f.shape
    N, plane = Z * Y * X, X * Y
    k = 4 if recipe is synth.TINY else 8
    whole = ndf.ndf_load_ensemble(ctx, f, M, Z, Y, X)
    bounds = bench.slab_bounds(Z, world)
    slabs = [ndf.ndf_load_ensemble(ctx, np.ascontiguousarray(f[:, z0:z1]), M, z1 - z0, Y, X)
             for z0, z1 in bounds]
    refs = [0, N // 2 + 3, N - 1]
    searches = [ndf.NDF_KSG_BLOCK, ndf.NDF_KSG_LANES, ndf.NDF_KSG_PRUNED]
    try:
        for ref in refs:
            owner = bench.slab_owner(ref, plane, bounds)
            col = torch.empty(M, dtype=torch.float32, device="cuda")
            ndf.ndf_field_column(ctx, slabs[owner], ref - bounds[owner][0] * plane, col)
            col_host = np.empty(M, np.float32)
            ndf.ndf_field_column(ctx, whole, ref, col_host)
            np.testing.assert_array_equal(col.cpu().numpy(), f.reshape(M, N)[:, ref])
            np.testing.assert_array_equal(col_host, f.reshape(M, N)[:, ref])
            want_r = np.empty(N, np.float32)
            ndf.ndf_pearson(ctx, whole, whole, ref, want_r)
            got_r = np.concatenate([_slab_out(ndf.ndf_pearson_column, ctx, col, s, b, plane)
                                    for s, b in zip(slabs, bounds)])
            np.testing.assert_array_equal(got_r, want_r)
            assert np.abs(got_r - oracle.pearson_volume(f, f, ref)).max() <= 1e-5
            mi_ref = oracle.ksg_volume(f, f, ref, k)
            for code in searches:
                ndf.ndf_set_ksg_algorithm(ctx, code)
                want_mi = np.empty(N, np.float32)
                ndf.ndf_mi_ksg(ctx, whole, whole, ref, k, want_mi)
                got_mi = np.concatenate([
                    _slab_out(lambda c, cl, s, o: ndf.ndf_mi_ksg_column(c, cl, s, k, o), ctx,
                              col_host, s, b, plane) for s, b in zip(slabs, bounds)])
                np.testing.assert_array_equal(got_mi, want_mi)
                assert (np.abs(got_mi - mi_ref) <= 1e-6 * np.abs(mi_ref) + 1e-9).all()
    finally:
        ndf.ndf_set_ksg_algorithm(ctx, ndf.NDF_KSG_LANES)
        ndf.ndf_free_ensemble(ctx, whole)
        for s in slabs:
            ndf.ndf_free_ensemble(ctx, s)


def _slab_out(fn, ctx, col, slab_id, bounds, plane):
    n = (bounds[1] - bounds[0]) * plane
    out = np.empty(n, np.float32)
    fn(ctx, col, slab_id, out)
    return out


def test_column_calls_reject_bad_arguments(ndf_mod, ctx, tiny_field):
    ndf = ndf_mod
    M, Z, Y, X = tiny_field.shape
    fid = ndf.ndf_load_ensemble(ctx, tiny_field, M, Z, Y, X)
    col = np.zeros(M, np.float32)
    out = np.empty(Z * Y * X, np.float32)
    for call in (lambda: ndf.ndf_field_column(ctx, fid, Z * Y * X, col),
                 lambda: ndf.ndf_field_column(ctx, fid, -1, col),
                 lambda: ndf.ndf_field_column(ctx, 1 << 20, 0, col),
                 lambda: ndf.ndf_pearson_column(ctx, None, fid, out),
                 lambda: ndf.ndf_mi_ksg_column(ctx, col, fid, M, out),
                 lambda: ndf.ndf_mi_ksg_column(ctx, col, fid, 0, out)):
        with pytest.raises(ndf.NdfError) as ei:
            call()
        assert ei.value.status == ndf.NDF_ERR_ARG
    ndf.ndf_free_ensemble(ctx, fid)
    with pytest.raises(ndf.NdfError) as ei:
        ndf.ndf_pearson_column(ctx, col, fid, out)
    assert ei.value.status == ndf.NDF_ERR_STATE
