"""The allocation-free Pearson entry point (ndf_pearson_noalloc), through the C
ABI, on two calls in a row, against the FP64 oracle and the regular entry point
(ndf_pearson).

ndf_pearson_noalloc exists for callers that cannot allocate device memory: its
only scratch is a fixed device array inside the library, and the caller passes
the ensemble and the output as its own device buffers.  Because every call
reuses that array, the second call must not see anything left over from the
first.  Each call is held to the Pearson tolerance (1e-5 absolute) against the
oracle's FP64 Eq. 1 directly, so the shifted single-pass accumulation of this
entry point is checked on its own and not only against another GPU path.  The
cases cover the 1024-thread staging kernel striding (M = 1000, 3000), constant
columns (r = 0 by definition), and the declared limit M = NDF_NOALLOC_MAX_M,
where the whole scratch array and its zero padding are in use."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
NOALLOC_MAX_M = 16384  # NDF_NOALLOC_MAX_M in include/ndf.h


def _fields(recipe, constant_vertex=None):
    a = synth.generate(recipe)
    b = synth.generate(synth.scaled(recipe, stream=1, share=0.6))
    if constant_vertex is not None:  # one constant column in each field
        M = a.shape[0]
        a.reshape(M, -1)[:, constant_vertex] = 0.75
        b.reshape(M, -1)[:, constant_vertex] = -2.5
    return a, b


@pytest.mark.parametrize("recipe,const", [
    (synth.TINY, None),
    (synth.scaled(synth.CSENS, M=700, Z=3, Y=5, X=7), None),
    (synth.scaled(synth.CSENS, M=1000, Z=2, Y=9, X=11), 17),
    (synth.scaled(synth.CSENS, M=3000, Z=1, Y=6, X=9), 5),
], ids=["tiny_16x16x4_m100", "m700_7x5x3_ragged", "m1000_11x9x2_const", "m3000_9x6x1_const"])
def test_noalloc_matches_oracle_twice(ndf_mod, ctx, recipe, const):
    ndf = ndf_mod
    a, b = _fields(recipe, const)
    M, Z, Y, X = a.shape
    N = Z * Y * X
    fa = ndf.ndf_load_ensemble(ctx, a, M, Z, Y, X)
    fb = ndf.ndf_load_ensemble(ctx, b, M, Z, Y, X)
    da = torch.from_numpy(a).cuda().contiguous()
    db = torch.from_numpy(b).cuda().contiguous()
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row: a self slice, then a cross-field slice with another
    # reference (with a constant column, the second call's reference is that column)
    ref2 = const if const is not None else N - 1
    calls = [(fa, fa, a, a, da, da, N // 3), (fa, fb, a, b, da, db, ref2)]
    outs = []
    for rid, qid, rh, qh, rdev, qdev, ref in calls:
        got = torch.full((N,), float("nan"), dtype=torch.float32, device="cuda")
        ndf.ndf_pearson_noalloc(rdev, qdev, M, N, ref, got, stream)
        outs.append((rid, qid, rh, qh, ref, got))
    torch.cuda.synchronize()
    for rid, qid, rh, qh, ref, got in outs:
        g = got.cpu().numpy()
        assert np.isfinite(g).all()
        want64 = oracle.pearson_volume(rh, qh, ref)
        assert np.abs(g.astype(np.float64) - want64).max() <= TOL
        want = np.empty(N, dtype=np.float32)
        ndf.ndf_pearson(ctx, rid, qid, ref, want)
        assert np.abs(g - want).max() <= 2 * TOL  # each within TOL of the oracle
        if const is not None:
            assert g[const] == 0.0  # a constant query column has no variance
            if ref == const:
                assert (g == 0.0).all()  # a constant reference column: r = 0 everywhere
    ndf.ndf_free_ensemble(ctx, fa)
    ndf.ndf_free_ensemble(ctx, fb)


def test_noalloc_at_the_member_limit(ndf_mod):
    """M = NDF_NOALLOC_MAX_M on a few vertices, two calls in a row (different
    references), against the oracle."""
    ndf = ndf_mod
    recipe = synth.scaled(synth.CSENS, M=NOALLOC_MAX_M, Z=1, Y=2, X=4)
    a = synth.generate(recipe)
    M, Z, Y, X = a.shape
    N = Z * Y * X
    da = torch.from_numpy(a).cuda().contiguous()
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for ref in (3, 6):
        got = torch.full((N,), float("nan"), dtype=torch.float32, device="cuda")
        ndf.ndf_pearson_noalloc(da, da, M, N, ref, got, stream)
        outs.append((ref, got))
    torch.cuda.synchronize()
    for ref, got in outs:
        want64 = oracle.pearson_volume(a, a, ref)
        assert np.abs(got.cpu().numpy().astype(np.float64) - want64).max() <= TOL


def test_noalloc_rejects_bad_arguments(ndf_mod):
    ndf = ndf_mod
    dev = torch.zeros(16, dtype=torch.float32, device="cuda")
    host = np.zeros(16, dtype=np.float32)
    for args in [(dev, dev, 1, 16, 0, dev),                           # M < 2
                 (dev, dev, 2, 8, 8, dev),                            # ref out of range
                 (host, dev, 2, 8, 0, dev),                           # host input
                 (dev, dev, 2, 8, 0, host)]:                          # host output
        with pytest.raises(ndf.NdfError) as ei:
            ndf.ndf_pearson_noalloc(*args)
        assert ei.value.status == ndf.NDF_ERR_ARG
    big = torch.zeros(NOALLOC_MAX_M + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(ndf.NdfError) as ei:  # one member beyond the fixed scratch array
        ndf.ndf_pearson_noalloc(big, big, NOALLOC_MAX_M + 1, 1, 0, big)
    assert ei.value.status == ndf.NDF_ERR_ARG
