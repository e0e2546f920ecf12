"""The allocation-free Pearson entry point (ndf_pearson_noalloc) against the
regular one (ndf_pearson), through the C ABI, on two calls in a row.

ndf_pearson_noalloc exists for callers that cannot allocate device memory: its
only scratch is a fixed device array inside the library, and the caller passes
the ensemble and the output as its own device buffers.  Because every call
reuses that array, the second call must not see anything left over from the
first; both must agree with ndf_pearson within the Pearson tolerance (1e-5)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
NOALLOC_MAX_M = 16384  # NDF_NOALLOC_MAX_M in include/ndf.h


@pytest.mark.parametrize("recipe", [synth.TINY,
                                    synth.scaled(synth.CSENS, M=700, Z=3, Y=5, X=7)],
                         ids=["tiny_16x16x4_m100", "m700_7x5x3_ragged"])
def test_noalloc_matches_pearson_twice(ndf_mod, ctx, recipe):
    ndf = ndf_mod
    a = synth.generate(recipe)
    b = synth.generate(synth.scaled(recipe, stream=1, share=0.6))
    M, Z, Y, X = a.shape
    N = Z * Y * X
    fa = ndf.ndf_load_ensemble(ctx, a, M, Z, Y, X)
    fb = ndf.ndf_load_ensemble(ctx, b, M, Z, Y, X)
    da = torch.from_numpy(a).cuda().contiguous()
    db = torch.from_numpy(b).cuda().contiguous()
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row: a self slice, then a cross-field slice with another reference
    calls = [(fa, fa, da, da, N // 3), (fa, fb, da, db, N - 1)]
    outs = []
    for rid, qid, rdev, qdev, ref in calls:
        got = torch.full((N,), float("nan"), dtype=torch.float32, device="cuda")
        ndf.ndf_pearson_noalloc(rdev, qdev, M, N, ref, got, stream)
        outs.append((rid, qid, ref, got))
    torch.cuda.synchronize()
    for rid, qid, ref, got in outs:
        want = np.empty(N, dtype=np.float32)
        ndf.ndf_pearson(ctx, rid, qid, ref, want)
        g = got.cpu().numpy()
        assert np.isfinite(g).all()
        assert np.abs(g - want).max() <= TOL
    ndf.ndf_free_ensemble(ctx, fa)
    ndf.ndf_free_ensemble(ctx, fb)


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
