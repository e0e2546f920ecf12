"""Batched multi-reference Pearson (Eq. 1 for R references in one call).

FP32 batches must equal the single-reference volumes bit for bit.  The tensor-core
precisions are compared with the FP64 oracle element by element; their error
bounds follow from the operand rounding (z has unit 2-norm per vertex):
  TF32    |dz| <= 2^-11 |z|            ->  |dr| <= 2^-10 + accumulation  (gate 1.5e-3)
  BF16x3  |z - hi - lo| <= 2^-17 |z|,  dropped lo*lo' <= 2^-16 |z||z'|
                                       ->  |dr| <= ~4e-5                 (gate 1e-4)
Both errors are printed (max and mean abs vs FP64)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

GATE = {"tf32": 1.5e-3, "bf16x3": 1e-4}


def prec_code(ndf, name):
    return {"fp32": ndf.NDF_PREC_FP32, "tf32": ndf.NDF_PREC_TF32,
            "bf16x3": ndf.NDF_PREC_BF16X3}[name]


def run_batch(ndf, ctx, fa, fb, refs, prec, N, device):
    if device:
        out = torch.full((len(refs), N), float("nan"), dtype=torch.float32, device="cuda")
        ndf.ndf_pearson_batch(ctx, fa, fb, refs, prec, out)
        ndf.ndf_synchronize(ctx)
        return out.cpu().numpy()
    out = np.full((len(refs), N), np.nan, dtype=np.float32)
    ndf.ndf_pearson_batch(ctx, fa, fb, refs, prec, out)
    return out


@pytest.mark.parametrize("shape,R", [((1000, 2, 10, 25), 64),   # N=500: ragged 128-vertex tile
                                     ((100, 4, 16, 16), 3),     # tiny grid, Rpad = 32
                                     ((1000, 1, 9, 41), 300),   # two GEMM chunks (256 + 44)
                                     ((64, 3, 7, 11), 32)])     # K padded from 64 members
def test_batch_precisions(ndf_mod, ctx, shape, R):
    ndf = ndf_mod
    rng = np.random.default_rng(R)
    a = synth.generate(synth.scaled(synth.CSENS, M=shape[0], Z=shape[1], Y=shape[2], X=shape[3],
                                    sigma=(2.0, 2.0, 1.0)))
    M = shape[0]
    N = a[0].size
    fid = ndf.ndf_load_ensemble(ctx, a, *a.shape)
    refs = [int(r) for r in rng.integers(0, N, size=R)]
    want = np.stack([oracle.pearson_volume(a, a, r) for r in refs])
    # exact path equals the single-reference kernel
    fp32 = run_batch(ndf, ctx, fid, fid, refs, ndf.NDF_PREC_FP32, N, device=False)
    for i in (0, R // 2, R - 1):
        single = np.empty(N, dtype=np.float32)
        ndf.ndf_pearson(ctx, fid, fid, refs[i], single)
        np.testing.assert_array_equal(fp32[i], single)
    assert np.abs(fp32 - want).max() <= 1e-5
    for name in ("tf32", "bf16x3"):
        for device in (True, False):
            got = run_batch(ndf, ctx, fid, fid, refs, prec_code(ndf, name), N, device)
            assert np.isfinite(got).all(), name
            err = np.abs(got.astype(np.float64) - want)
            print(f"{name} M={M} N={N} R={R}: max {err.max():.3e} mean {err.mean():.3e}")
            assert err.max() <= GATE[name], (name, err.max())
            # the self-correlation entries are 1 up to the same bound
            for i, r in enumerate(refs[:8]):
                assert abs(got[i, r] - 1.0) <= GATE[name]
    ndf.ndf_free_ensemble(ctx, fid)


def test_batch_cross_field(ndf_mod, ctx):
    ndf = ndf_mod
    ra = synth.scaled(synth.CSENS, M=500, Z=2, Y=12, X=20, sigma=(3.0, 3.0, 1.0))
    a = synth.generate(ra)
    b = synth.generate(synth.scaled(ra, stream=1, share=0.6))
    N = a[0].size
    fa = ndf.ndf_load_ensemble(ctx, a, *a.shape)
    fb = ndf.ndf_load_ensemble(ctx, b, *b.shape)
    refs = [0, 17, N - 1, 200]
    want = np.stack([oracle.pearson_volume(a, b, r) for r in refs])
    for name in ("tf32", "bf16x3"):
        got = run_batch(ndf, ctx, fa, fb, refs, prec_code(ndf, name), N, device=True)
        assert np.abs(got - want).max() <= GATE[name], name
    ndf.ndf_free_ensemble(ctx, fa)
    ndf.ndf_free_ensemble(ctx, fb)


def test_batch_argument_errors(ndf_mod, ctx, tiny_field):
    ndf = ndf_mod
    fid = ndf.ndf_load_ensemble(ctx, tiny_field, *tiny_field.shape)
    N = tiny_field[0].size
    out = np.empty((2, N), dtype=np.float32)
    for refs, prec in [([0, N], ndf.NDF_PREC_TF32), ([-1, 0], ndf.NDF_PREC_FP32),
                       ([0, 1], 7)]:
        with pytest.raises(ndf.NdfError) as ei:
            ndf.ndf_pearson_batch(ctx, fid, fid, refs, prec, out)
        assert ei.value.status == ndf.NDF_ERR_ARG
    with pytest.raises(ndf.NdfError):
        ndf.ndf_pearson_batch(ctx, fid, fid, [], ndf.NDF_PREC_TF32, out)
    ndf.ndf_free_ensemble(ctx, fid)
