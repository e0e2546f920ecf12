"""Continuous-position training samples (Sec. 4.3) against the oracle: uniform
random positions, member columns by trilinear interpolation (FP32, the same
rounding on both sides, so the columns agree bit for bit), and the estimators on
the interpolated columns; then a network trained on renewed continuous samples."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def sample(ndf_mod, ctx, fa, fb, measure, k, n, seed):
    pr = np.empty((n, 3), np.float32)
    pq = np.empty((n, 3), np.float32)
    t = np.empty(n, np.float32)
    ndf_mod.ndf_sample_triples(ctx, fa, fb, measure, k, n, seed, pr, pq, t)
    return pr, pq, t


def test_pearson_targets_and_positions(ndf_mod, ctx, tiny_field):
    M, Z, Y, X = tiny_field.shape
    fid = ndf_mod.ndf_load_ensemble(ctx, tiny_field, M, Z, Y, X)
    pr, pq, t = sample(ndf_mod, ctx, fid, fid, ndf_mod.NDF_MEASURE_PEARSON, 0, 3000, 11)
    assert (pr >= -1).all() and (pr < 1).all() and (pq >= -1).all() and (pq < 1).all()
    # uniform: every octant of the cube is visited about equally
    octant = (pr > 0).astype(int) @ np.array([1, 2, 4])
    assert np.bincount(octant, minlength=8).min() > 3000 / 8 * 0.75
    pr2, _, t2 = sample(ndf_mod, ctx, fid, fid, ndf_mod.NDF_MEASURE_PEARSON, 0, 3000, 11)
    np.testing.assert_array_equal(pr, pr2)  # seeded
    np.testing.assert_array_equal(t, t2)
    pr3, _, _ = sample(ndf_mod, ctx, fid, fid, ndf_mod.NDF_MEASURE_PEARSON, 0, 3000, 12)
    assert not np.array_equal(pr, pr3)
    for i in range(0, 3000, 15):
        x = oracle.interp_column(tiny_field, pr[i])
        y = oracle.interp_column(tiny_field, pq[i])
        assert abs(t[i] - oracle.pearson(x, y)) <= 1e-5, i
    ndf_mod.ndf_free_ensemble(ctx, fid)


def test_ksg_targets_cross_field(ndf_mod, ctx):
    ra = synth.scaled(synth.CSENS, M=300, Z=3, Y=11, X=13)
    rb = synth.scaled(synth.CSENS_B, M=300, Z=3, Y=11, X=13)
    a, b = synth.generate(ra), synth.generate(rb)
    M, Z, Y, X = a.shape
    fa = ndf_mod.ndf_load_ensemble(ctx, a, M, Z, Y, X)
    fb = ndf_mod.ndf_load_ensemble(ctx, b, M, Z, Y, X)
    pr, pq, t = sample(ndf_mod, ctx, fa, fb, ndf_mod.NDF_MEASURE_MI_KSG, 6, 700, 5)
    for i in range(0, 700, 7):
        x = oracle.interp_column(a, pr[i])
        y = oracle.interp_column(b, pq[i])
        mi = oracle.ksg_pair(x, y, 6)[0]
        assert abs(t[i] - mi) <= 1e-6 * abs(mi) + 1e-9, (i, t[i], mi)
    ndf_mod.ndf_free_ensemble(ctx, fa)
    ndf_mod.ndf_free_ensemble(ctx, fb)


def test_sampler_argument_errors(ndf_mod, ctx, tiny_field):
    M, Z, Y, X = tiny_field.shape
    fid = ndf_mod.ndf_load_ensemble(ctx, tiny_field, M, Z, Y, X)
    pr = np.empty((4, 3), np.float32)
    t = np.empty(4, np.float32)
    for args in ((fid, fid, 9, 0, 4), (fid, fid, ndf_mod.NDF_MEASURE_MI_KSG, 0, 4),
                 (fid, fid, ndf_mod.NDF_MEASURE_PEARSON, 0, 0), (fid, 1 << 20, 0, 0, 4)):
        with pytest.raises(ndf_mod.NdfError):
            ndf_mod.ndf_sample_triples(ctx, *args, 1, pr, pr, t)
    ndf_mod.ndf_free_ensemble(ctx, fid)


def test_training_on_continuous_samples(ndf_mod, ctx):
    """Renewed continuous samples every pass: the decoded Pearson volumes at the
    grid vertices must beat the best constant volume by a wide margin."""
    field = synth.generate(synth.TINY)
    M, Z, Y, X = field.shape
    N = Z * Y * X
    fid = ndf_mod.ndf_load_ensemble(ctx, field, M, Z, Y, X)
    cfg = ndf_mod.ndf_train_cfg_default()
    cfg.res[:] = [4, 8, 16, 16]
    cfg.n_triples = 1 << 17
    cfg.batch = 1 << 12
    cfg.max_passes = 40
    cfg.lr = 3e-3
    cfg.continuous = 1
    model = ndf_mod.ndf_train(ctx, fid, fid, ndf_mod.NDF_MEASURE_PEARSON, 0, cfg)
    info = ndf_mod.ndf_model_info(model)
    assert info["passes"] >= 2 and np.isfinite(info["last_loss"])
    refs = synth.sample_vertices(synth.TINY, 12, seed=9)
    dec = np.empty((len(refs), N), dtype=np.float32)
    ndf_mod.ndf_infer_batch(model, refs, dec)
    exact = np.stack([oracle.pearson_volume(field, field, int(r)) for r in refs])
    mae = np.abs(dec - exact).mean()
    const = np.abs(exact - np.median(exact)).mean()
    print(f"continuous-sample NDF MAE {mae:.4f} vs best-constant MAE {const:.4f}")
    assert mae < 0.5 * const
    ndf_mod.ndf_model_free(model)
    ndf_mod.ndf_free_ensemble(ctx, fid)
