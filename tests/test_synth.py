"""The seeded generator: deterministic, shaped as stated, no method arithmetic."""
import numpy as np

import synth


def test_deterministic_and_shaped():
    r = synth.scaled(synth.CSENS, M=3, Z=4, Y=20, X=24)
    a = synth.generate(r)
    b = synth.generate(r)
    assert a.shape == (3, 4, 20, 24) and a.dtype == np.float32
    np.testing.assert_array_equal(a, b)
    c = synth.generate(synth.scaled(r, seed=r.seed + 1))
    assert not np.array_equal(a, c)


def test_white_noise_moments():
    # counter-based Box-Muller draws: mean 0, variance 1
    v = np.array([synth.normal(synth.SEED, 0x100, c) for c in range(20000)])
    assert abs(v.mean()) < 0.03 and abs(v.var() - 1.0) < 0.05


def test_unsmoothed_untransformed_is_white():
    r = synth.Recipe(M=64, Z=2, Y=8, X=8)
    f = synth.generate(r).reshape(64, -1)
    assert abs(f.mean()) < 0.05 and abs(f.var() - 1.0) < 0.05


def test_second_field_is_correlated():
    a = synth.generate(synth.scaled(synth.CSENS, M=200, Z=2, Y=16, X=16))
    b = synth.generate(synth.scaled(synth.CSENS_B, M=200, Z=2, Y=16, X=16))
    r = [np.corrcoef(a[:, 0, i, i], b[:, 0, i, i])[0, 1] for i in range(16)]
    assert 0.3 < float(np.mean(r)) < 0.9


def test_sample_vertices():
    v = synth.sample_vertices(synth.TINY, 100, seed=3)
    assert len(np.unique(v)) == 100 and v.min() >= 0 and v.max() < synth.TINY.N
