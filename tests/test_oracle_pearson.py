"""Pins for the oracle's Pearson r (Sec. 3.1, Eq. 1) against things other than itself."""
import numpy as np
import pytest

import oracle
from golden_io import pearson_hand_cases


def test_hand_example():
    for c in pearson_hand_cases():
        assert oracle.pearson(c["x"], c["y"]) == pytest.approx(c["r"], abs=1e-15)


def test_matches_numpy_corrcoef():
    rng = np.random.default_rng(1)
    for M in (2, 3, 17, 100, 1000):
        for _ in range(5):
            x = rng.normal(size=M).astype(np.float32)
            y = (0.4 * x + rng.normal(size=M)).astype(np.float32) + 3.0
            ref = np.corrcoef(x.astype(np.float64), y.astype(np.float64))[0, 1]
            assert oracle.pearson(x, y) == pytest.approx(ref, abs=1e-12)


def test_invariants():
    rng = np.random.default_rng(2)
    x = rng.normal(size=200).astype(np.float32)
    y = (np.sin(x) + 0.3 * rng.normal(size=200)).astype(np.float32)
    r = oracle.pearson(x, y)
    assert oracle.pearson(x, x) == pytest.approx(1.0, abs=1e-14)
    assert oracle.pearson(y, x) == r  # S_mu symmetry (Sec. 3)
    assert oracle.pearson(x, -y) == pytest.approx(-r, abs=1e-14)
    assert oracle.pearson(2.0 * x + 7.0, y) == pytest.approx(r, abs=1e-6)
    assert -1.0 <= r <= 1.0


def test_zero_variance_reads_zero():
    x = np.ones(10, dtype=np.float32)
    y = np.arange(10, dtype=np.float32)
    assert oracle.pearson(x, y) == 0.0


def test_volume_matches_pairs(tiny_field, tiny_ref):
    M = tiny_field.shape[0]
    f2 = tiny_field.reshape(M, -1)
    vol = oracle.pearson_volume(tiny_field, tiny_field, tiny_ref)
    assert vol.shape == (f2.shape[1],)
    assert vol[tiny_ref] == pytest.approx(1.0, abs=1e-14)
    idx = [0, 5, 77, 511, 1023]
    for v in idx:
        ref = np.corrcoef(f2[:, tiny_ref].astype(np.float64), f2[:, v].astype(np.float64))[0, 1]
        assert vol[v] == pytest.approx(ref, abs=1e-12)
    sub = oracle.pearson_volume(tiny_field, tiny_field, tiny_ref, verts=idx)
    np.testing.assert_array_equal(sub, vol[idx])


def test_volume_rejects_bad_ref(tiny_field):
    with pytest.raises(ValueError):
        oracle.pearson_volume(tiny_field, tiny_field, 10**6)


def test_volume_cross_field_reference_from_first_field():
    """A -> B volumes: r(A[:, ref], B[:, v]) against numpy's corrcoef; the
    swapped call reads other columns and differs."""
    rng = np.random.default_rng(41)
    M, N, ref = 300, 20, 7
    a = rng.normal(size=(M, 1, 2, N // 2)).astype(np.float32)
    b = (0.7 * a[:, :, ::-1] + 0.5 * rng.normal(size=a.shape)).astype(np.float32)
    a2, b2 = a.reshape(M, N), b.reshape(M, N)
    vol = oracle.pearson_volume(a, b, ref)
    for v in range(N):
        want = np.corrcoef(a2[:, ref].astype(np.float64), b2[:, v].astype(np.float64))[0, 1]
        assert vol[v] == pytest.approx(want, abs=1e-12)
    assert np.abs(oracle.pearson_volume(b, a, ref) - vol).max() > 1e-2
