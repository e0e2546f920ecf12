"""Pins for the oracle's KSG algorithm-1 estimator (Sec. 3.2, Sec. 6.2) and digamma.

Each pin is fixed by something other than the oracle itself: a hand-enumerated
table, a closed form, an invariant of the definition, a textbook routine
(scipy's digamma) or the Gaussian theory value."""
from concurrent.futures import ThreadPoolExecutor
from fractions import Fraction

import numpy as np
import pytest

import oracle
from golden_io import ksg2_hand_cases, ksg_hand_cases

EULER_GAMMA = 0.57721566490153286061


def psi_exact(n):
    """psi(n) = H_{n-1} - gamma as an exact harmonic fraction plus gamma."""
    return float(sum(Fraction(1, j) for j in range(1, n))) - EULER_GAMMA


def test_digamma_closed_forms():
    assert oracle.digamma_int(1) == pytest.approx(-EULER_GAMMA, abs=1e-16)
    assert oracle.digamma_int(2) == pytest.approx(1.0 - EULER_GAMMA, abs=1e-16)
    for n in (3, 10, 57, 1000):
        assert oracle.digamma_int(n) == pytest.approx(psi_exact(n), abs=1e-13)


def test_digamma_vs_scipy():
    sp = pytest.importorskip("scipy.special")
    for n in (1, 2, 5, 9, 64, 1001, 4097):
        assert oracle.digamma_int(n) == pytest.approx(float(sp.digamma(n)), abs=1e-13)


@pytest.mark.parametrize("case", ksg_hand_cases(), ids=lambda c: c["name"])
def test_hand_enumerated(case):
    mi, eps, nx, ny = oracle.ksg_pair(case["x"], case["y"], case["k"])
    np.testing.assert_array_equal(eps, np.array(case["eps"], dtype=np.float32))
    np.testing.assert_array_equal(nx, case["nx"])
    np.testing.assert_array_equal(ny, case["ny"])
    assert mi == pytest.approx(float(case["mi"]), abs=1e-14)


def _no_tie_sample(M, seed):
    """distinct values whose sorted gaps are distinct (no distance ties)"""
    rng = np.random.default_rng(seed)
    while True:
        x = rng.random(M).astype(np.float32)
        s = np.sort(x.astype(np.float64))
        gaps = np.diff(s)
        if len(np.unique(x)) == M and len(np.unique(np.round(gaps, 12))) == M - 1:
            return x


@pytest.mark.parametrize("M,k", [(100, 4), (1000, 8), (37, 1), (50, 49)])
def test_self_pair_closed_form(M, k):
    # x == y with no distance ties: the k-1 nearer neighbours are counted in each
    # marginal, so I = psi(k) + psi(M) - 2 psi(k) = psi(M) - psi(k).
    x = _no_tie_sample(M, seed=M + k)
    # the x-sorted neighbour distances of each point must be tie-free for the
    # count k-1 to hold exactly; check on the data itself
    for i in range(M):
        d = np.sort(np.abs(x[i] - np.delete(x, i)))
        if k < M - 1:
            assert d[k - 1] != d[k]
    mi, eps, nx, ny = oracle.ksg_pair(x, x, k)
    assert (nx == k - 1).all() and (ny == k - 1).all()
    assert mi == pytest.approx(psi_exact(M) - psi_exact(k), abs=1e-12)


def test_symmetry_bit_identical():
    rng = np.random.default_rng(5)
    x = rng.normal(size=300).astype(np.float32)
    y = (x ** 3 + rng.normal(size=300)).astype(np.float32)
    a = oracle.ksg_pair(x, y, 8)
    b = oracle.ksg_pair(y, x, 8)
    assert a[0] == b[0]  # Eq. 2: I(X1;X2) = I(X2;X1)
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[3])
    np.testing.assert_array_equal(a[3], b[2])


@pytest.mark.parametrize("scale", [2.0, 0.5, 1024.0])
def test_power_of_two_scaling(scale):
    rng = np.random.default_rng(6)
    x = rng.normal(size=400).astype(np.float32)
    y = (np.tanh(x) + 0.5 * rng.normal(size=400)).astype(np.float32)
    a = oracle.ksg_pair(x, y, 8)
    b = oracle.ksg_pair(x * np.float32(scale), y * np.float32(scale), 8)
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[2], b[2])
    np.testing.assert_array_equal(a[3], b[3])
    np.testing.assert_array_equal(a[1] * np.float32(scale), b[1])


def test_member_permutation():
    rng = np.random.default_rng(7)
    x = rng.normal(size=500).astype(np.float32)
    y = (x + rng.normal(size=500)).astype(np.float32)
    perm = rng.permutation(500)
    a = oracle.ksg_pair(x, y, 8)
    b = oracle.ksg_pair(x[perm], y[perm], 8)
    np.testing.assert_array_equal(a[2][perm], b[2])
    np.testing.assert_array_equal(a[3][perm], b[3])
    assert a[0] == pytest.approx(b[0], abs=1e-13)


def test_rejects_bad_k():
    with pytest.raises(ValueError):
        oracle.ksg_pair([0, 1, 2], [0, 1, 2], 3)
    with pytest.raises(ValueError):
        oracle.ksg_pair([0, 1, 2], [0, 1, 2], 0)


def _gauss_estimates(rho, M, seeds, k=8, transform=None):
    def one(s):
        rng = np.random.default_rng(1000 + s)
        x = rng.normal(size=M)
        y = rho * x + np.sqrt(1 - rho * rho) * rng.normal(size=M)
        if transform is not None:
            x = transform(x)
        return oracle.ksg_pair(x.astype(np.float32), y.astype(np.float32), k)[0]

    with ThreadPoolExecutor(max_workers=8) as ex:
        return np.array(list(ex.map(one, range(seeds))))


@pytest.mark.parametrize("rho", [0.0, 0.3, 0.6, 0.9])
def test_bivariate_gaussian_theory(rho):
    # I = -1/2 log(1 - rho^2) for a bivariate Gaussian; the spread is measured
    # over 32 seeds and the mean must sit within 4 standard deviations.
    est = _gauss_estimates(rho, 10_000, 32)
    truth = -0.5 * np.log(1.0 - rho * rho)
    sd = est.std(ddof=1)
    assert abs(est.mean() - truth) <= 4.0 * sd, (est.mean(), truth, sd)
    assert sd < 0.05


def test_monotone_transform_within_spread():
    # MI is invariant under monotone per-variable maps; max-norm KSG is only
    # approximately so, so the shift must stay within the seed spread.
    base = _gauss_estimates(0.6, 5000, 16)
    expd = _gauss_estimates(0.6, 5000, 16, transform=np.exp)
    cube = _gauss_estimates(0.6, 5000, 16, transform=lambda v: v ** 3)
    sd = max(base.std(ddof=1), expd.std(ddof=1), cube.std(ddof=1))
    assert abs(expd.mean() - base.mean()) <= 4.0 * sd
    assert abs(cube.mean() - base.mean()) <= 4.0 * sd


def test_volume_matches_pairs(tiny_field, tiny_ref):
    M = tiny_field.shape[0]
    f2 = tiny_field.reshape(M, -1)
    verts = [0, 3, tiny_ref, 700, 1023]
    vol = oracle.ksg_volume(tiny_field, tiny_field, tiny_ref, 4, verts=verts)
    for i, v in enumerate(verts):
        assert vol[i] == oracle.ksg_pair(f2[:, tiny_ref], f2[:, v], 4)[0]
    # the self pair is the closed form psi(M) - psi(k) when no distance ties
    assert vol[2] == pytest.approx(psi_exact(M) - psi_exact(4), abs=1e-9)


def test_pairs_match_single_pairs(tiny_field, tiny_ref):
    """ksg_pairs (the parallel per-member form used by the paper-scale GPU
    parity) gives, row by row, what ksg_pair gives for the same columns."""
    M = tiny_field.shape[0]
    f2 = tiny_field.reshape(M, -1)
    verts = np.array([0, 3, tiny_ref, 700, 1023], dtype=np.int64)
    mi, eps, nx, ny = oracle.ksg_pairs(tiny_field, tiny_field, tiny_ref, 4, verts)
    for i, v in enumerate(verts):
        o = oracle.ksg_pair(f2[:, tiny_ref], f2[:, v], 4)
        assert mi[i] == o[0]
        np.testing.assert_array_equal(eps[i], o[1])
        np.testing.assert_array_equal(nx[i], o[2])
        np.testing.assert_array_equal(ny[i], o[3])
    # self pair without ties: every member has n_x = n_y = k - 1
    assert (nx[2] == 3).all() and (ny[2] == 3).all()
    with pytest.raises(ValueError):
        oracle.ksg_pairs(tiny_field, tiny_field, tiny_ref, 4, np.array([1 << 20]))


def test_volumes_take_reference_from_ref_field():
    """Cross-field volumes (the A -> B case): the reference column comes from the
    first field and every query column from the second, vertex by vertex, for
    both estimators (a swapped pair of fields gives other columns and fails)."""
    rng = np.random.default_rng(31)
    M, N, r = 200, 12, 5
    a = rng.normal(size=(M, 1, 1, N)).astype(np.float32)
    b = (np.tanh(a[:, :, :, ::-1]) + 0.4 * rng.normal(size=(M, 1, 1, N))).astype(np.float32)
    a2, b2 = a.reshape(M, N), b.reshape(M, N)
    verts = list(range(N))
    v1 = oracle.ksg_volume(a, b, r, 4, verts=verts)
    v2 = oracle.ksg2_volume(a, b, r, 4, verts=verts)
    for v in verts:
        assert v1[v] == oracle.ksg_pair(a2[:, r], b2[:, v], 4)[0]
        assert v2[v] == oracle.ksg2_pair(a2[:, r], b2[:, v], 4)[0]
    swapped = oracle.ksg_volume(b, a, r, 4, verts=verts)
    assert np.abs(swapped - v1).max() > 1e-3


# ---------------------------------------------------------------- algorithm 2
@pytest.mark.parametrize("case", ksg2_hand_cases(), ids=lambda c: "alg2_" + c["name"])
def test_alg2_hand_enumerated(case):
    mi, ex, ey, nx, ny = oracle.ksg2_pair(case["x"], case["y"], case["k"])
    np.testing.assert_array_equal(ex, np.array(case["ex"], dtype=np.float32))
    np.testing.assert_array_equal(ey, np.array(case["ey"], dtype=np.float32))
    np.testing.assert_array_equal(nx, case["nx"])
    np.testing.assert_array_equal(ny, case["ny"])
    assert mi == pytest.approx(float(case["mi"]), abs=1e-14)


@pytest.mark.parametrize("M,k", [(100, 4), (1000, 8), (37, 1)])
def test_alg2_self_pair_closed_form(M, k):
    # x == y with no distance ties: the neighbour set is the k nearest in x, so
    # ex = ey = the k-th nearest |dx| and nx = ny = k:
    # I2 = psi(k) - 1/k + psi(M) - 2 psi(k) = psi(M) - psi(k) - 1/k.
    x = _no_tie_sample(M, seed=3 * M + k)
    for i in range(M):
        d = np.sort(np.abs(x[i] - np.delete(x, i)))
        assert d[k - 1] != d[k]
    mi, ex, ey, nx, ny = oracle.ksg2_pair(x, x, k)
    np.testing.assert_array_equal(ex, ey)
    assert (nx == k).all() and (ny == k).all()
    assert mi == pytest.approx(psi_exact(M) - psi_exact(k) - 1.0 / k, abs=1e-12)


def test_alg2_symmetry_and_count_bounds():
    rng = np.random.default_rng(9)
    x = rng.normal(size=400).astype(np.float32)
    y = (np.sin(2 * x) + 0.5 * rng.normal(size=400)).astype(np.float32)
    a = oracle.ksg2_pair(x, y, 6)
    b = oracle.ksg2_pair(y, x, 6)
    assert a[0] == b[0]  # the definition is symmetric in the two variables
    np.testing.assert_array_equal(a[1], b[2])
    np.testing.assert_array_equal(a[3], b[4])
    # every member of a neighbour set lies within both extents: counts >= k
    assert (a[3] >= 6).all() and (a[4] >= 6).all()
    # the set's extents are at most eps (alg. 1) and one of them equals it
    _, eps, _, _ = oracle.ksg_pair(x, y, 6)
    assert (np.maximum(a[1], a[2]) == eps).all()


def test_alg2_gaussian_theory():
    # bivariate normal, rho = 0.6: I = -ln(1 - rho^2) / 2 = 0.2231 nats; the
    # estimator's spread at M = 2000 is about 0.02 (three seeds averaged)
    rho = 0.6
    vals = []
    for seed in range(3):
        rng = np.random.default_rng(100 + seed)
        z = rng.normal(size=(2, 2000))
        x = z[0].astype(np.float32)
        y = (rho * z[0] + np.sqrt(1 - rho ** 2) * z[1]).astype(np.float32)
        vals.append(oracle.ksg2_pair(x, y, 4)[0])
    assert np.mean(vals) == pytest.approx(-0.5 * np.log(1 - rho ** 2), abs=0.04)


def test_alg2_volume_matches_pairs(tiny_field, tiny_ref):
    M = tiny_field.shape[0]
    f2 = tiny_field.reshape(M, -1)
    verts = [0, 3, tiny_ref, 700, 1023]
    vol = oracle.ksg2_volume(tiny_field, tiny_field, tiny_ref, 4, verts=verts)
    for i, v in enumerate(verts):
        assert vol[i] == oracle.ksg2_pair(f2[:, tiny_ref], f2[:, v], 4)[0]
    # the self pair: psi(M) - psi(k) - 1/k when the k-th and (k+1)-th nearest
    # |dx| of every member differ
    x = f2[:, tiny_ref].astype(np.float64)
    for i in range(M):
        d = np.sort(np.abs(np.float32(x[i]) - np.delete(f2[:, tiny_ref], i)))
        assert d[3] != d[4]
    assert vol[2] == pytest.approx(psi_exact(M) - psi_exact(4) - 0.25, abs=1e-9)
    # the whole volume equals the listed vertices where they overlap
    full = oracle.ksg2_volume(tiny_field, tiny_field, tiny_ref, 4)
    np.testing.assert_array_equal(full[verts], vol)

