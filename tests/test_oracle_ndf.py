"""Pins for the FP64 NDF oracle (Sec. 4): gradients against central finite
differences, trilinear encoding against closed forms, the symmetry the
architecture guarantees (Sec. 4.1), the output activations, and Adam against its
closed form under a constant gradient."""
import numpy as np
import pytest

import oracle

SHAPE_ARGS = ([4, 8], 2, 16)


def tiny(measure):
    return oracle.net_shape(*SHAPE_ARGS, measure)


def random_params(shape, seed, scale=0.4):
    return np.random.default_rng(seed).normal(size=oracle.ndf_param_count(shape)) * scale


def positions(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, size=(n, 3)), rng.uniform(-1, 1, size=(n, 3))


def test_param_count():
    s = tiny(0)
    grid = (4 ** 3 + 8 ** 3) * 2
    mlp = 16 * 8 + 16 + 2 * (16 * 16 + 16) + 16 + 1
    assert oracle.ndf_param_count(s) == grid + mlp
    # the benchmark network: 4 dense levels 32/64/128/256, 16 features, 128-wide MLP
    big = oracle.net_shape([32, 64, 128, 256], 16, 128, 0)
    n_grid = (32 ** 3 + 64 ** 3 + 128 ** 3 + 256 ** 3) * 16
    assert oracle.ndf_param_count(big) == n_grid + 128 * 128 * 3 + 128 * 3 + 128 + 1
    assert n_grid == 306_708_480


@pytest.mark.parametrize("measure", [0, 1])
def test_gradient_vs_central_differences(measure):
    s = tiny(measure)
    p = random_params(s, 1 + measure)
    pr, pq = positions(6, 3)
    target = np.random.default_rng(4).uniform(-0.5, 0.8, size=6)
    _, g = oracle.ndf_loss_grad(s, p, pr, pq, target)
    h = 1e-6
    rng = np.random.default_rng(5)
    # every MLP parameter and a sample of grid entries (most grid entries are untouched: 0)
    n_grid = (4 ** 3 + 8 ** 3) * 2
    idx = np.concatenate([rng.choice(n_grid, 200, replace=False), np.arange(n_grid, p.size)])
    for i in idx:
        q = p.copy()
        q[i] += h
        lp, _ = oracle.ndf_loss_grad(s, q, pr, pq, target, want_grad=False)
        q[i] -= 2 * h
        lm, _ = oracle.ndf_loss_grad(s, q, pr, pq, target, want_grad=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])


def test_encoding_at_grid_points_and_linear_fields():
    s = tiny(0)
    p = np.zeros(oracle.ndf_param_count(s))
    # level 0 (R=4): feature 0 = the point's x coordinate in [-1,1], feature 1 = 2y - z + 0.5
    off = 0
    for lvl, R in enumerate([4, 8]):
        for z in range(R):
            for y in range(R):
                for x in range(R):
                    c = np.array([x, y, z]) * 2.0 / (R - 1) - 1.0
                    k = off + ((z * R + y) * R + x) * 2
                    p[k] = c[0]
                    p[k + 1] = 2 * c[1] - c[2] + 0.5
        off += R ** 3 * 2
    rng = np.random.default_rng(7)
    for pos in rng.uniform(-1, 1, size=(50, 3)):
        f = oracle.ndf_encode(s, p, pos)
        # trilinear interpolation reproduces linear fields exactly on both levels
        for lvl in range(2):
            assert f[2 * lvl] == pytest.approx(pos[0], abs=1e-12)
            assert f[2 * lvl + 1] == pytest.approx(2 * pos[1] - pos[2] + 0.5, abs=1e-12)
    # at a grid point the stored value comes back exactly
    corner = np.array([-1.0, 1.0, -1.0 + 2.0 / 3.0])
    assert oracle.ndf_encode(s, p, corner)[0] == -1.0


@pytest.mark.parametrize("measure", [0, 1])
def test_symmetry_and_output_range(measure):
    s = tiny(measure)
    p = random_params(s, 11, scale=1.5)
    pr, pq = positions(64, 12)
    a = oracle.ndf_forward(s, p, pr, pq)
    b = oracle.ndf_forward(s, p, pq, pr)
    np.testing.assert_array_equal(a, b)  # Phi(p1, p2) = Phi(p2, p1) by construction
    if measure == 0:
        assert (np.abs(a) <= 1.0).all()  # tanh saturates to 1 in FP64 for |o| > 19
    else:
        assert (a > 0.0).all()


def test_constant_network_closed_form():
    for measure, act in [(0, np.tanh), (1, lambda o: np.log1p(np.exp(o)))]:
        s = tiny(measure)
        p = np.zeros(oracle.ndf_param_count(s))
        p[-1] = 0.37  # b4
        pr, pq = positions(5, 2)
        y = oracle.ndf_forward(s, p, pr, pq)
        np.testing.assert_allclose(y, act(0.37), rtol=0, atol=1e-15)
        t = np.linspace(-0.5, 0.5, 5)
        loss, g = oracle.ndf_loss_grad(s, p, pr, pq, t)
        assert loss == pytest.approx(np.mean(np.abs(act(0.37) - t)), abs=1e-15)
        # only b4 moves: dL/db4 = mean(sign(y - t)) * act'(b4)
        d = (1 - np.tanh(0.37) ** 2) if measure == 0 else 1 / (1 + np.exp(-0.37))
        assert g[-1] == pytest.approx(np.mean(np.sign(act(0.37) - t)) * d, abs=1e-15)
        assert np.count_nonzero(g[:-1]) == 0


def test_adam_constant_gradient_closed_form():
    # with g constant, m_hat = g and v_hat = g^2 at every step, so each step moves
    # every parameter by exactly lr * g / (|g| + eps)
    rng = np.random.default_rng(8)
    g = rng.normal(size=16)
    g[3] = 0.0
    p = rng.normal(size=16)
    m = np.zeros(16)
    v = np.zeros(16)
    lr, eps = 3e-4, 1e-8
    start = p.copy()
    for t in range(1, 6):
        before = p.copy()
        oracle.adam_step(p, g, m, v, t, lr=lr, eps=eps)
        np.testing.assert_allclose(before - p, lr * g / (np.abs(g) + eps), rtol=1e-9, atol=1e-18)
    assert p[3] == start[3]


def test_abs_term_gradient_consistent():
    # the per-sample accumulation returns the same loss and gradient, and the
    # summed magnitudes bound the (cancelling) sum element by element
    s = tiny(1)
    p = random_params(s, 13)
    pr, pq = positions(40, 14)
    t = np.random.default_rng(15).uniform(0.0, 1.5, size=40)
    l1, g1 = oracle.ndf_loss_grad(s, p, pr, pq, t)
    l2, g2, ga = oracle.ndf_loss_grad_abs(s, p, pr, pq, t)
    assert l1 == pytest.approx(l2, abs=1e-15)
    np.testing.assert_allclose(g1, g2, rtol=0, atol=1e-15)
    assert (ga >= np.abs(g2) - 1e-15).all()
