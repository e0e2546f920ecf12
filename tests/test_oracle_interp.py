"""Pins for the oracle's trilinear sampling of member columns at continuous
positions (Sec. 4.3): affine fields are reproduced, vertices return their own
column, and the weights of a cell sum to one."""
import numpy as np
import pytest

import oracle


def vertex_pos(i, n):
    return -1.0 + 2.0 * i / (n - 1) if n > 1 else 0.0


def test_vertices_return_their_column():
    rng = np.random.default_rng(1)
    f = rng.normal(size=(5, 3, 4, 6)).astype(np.float32)
    for (x, y, z) in [(0, 0, 0), (5, 3, 2), (2, 1, 1), (4, 2, 0)]:
        p = [vertex_pos(x, 6), vertex_pos(y, 4), vertex_pos(z, 3)]
        got = oracle.interp_column(f, p)
        np.testing.assert_allclose(got, f[:, z, y, x], rtol=0, atol=2e-6)


def test_affine_field_is_reproduced():
    # member m: e = a_m x + b_m y + c_m z + d_m at the vertices; trilinear
    # interpolation of an affine function is that function
    M, Z, Y, X = 4, 5, 7, 9
    rng = np.random.default_rng(2)
    coef = rng.normal(size=(M, 4))
    g = [np.array([vertex_pos(i, n) for i in range(n)]) for n in (X, Y, Z)]
    z, y, x = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    f = np.stack([c[0] * x + c[1] * y + c[2] * z + c[3] for c in coef]).astype(np.float32)
    for _ in range(20):
        p = rng.uniform(-1, 1, 3).astype(np.float32)
        want = coef[:, :3] @ p.astype(np.float64) + coef[:, 3]
        np.testing.assert_allclose(oracle.interp_column(f, p), want, rtol=0, atol=1e-5)


def test_constant_field_and_clamping():
    f = np.full((3, 2, 2, 2), 1.25, np.float32)
    for p in ([0.3, -0.7, 0.1], [1.0, 1.0, 1.0], [-1.0, 0.0, 1.0], [2.0, -3.0, 0.5]):
        assert (oracle.interp_column(f, p) == 1.25).all()


def test_single_vertex_axis():
    rng = np.random.default_rng(3)
    f = rng.normal(size=(4, 1, 3, 3)).astype(np.float32)  # Z = 1
    got = oracle.interp_column(f, [vertex_pos(2, 3), vertex_pos(0, 3), 0.4])
    np.testing.assert_allclose(got, f[:, 0, 0, 2], atol=2e-6)
