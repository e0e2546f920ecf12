"""Pins for the ray-march oracle (Sec. 5 direct volume rendering / iso-surface,
Sec. 6.5 difference fields).  Each pin comes from a closed form of the
compositing integral, the geometry of a sphere, or an exact linearity."""
import math

import numpy as np
import pytest

import oracle

CAM = dict(eye=(0.0, 0.0, 4.0), target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fov_y_deg=30.0)


def test_constant_volume_closed_form():
    # centre ray along -z: t0 = 3, t1 = 5; samples t_k = 3 + (k + 1/2) step < 5, so
    # n = 2 / step samples; T = 1 - exp(-A step)^n, C = rgb T, black background
    a_len, step = 1.5, 0.02
    v = np.full((4, 5, 6), 0.25, np.float32)
    tf = np.array([[0.0, 0.0, 0.0, a_len], [1.0, 0.8, 0.4, a_len]])  # colour = 0.25 of the top
    img = oracle.render(v, None, width=9, height=9, step=step, mode=0, tf=tf, vmin=0.0, vmax=1.0,
                        **CAM)
    n = 100
    T = 1.0 - math.exp(-a_len * step) ** n
    np.testing.assert_allclose(img[4, 4], [0.25 * T, 0.2 * T, 0.1 * T, T], rtol=1e-12)


def test_miss_is_background():
    v = np.zeros((3, 3, 3), np.float32)
    bg = (0.1, 0.2, 0.3, 0.4)
    img = oracle.render(v, None, eye=(5.0, 5.0, 5.0), target=(6.0, 6.0, 6.0), up=(0.0, 1.0, 0.0),
                        fov_y_deg=10.0, width=4, height=4, step=0.01, mode=0,
                        tf=[[1, 1, 1, 5.0]], vmin=0.0, vmax=1.0, background=bg)
    assert (img == np.array(bg)).all()


def test_difference_field_is_linear():
    rng = np.random.default_rng(3)
    a = (rng.integers(-8, 8, size=(6, 7, 8)) * 0.25).astype(np.float32)
    b = (rng.integers(-8, 8, size=(6, 7, 8)) * 0.25).astype(np.float32)  # a - b exact in FP32
    tf = np.array([[0.0, 0.0, 1.0, 0.5], [1.0, 1.0, 1.0, 0.1], [1.0, 0.0, 0.0, 2.0]])
    kw = dict(width=17, height=13, step=0.013, mode=0, tf=tf, vmin=-3.0, vmax=3.0, **CAM)
    np.testing.assert_allclose(oracle.render(a, b, **kw), oracle.render(a - b, None, **kw),
                               atol=1e-12)


def _sphere_field(n):
    g = np.linspace(-1.0, 1.0, n)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.sqrt(x * x + y * y + z * z).astype(np.float32)


def test_iso_sphere_silhouette_and_shading():
    r, n, W = 0.6, 48, 129
    tf = np.array([[0.9, 0.6, 0.3, 1.0]])
    img = oracle.render(_sphere_field(n), None, width=W, height=W, step=0.004, mode=1, iso=r,
                        tf=tf, vmin=0.0, vmax=2.0, ambient=0.2, **CAM)
    hit = img[..., 3] == 1.0
    # the sphere subtends asin(r / 4) around the view axis
    rad_px = math.tan(math.asin(r / 4.0)) / math.tan(math.radians(15.0)) * (W / 2)
    assert hit.sum() == pytest.approx(math.pi * rad_px ** 2, rel=0.03)
    # the centre pixel sees the surface head-on: full Lambert term
    np.testing.assert_allclose(img[W // 2, W // 2, :3], tf[0, :3], atol=2e-3)
    # the rim is darker than the centre
    row = img[W // 2, :, 0]
    first = np.argmax(hit[W // 2])
    assert row[first] < 0.5 * row[W // 2]


def test_iso_no_crossing_is_background():
    v = np.full((4, 4, 4), 0.1, np.float32)
    img = oracle.render(v, None, width=5, height=5, step=0.05, mode=1, iso=0.5,
                        tf=[[1, 1, 1, 1.0]], vmin=0.0, vmax=1.0, **CAM)
    assert (img == 0.0).all()
