"""Seeded synthetic ensembles shaped like the paper's CSEns data (Sec. 6.1).

Input generation only: this package holds none of the method's arithmetic.  The
CPU oracle and the CUDA library are both fed from the arrays it returns, so the
two sides always read the same bytes.  The generator itself is plain C
(``synth.c``), compiled with gcc and OpenMP, because the paper-scale ensemble
(1000 members x 250 x 352 x 20 = 7.04 GB) is too slow to build in numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None

LATENT_NONE, LATENT_SINX, LATENT_THREE_MODES = 0, 1, 2
TRANSFORM_NONE, TRANSFORM_QUAD, TRANSFORM_ALTERNATING = 0, 1, 2

SEED = 20230705


class _Params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("stream", ctypes.c_int),
        ("sigma", ctypes.c_double * 3),
        ("latent_kind", ctypes.c_int),
        ("latent_period_x", ctypes.c_double),
        ("transform", ctypes.c_int),
        ("share", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` in-tree (gcc, OpenMP); returns its path."""
    src = os.path.join(_HERE, "synth.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "synth.h"))
    ):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.synth_field.restype = ctypes.c_int
            lib.synth_field.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_int64, ctypes.c_int64,
                                        ctypes.POINTER(_Params), ctypes.c_int]
            lib.synth_normal.restype = ctypes.c_double
            lib.synth_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            _lib = lib
    return _lib


@dataclass(frozen=True)
class Recipe:
    """One synthetic field: shape, smoothing, latent modes, transform, seed."""

    M: int
    Z: int
    Y: int
    X: int
    sigma: tuple = (0.0, 0.0, 0.0)  # (x, y, z) in vertices
    latent_kind: int = LATENT_NONE
    latent_period_x: float = 16.0
    transform: int = TRANSFORM_NONE
    seed: int = SEED
    stream: int = 0
    share: float = 0.0
    extra: dict = field(default_factory=dict, compare=False)

    @property
    def N(self) -> int:
        return self.Z * self.Y * self.X

    @property
    def nbytes(self) -> int:
        return self.M * self.N * 4


# The two exact-path workloads and the second (cross-variable) field.
TINY = Recipe(M=100, Z=4, Y=16, X=16, sigma=(3.0, 3.0, 1.0), latent_kind=LATENT_SINX,
              latent_period_x=16.0, transform=TRANSFORM_QUAD)
TINY_REF = (8, 8, 2)  # (x, y, z)
CSENS = Recipe(M=1000, Z=20, Y=352, X=250, sigma=(12.0, 12.0, 3.0),
               latent_kind=LATENT_THREE_MODES, transform=TRANSFORM_ALTERNATING)
CSENS_B = Recipe(M=1000, Z=20, Y=352, X=250, sigma=(12.0, 12.0, 3.0),
                 latent_kind=LATENT_THREE_MODES, transform=TRANSFORM_ALTERNATING,
                 stream=1, share=0.6)


def scaled(base: Recipe, **kw) -> Recipe:
    """A copy of ``base`` with some fields replaced (smaller grids for tests)."""
    d = dict(M=base.M, Z=base.Z, Y=base.Y, X=base.X, sigma=base.sigma,
             latent_kind=base.latent_kind, latent_period_x=base.latent_period_x,
             transform=base.transform, seed=base.seed, stream=base.stream, share=base.share)
    d.update(kw)
    return Recipe(**d)


def generate(recipe: Recipe, out: np.ndarray | None = None, nthreads: int = 0) -> np.ndarray:
    """Return the field as a C-contiguous float32 array of shape [M, Z, Y, X].

    ``out`` may be any writable C-contiguous float32 buffer of that shape (for
    instance a numpy view of pinned host memory)."""
    lib = _load()
    shape = (recipe.M, recipe.Z, recipe.Y, recipe.X)
    if out is None:
        out = np.empty(shape, dtype=np.float32)
    if out.dtype != np.float32 or not out.flags.c_contiguous or out.size != recipe.M * recipe.N:
        raise ValueError("out must be a C-contiguous float32 array of shape %r" % (shape,))
    p = _Params(recipe.seed, recipe.stream, (ctypes.c_double * 3)(*recipe.sigma),
                recipe.latent_kind, recipe.latent_period_x, recipe.transform, recipe.share)
    rc = lib.synth_field(out.ctypes.data, recipe.M, recipe.Z, recipe.Y, recipe.X,
                         ctypes.byref(p), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"synth_field failed with code {rc}")
    return out.reshape(shape)


def normal(seed: int, domain: int, counter: int) -> float:
    """One draw of the counter-based N(0,1) generator (for tests)."""
    return _load().synth_normal(seed, domain, counter)


def vertex_index(x: int, y: int, z: int, recipe: Recipe) -> int:
    """Flat vertex index v = (z*Y + y)*X + x."""
    return (z * recipe.Y + y) * recipe.X + x


def sample_vertices(recipe: Recipe, count: int, seed: int) -> np.ndarray:
    """``count`` distinct seeded vertex indices, sorted (uniform over the grid)."""
    rng = np.random.default_rng(seed)
    count = min(count, recipe.N)
    return np.sort(rng.choice(recipe.N, size=count, replace=False)).astype(np.int64)
