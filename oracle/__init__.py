"""CPU oracle for the dependence-volume hot path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  The CUDA
library never calls it and shares no code with it: the oracle has its own C++
source (``ndf_oracle.cpp``, ``ndf_net_oracle.cpp``), its own digamma table and
its own build.

Functions and the passages they follow:
  pearson / pearson_volume -- Sec. 3.1, Eq. 1 (FP64, two-pass, plain definition)
  ksg_pair / ksg_pairs /
  ksg_volume               -- Sec. 3.2 / Sec. 6.2: the cited KSG estimator,
                              algorithm 1, brute force (FP32 max-norm distances,
                              k-th order statistic by nth_element, linear-scan
                              strict counts, long-double digamma sum)
  digamma_int              -- psi(1) = -gamma, psi(n+1) = psi(n) + 1/n
  ndf_*, adam_step         -- Sec. 4: dense-grid NDF forward, L1 loss (Eq. 3), hand-written
                              backward, Adam update, all FP64
  hash_*                   -- Sec. 4.1-4.2: the paper's NDF architecture (hash grid, Fourier
                              features, Snake/SnakeAlt MLP encoders, product merge, decoder),
                              forward and hand-written backward in FP64 (hash_net_oracle.h)
  render                   -- Sec. 5 / Sec. 6.5: headless ray-march of a dependence volume
                              (DVR with a transfer function, iso-surface, difference of two
                              fields), FP64 per pixel (render_oracle.h has the definitions)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libndf_oracle.so")
_SOURCES = ["ndf_oracle.cpp", "ndf_net_oracle.cpp", "render_oracle.cpp", "hash_net_oracle.cpp"]
_HEADERS = ["ndf_oracle.h", "ndf_net_oracle.h", "render_oracle.h", "hash_net_oracle.h"]
_lock = threading.Lock()
_lib = None

_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def _existing(names):
    return [os.path.join(_HERE, n) for n in names if os.path.exists(os.path.join(_HERE, n))]


def build(force: bool = False) -> str:
    """Compile the oracle (g++ -O2, OpenMP, no fast-math, no FMA contraction)."""
    srcs = _existing(_SOURCES)
    deps = srcs + _existing(_HEADERS)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(p) for p in deps
    ):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class RenderCfg(ctypes.Structure):
    """Camera, ray step, mode and transfer function of the ray-march oracle."""

    _fields_ = [("eye", ctypes.c_double * 3), ("target", ctypes.c_double * 3),
                ("up", ctypes.c_double * 3), ("fov_y_deg", ctypes.c_double),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("step", ctypes.c_double),
                ("mode", ctypes.c_int32), ("iso", ctypes.c_double), ("vmin", ctypes.c_double),
                ("vmax", ctypes.c_double), ("background", ctypes.c_double * 4),
                ("ambient", ctypes.c_double), ("n_tf", ctypes.c_int32),
                ("tf", ctypes.POINTER(ctypes.c_double))]


class HashShape(ctypes.Structure):
    """Shape of the paper's NDF architecture (see hash_net_oracle.h)."""

    _fields_ = [(n, ctypes.c_int32) for n in ("levels", "base_res", "log2_table", "feat", "n_freq",
                                               "width", "enc_layers", "dec_layers", "n_enc",
                                               "measure", "act", "merge")]


def hash_shape(**kw):
    """Fields of HashShape by name; merge defaults to 0 (product)."""
    s = HashShape()
    for n, _ in HashShape._fields_:
        setattr(s, n, int(kw.get(n, 0) if n == "merge" else kw[n]))
    return s


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.oracle_pearson.restype = ctypes.c_double
            lib.oracle_pearson.argtypes = [_f32p, _f32p, ctypes.c_int64]
            lib.oracle_pearson_volume.restype = ctypes.c_int
            lib.oracle_pearson_volume.argtypes = [_f32p, _f32p, ctypes.c_int64, ctypes.c_int64,
                                                  ctypes.c_int64, _i64p, ctypes.c_int64, _f64p,
                                                  ctypes.c_int]
            lib.oracle_digamma_int.restype = ctypes.c_double
            lib.oracle_digamma_int.argtypes = [ctypes.c_int64]
            lib.oracle_ksg_pair.restype = ctypes.c_double
            lib.oracle_ksg_pair.argtypes = [_f32p, _f32p, ctypes.c_int64, ctypes.c_int, _f32p,
                                            _i32p, _i32p]
            lib.oracle_ksg_volume.restype = ctypes.c_int
            lib.oracle_ksg_volume.argtypes = [_f32p, _f32p, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.c_int64, ctypes.c_int, _i64p, ctypes.c_int64,
                                              _f64p, ctypes.c_int]
            lib.oracle_ksg_pairs.restype = ctypes.c_int
            lib.oracle_ksg_pairs.argtypes = [_f32p, _f32p, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int64, ctypes.c_int, _i64p, ctypes.c_int64,
                                             _f32p, _i32p, _i32p, _f64p, ctypes.c_int]
            lib.oracle_ksg2_pair.restype = ctypes.c_double
            lib.oracle_ksg2_pair.argtypes = [_f32p, _f32p, ctypes.c_int64, ctypes.c_int, _f32p,
                                             _f32p, _i32p, _i32p]
            lib.oracle_ksg2_volume.restype = ctypes.c_int
            lib.oracle_ksg2_volume.argtypes = lib.oracle_ksg_volume.argtypes
            lib.oracle_interp_column.restype = ctypes.c_int
            lib.oracle_interp_column.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int64,
                                                 ctypes.c_int64, ctypes.c_int64, _f32p, _f32p]
            lib.oracle_hash_param_count.restype = ctypes.c_int64
            lib.oracle_hash_param_count.argtypes = [ctypes.POINTER(HashShape)]
            lib.oracle_hash_forward.restype = ctypes.c_int
            lib.oracle_hash_forward.argtypes = [ctypes.POINTER(HashShape), _f64p, ctypes.c_int64,
                                                _f64p, _f64p, _f64p]
            lib.oracle_hash_forward_bf16.restype = ctypes.c_int
            lib.oracle_hash_forward_bf16.argtypes = lib.oracle_hash_forward.argtypes
            lib.oracle_bf16_round.restype = ctypes.c_double
            lib.oracle_bf16_round.argtypes = [ctypes.c_double]
            lib.oracle_hash_loss_grad.restype = ctypes.c_int
            lib.oracle_hash_loss_grad.argtypes = [ctypes.POINTER(HashShape), _f64p, ctypes.c_int64,
                                                  _f64p, _f64p, _f64p, _f64p, _f64p]
            lib.oracle_threads.restype = ctypes.c_int
            lib.oracle_threads.argtypes = [ctypes.c_int]
            lib.oracle_render.restype = ctypes.c_int
            lib.oracle_render.argtypes = [_f32p, _f32p, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int64, ctypes.POINTER(RenderCfg), _f64p,
                                          ctypes.c_int]
            _lib = lib
    return _lib


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(_f32p)


def threads(n: int = 0) -> int:
    """Threads the oracle's parallel loops use for a request of ``n`` (0 = all)."""
    return _load().oracle_threads(int(n))


def pearson(x, y) -> float:
    """Eq. 1 for one pair of samples (FP64)."""
    x, px = _f32(x)
    y, py = _f32(y)
    if x.shape != y.shape or x.ndim != 1:
        raise ValueError("x and y must be 1-D of equal length")
    return _load().oracle_pearson(px, py, x.shape[0])


def _field2d(field):
    f = np.ascontiguousarray(field, dtype=np.float32)
    M = f.shape[0]
    return f.reshape(M, -1), M


def pearson_volume(ref_field, q_field, ref_idx: int, verts=None, nthreads: int = 0) -> np.ndarray:
    """r(reference vertex of ref_field, v of q_field) for all / selected v."""
    rf, M = _field2d(ref_field)
    qf, Mq = _field2d(q_field)
    if Mq != M or rf.shape != qf.shape:
        raise ValueError("fields differ in shape")
    N = rf.shape[1]
    if verts is None:
        out = np.empty(N, dtype=np.float64)
        vp, nv = None, 0
    else:
        verts = np.ascontiguousarray(verts, dtype=np.int64)
        out = np.empty(verts.shape[0], dtype=np.float64)
        vp, nv = verts.ctypes.data_as(_i64p), verts.shape[0]
    rc = _load().oracle_pearson_volume(rf.ctypes.data_as(_f32p), qf.ctypes.data_as(_f32p), M, N,
                                       int(ref_idx), vp, nv, out.ctypes.data_as(_f64p),
                                       int(nthreads))
    if rc != 0:
        raise ValueError("oracle_pearson_volume: bad arguments")
    return out


def digamma_int(n: int) -> float:
    return _load().oracle_digamma_int(int(n))


def ksg_pair(x, y, k: int):
    """KSG algorithm 1 on one pair: returns (mi, eps[M], nx[M], ny[M])."""
    x, px = _f32(x)
    y, py = _f32(y)
    if x.shape != y.shape or x.ndim != 1:
        raise ValueError("x and y must be 1-D of equal length")
    M = x.shape[0]
    eps = np.empty(M, dtype=np.float32)
    nx = np.empty(M, dtype=np.int32)
    ny = np.empty(M, dtype=np.int32)
    mi = _load().oracle_ksg_pair(px, py, M, int(k), eps.ctypes.data_as(_f32p),
                                 nx.ctypes.data_as(_i32p), ny.ctypes.data_as(_i32p))
    if np.isnan(mi):
        raise ValueError("oracle_ksg_pair: bad arguments (need 1 <= k < M)")
    return mi, eps, nx, ny


def ksg_volume(ref_field, q_field, ref_idx: int, k: int, verts=None, nthreads: int = 0):
    """KSG MI (reference vertex of ref_field, v of q_field) for all / selected v."""
    rf, M = _field2d(ref_field)
    qf, Mq = _field2d(q_field)
    if Mq != M or rf.shape != qf.shape:
        raise ValueError("fields differ in shape")
    N = rf.shape[1]
    if verts is None:
        out = np.empty(N, dtype=np.float64)
        vp, nv = None, 0
    else:
        verts = np.ascontiguousarray(verts, dtype=np.int64)
        out = np.empty(verts.shape[0], dtype=np.float64)
        vp, nv = verts.ctypes.data_as(_i64p), verts.shape[0]
    rc = _load().oracle_ksg_volume(rf.ctypes.data_as(_f32p), qf.ctypes.data_as(_f32p), M, N,
                                   int(ref_idx), int(k), vp, nv, out.ctypes.data_as(_f64p),
                                   int(nthreads))
    if rc != 0:
        raise ValueError("oracle_ksg_volume: bad arguments")
    return out


def ksg_pairs(ref_field, q_field, ref_idx: int, k: int, verts, nthreads: int = 0):
    """ksg_pair of the reference column against each listed query column, in
    parallel: returns (mi[n], eps[n][M], nx[n][M], ny[n][M])."""
    rf, M = _field2d(ref_field)
    qf, Mq = _field2d(q_field)
    if Mq != M or rf.shape != qf.shape:
        raise ValueError("fields differ in shape")
    N = rf.shape[1]
    verts = np.ascontiguousarray(verts, dtype=np.int64)
    n = verts.shape[0]
    eps = np.empty((n, M), dtype=np.float32)
    nx = np.empty((n, M), dtype=np.int32)
    ny = np.empty((n, M), dtype=np.int32)
    mi = np.empty(n, dtype=np.float64)
    rc = _load().oracle_ksg_pairs(rf.ctypes.data_as(_f32p), qf.ctypes.data_as(_f32p), M, N,
                                  int(ref_idx), int(k), verts.ctypes.data_as(_i64p), n,
                                  eps.ctypes.data_as(_f32p), nx.ctypes.data_as(_i32p),
                                  ny.ctypes.data_as(_i32p), mi.ctypes.data_as(_f64p),
                                  int(nthreads))
    if rc != 0:
        raise ValueError("oracle_ksg_pairs: bad arguments")
    return mi, eps, nx, ny


def ksg2_pair(x, y, k: int):
    """KSG algorithm 2 on one pair: returns (mi, ex[M], ey[M], nx[M], ny[M])."""
    x, px = _f32(x)
    y, py = _f32(y)
    if x.shape != y.shape or x.ndim != 1:
        raise ValueError("x and y must be 1-D of equal length")
    M = x.shape[0]
    ex = np.empty(M, dtype=np.float32)
    ey = np.empty(M, dtype=np.float32)
    nx = np.empty(M, dtype=np.int32)
    ny = np.empty(M, dtype=np.int32)
    mi = _load().oracle_ksg2_pair(px, py, M, int(k), ex.ctypes.data_as(_f32p),
                                  ey.ctypes.data_as(_f32p), nx.ctypes.data_as(_i32p),
                                  ny.ctypes.data_as(_i32p))
    if np.isnan(mi):
        raise ValueError("oracle_ksg2_pair: bad arguments (need 1 <= k < M)")
    return mi, ex, ey, nx, ny


def ksg2_volume(ref_field, q_field, ref_idx: int, k: int, verts=None, nthreads: int = 0):
    """KSG algorithm-2 MI (reference vertex of ref_field, v of q_field)."""
    rf, M = _field2d(ref_field)
    qf, Mq = _field2d(q_field)
    if Mq != M or rf.shape != qf.shape:
        raise ValueError("fields differ in shape")
    N = rf.shape[1]
    if verts is None:
        out = np.empty(N, dtype=np.float64)
        vp, nv = None, 0
    else:
        verts = np.ascontiguousarray(verts, dtype=np.int64)
        out = np.empty(verts.shape[0], dtype=np.float64)
        vp, nv = verts.ctypes.data_as(_i64p), verts.shape[0]
    rc = _load().oracle_ksg2_volume(rf.ctypes.data_as(_f32p), qf.ctypes.data_as(_f32p), M, N,
                                    int(ref_idx), int(k), vp, nv, out.ctypes.data_as(_f64p),
                                    int(nthreads))
    if rc != 0:
        raise ValueError("oracle_ksg2_volume: bad arguments")
    return out


def interp_column(field, p):
    """Member column of field[M][Z][Y][X] at the continuous position p (FP32 trilinear,
    see oracle_interp_column)."""
    f = np.ascontiguousarray(field, dtype=np.float32)
    M, Z, Y, X = f.shape
    pp = np.ascontiguousarray(p, dtype=np.float32).reshape(3)
    out = np.empty(M, dtype=np.float32)
    rc = _load().oracle_interp_column(f.ctypes.data_as(_f32p), M, X, Y, Z,
                                      pp.ctypes.data_as(_f32p), out.ctypes.data_as(_f32p))
    if rc != 0:
        raise ValueError("oracle_interp_column: bad arguments")
    return out


def hash_param_count(shape) -> int:
    n = _load().oracle_hash_param_count(ctypes.byref(shape))
    if n < 0:
        raise ValueError("bad hash-network shape")
    return int(n)


def hash_forward(shape, params, pr, pq):
    p = np.ascontiguousarray(params, dtype=np.float64)
    a = np.ascontiguousarray(pr, dtype=np.float64).reshape(-1, 3)
    b = np.ascontiguousarray(pq, dtype=np.float64).reshape(-1, 3)
    out = np.empty(a.shape[0], dtype=np.float64)
    rc = _load().oracle_hash_forward(ctypes.byref(shape), p.ctypes.data_as(_f64p), a.shape[0],
                                     a.ctypes.data_as(_f64p), b.ctypes.data_as(_f64p),
                                     out.ctypes.data_as(_f64p))
    if rc != 0:
        raise ValueError("oracle_hash_forward: bad arguments")
    return out


def hash_forward_bf16(shape, params, pr, pq):
    """hash_forward with BF16 operands in every layer's product but the output layer's."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    a = np.ascontiguousarray(pr, dtype=np.float64).reshape(-1, 3)
    b = np.ascontiguousarray(pq, dtype=np.float64).reshape(-1, 3)
    out = np.empty(a.shape[0], dtype=np.float64)
    rc = _load().oracle_hash_forward_bf16(ctypes.byref(shape), p.ctypes.data_as(_f64p), a.shape[0],
                                          a.ctypes.data_as(_f64p), b.ctypes.data_as(_f64p),
                                          out.ctypes.data_as(_f64p))
    if rc != 0:
        raise ValueError("oracle_hash_forward_bf16: bad arguments")
    return out


def bf16_round(x) -> float:
    return float(_load().oracle_bf16_round(float(x)))


def hash_loss_grad(shape, params, pr, pq, target):
    p = np.ascontiguousarray(params, dtype=np.float64)
    a = np.ascontiguousarray(pr, dtype=np.float64).reshape(-1, 3)
    b = np.ascontiguousarray(pq, dtype=np.float64).reshape(-1, 3)
    t = np.ascontiguousarray(target, dtype=np.float64)
    loss = ctypes.c_double(0.0)
    grad = np.empty(p.shape[0], dtype=np.float64)
    rc = _load().oracle_hash_loss_grad(ctypes.byref(shape), p.ctypes.data_as(_f64p), a.shape[0],
                                       a.ctypes.data_as(_f64p), b.ctypes.data_as(_f64p),
                                       t.ctypes.data_as(_f64p), ctypes.byref(loss),
                                       grad.ctypes.data_as(_f64p))
    if rc != 0:
        raise ValueError("oracle_hash_loss_grad: bad arguments")
    return loss.value, grad


def render(vol_a, vol_b, *, eye, target, up, fov_y_deg, width, height, step, mode, tf,
           vmin, vmax, iso=0.0, background=(0.0, 0.0, 0.0, 0.0), ambient=0.2, nthreads=0):
    """Ray-march the volume(s) float[Z][Y][X] (vol_b may be None: the difference
    vol_a - vol_b is rendered otherwise).  mode 0 = DVR, 1 = iso-surface.  tf is
    an [n][4] RGBA table over [vmin, vmax] (A = opacity per unit length).
    Returns float64 [height][width][4]."""
    a = np.ascontiguousarray(vol_a, dtype=np.float32)
    if a.ndim != 3:
        raise ValueError("volume must be [Z][Y][X]")
    b = None if vol_b is None else np.ascontiguousarray(vol_b, dtype=np.float32)
    if b is not None and b.shape != a.shape:
        raise ValueError("volumes differ in shape")
    tfa = np.ascontiguousarray(tf, dtype=np.float64)
    c = RenderCfg()
    c.eye[:], c.target[:], c.up[:] = list(eye), list(target), list(up)
    c.fov_y_deg, c.width, c.height, c.step = fov_y_deg, width, height, step
    c.mode, c.iso, c.vmin, c.vmax = mode, iso, vmin, vmax
    c.background[:] = list(background)
    c.ambient, c.n_tf = ambient, tfa.shape[0]
    c.tf = tfa.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    out = np.empty((height, width, 4), dtype=np.float64)
    Z, Y, X = a.shape
    rc = _load().oracle_render(a.ctypes.data_as(_f32p),
                               None if b is None else b.ctypes.data_as(_f32p), X, Y, Z,
                               ctypes.byref(c), out.ctypes.data_as(_f64p), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_render: bad arguments")
    return out


# ---------------------------------------------------------------- neural dependence field
class NetShape(ctypes.Structure):
    """Shape of the dense-grid NDF (see ndf_net_oracle.h)."""

    _fields_ = [("levels", ctypes.c_int), ("res", ctypes.c_int * 8), ("feat", ctypes.c_int),
                ("hidden", ctypes.c_int), ("measure", ctypes.c_int)]


def net_shape(res, feat, hidden, measure):
    s = NetShape()
    s.levels = len(res)
    for i, r in enumerate(res):
        s.res[i] = int(r)
    s.feat = int(feat)
    s.hidden = int(hidden)
    s.measure = int(measure)
    return s


def _net_lib():
    lib = _load()
    if not hasattr(lib, "_net_ready"):
        sp = ctypes.POINTER(NetShape)
        lib.oracle_ndf_param_count.restype = ctypes.c_int64
        lib.oracle_ndf_param_count.argtypes = [sp]
        lib.oracle_ndf_encode.restype = None
        lib.oracle_ndf_encode.argtypes = [sp, _f64p, _f64p, _f64p]
        lib.oracle_ndf_forward.restype = None
        lib.oracle_ndf_forward.argtypes = [sp, _f64p, ctypes.c_int64, _f64p, _f64p, _f64p]
        lib.oracle_ndf_loss_grad.restype = ctypes.c_double
        lib.oracle_ndf_loss_grad.argtypes = [sp, _f64p, ctypes.c_int64, _f64p, _f64p, _f64p,
                                             _f64p]
        lib.oracle_ndf_loss_grad_abs.restype = ctypes.c_double
        lib.oracle_ndf_loss_grad_abs.argtypes = [sp, _f64p, ctypes.c_int64, _f64p, _f64p, _f64p,
                                                 _f64p, _f64p]
        lib.oracle_adam_step.restype = None
        lib.oracle_adam_step.argtypes = [ctypes.c_int64, _f64p, _f64p, _f64p, _f64p,
                                         ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double]
        lib._net_ready = True
    return lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_f64p)


def ndf_param_count(shape) -> int:
    return int(_net_lib().oracle_ndf_param_count(ctypes.byref(shape)))


def ndf_encode(shape, params, p):
    params, pp = _d(params)
    p, ppos = _d(p)
    out = np.empty(shape.levels * shape.feat)
    _net_lib().oracle_ndf_encode(ctypes.byref(shape), pp, ppos, out.ctypes.data_as(_f64p))
    return out


def ndf_forward(shape, params, pr, pq):
    params, pp = _d(params)
    pr, a = _d(pr)
    pq, b = _d(pq)
    B = pr.shape[0]
    y = np.empty(B)
    _net_lib().oracle_ndf_forward(ctypes.byref(shape), pp, B, a, b, y.ctypes.data_as(_f64p))
    return y


def ndf_loss_grad(shape, params, pr, pq, target, want_grad=True):
    params, pp = _d(params)
    pr, a = _d(pr)
    pq, b = _d(pq)
    target, t = _d(target)
    grad = np.empty(params.shape[0]) if want_grad else None
    loss = _net_lib().oracle_ndf_loss_grad(ctypes.byref(shape), pp, pr.shape[0], a, b, t,
                                           grad.ctypes.data_as(_f64p) if want_grad else None)
    return loss, grad


def ndf_loss_grad_abs(shape, params, pr, pq, target):
    """(loss, grad, gabs): gabs = mean over samples of |per-sample gradient|."""
    params, pp = _d(params)
    pr, a = _d(pr)
    pq, b = _d(pq)
    target, t = _d(target)
    grad = np.empty(params.shape[0])
    gabs = np.empty(params.shape[0])
    loss = _net_lib().oracle_ndf_loss_grad_abs(ctypes.byref(shape), pp, pr.shape[0], a, b, t,
                                               grad.ctypes.data_as(_f64p),
                                               gabs.ctypes.data_as(_f64p))
    return loss, grad, gabs


def adam_step(params, grad, m, v, t, lr=3e-4, beta1=0.9, beta2=0.999, eps=1e-8):
    """In place on float64 arrays (params, m, v); returns nothing."""
    for arr in (params, grad, m, v):
        assert arr.dtype == np.float64 and arr.flags.c_contiguous
    _net_lib().oracle_adam_step(params.shape[0], params.ctypes.data_as(_f64p),
                                grad.ctypes.data_as(_f64p), m.ctypes.data_as(_f64p),
                                v.ctypes.data_as(_f64p), int(t), lr, beta1, beta2, eps)
