"""Thin ctypes binding of libndf.so: the C-ABI calls under the same names.

Argument marshalling only -- every step of the computation runs in the
library's CUDA kernels.  Arrays may be torch tensors (host or CUDA), numpy
arrays or raw integer addresses; the library itself detects host vs device
memory.  A non-zero status raises :class:`NdfError` carrying the library's
last-error string.  There is no CPU fallback: if ``libndf.so`` has not been
built, importing this module raises ``ImportError``.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libndf.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -m paper_2307_02203_gb300.build` "
        "(the library has no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

NDF_OK, NDF_ERR_ARG, NDF_ERR_OOM, NDF_ERR_CUDA = 0, -1, -2, -3
NDF_ERR_TIMEOUT, NDF_ERR_STATE, NDF_ERR_IO = -4, -5, -6
NDF_PREC_FP32, NDF_PREC_BF16X3, NDF_PREC_TF32 = 0, 1, 2
NDF_MEASURE_PEARSON, NDF_MEASURE_MI_KSG = 0, 1
NDF_KSG_BRUTE, NDF_KSG_PRUNED, NDF_KSG_BLOCK, NDF_KSG_LANES = 0, 1, 2, 3
NDF_RENDER_DVR, NDF_RENDER_ISO = 0, 1
NDF_ACT_RELU, NDF_ACT_SNAKE, NDF_ACT_SNAKEALT = 0, 1, 2
NDF_MERGE_PRODUCT, NDF_MERGE_SUM, NDF_MERGE_ABSDIFF, NDF_MERGE_CONCAT = 0, 1, 2, 3
NDF_HASH_DECODE_FP32, NDF_HASH_DECODE_TC = 0, 1


class HashArch(ctypes.Structure):
    """ndf_hash_arch (include/ndf.h); fill with ndf_hash_arch_default()."""

    _fields_ = [(n, ctypes.c_int32) for n in ("levels", "base_res", "log2_table", "feat", "n_freq",
                                               "width", "enc_layers", "dec_layers", "act", "merge")]


class RenderCfg(ctypes.Structure):
    """ndf_render_cfg (include/ndf.h)."""

    _fields_ = [("eye", ctypes.c_float * 3), ("target", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("fov_y_deg", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("step", ctypes.c_float),
                ("mode", ctypes.c_int32), ("iso", ctypes.c_float), ("vmin", ctypes.c_float),
                ("vmax", ctypes.c_float), ("background", ctypes.c_float * 4),
                ("ambient", ctypes.c_float), ("n_tf", ctypes.c_int32),
                ("tf", ctypes.POINTER(ctypes.c_float))]

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


class NdfError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: {_lib.ndf_status_str(status).decode()} ({status}): {detail}")


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("ndf_status_str", ctypes.c_char_p, [ctypes.c_int])
_sig("ndf_last_error", ctypes.c_char_p, [_vp])
_sig("ndf_create", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _vp])
_sig("ndf_destroy", None, [_vp])
_sig("ndf_set_stream", ctypes.c_int, [_vp, _vp])
_sig("ndf_synchronize", ctypes.c_int, [_vp])
_sig("ndf_launch_count", ctypes.c_uint64, [_vp])
_sig("ndf_index", _i64, [_i64, _i64, _i64, _i64, _i64, _i64])
_sig("ndf_load_ensemble", ctypes.c_int, [_vp, _vp, _i64, _i64, _i64, _i64,
                                         ctypes.POINTER(ctypes.c_int)])
_sig("ndf_load_and_compute", ctypes.c_int, [_vp, _vp, _i64, _i64, _i64, _i64, _i64, ctypes.c_int,
                                            _vp, _vp, ctypes.POINTER(ctypes.c_int)])
_sig("ndf_free_ensemble", ctypes.c_int, [_vp, ctypes.c_int])
_sig("ndf_trim_cache", ctypes.c_int, [_vp])
_sig("ndf_selftest_timeout", ctypes.c_int, [_vp])
_sig("ndf_field_shape", ctypes.c_int, [_vp, ctypes.c_int] + [ctypes.POINTER(_i64)] * 4)
_sig("ndf_field_stats", ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp])
_sig("ndf_field_sorted_columns", ctypes.c_int, [_vp, ctypes.c_int, _i64, _i64, _vp])
_sig("ndf_pearson", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _i64, _vp])
_sig("ndf_mi_ksg", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _i64, ctypes.c_int, _vp])
_sig("ndf_mi_ksg2", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _i64, ctypes.c_int, _vp])
_sig("ndf_sample_triples", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, _i64, ctypes.c_uint64, _vp, _vp, _vp])
_sig("ndf_render_volume", ctypes.c_int, [_vp, _vp, _vp, _i64, _i64, _i64, _vp, _vp])
_sig("ndf_hash_arch_default", None, [_vp])
_sig("ndf_hash_model_create", ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                             _i64, _i64, _i64, ctypes.POINTER(_vp)])
_sig("ndf_hash_model_free", None, [_vp])
_sig("ndf_hash_model_param_count", _i64, [_vp])
_sig("ndf_hash_model_get_params", ctypes.c_int, [_vp, _vp])
_sig("ndf_hash_model_set_params", ctypes.c_int, [_vp, _vp])
_sig("ndf_hash_model_forward", ctypes.c_int, [_vp, _vp, _vp, _i64, _vp])
_sig("ndf_hash_model_step", ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, ctypes.c_float, ctypes.c_int,
                                           _vp, ctypes.POINTER(ctypes.c_double)])
_sig("ndf_hash_train", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      _vp, _vp, ctypes.POINTER(_vp)])
_sig("ndf_hash_model_info", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(_i64)])
_sig("ndf_hash_infer", ctypes.c_int, [_vp, _i64, _vp])
_sig("ndf_hash_infer_batch", ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp])
_sig("ndf_hash_set_decode", ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32])
_sig("ndf_hash_get_decode", ctypes.c_int32, [_vp])
_sig("ndf_pearson_batch", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int,
                                         ctypes.c_int, _vp])
_sig("ndf_set_ksg_algorithm", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int])
_sig("ndf_ksg_set_schedule", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int])
_sig("ndf_ksg_take_eval_count", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64)])
_sig("ndf_mi_ksg_batch", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int,
                                        ctypes.c_int, _vp])
_sig("ndf_ksg_autotune_search", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int)])
_sig("ndf_ksg_autotune", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)])
_sig("ndf_pearson_noalloc", ctypes.c_int, [_vp, _vp, _i64, _i64, _i64, _vp, _vp])
_sig("ndf_field_column", ctypes.c_int, [_vp, ctypes.c_int, _i64, _vp])
_sig("ndf_pearson_column", ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp])
_sig("ndf_mi_ksg_column", ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp])
_sig("ndf_noalloc_pointer_usable", ctypes.c_int, [ctypes.c_int] * 4)
_sig("ndf_ksg_debug_pair", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _i64, _i64,
                                          ctypes.c_int, _vp, _vp, _vp, _vp])
_sig("ndf_ksg2_debug_pair", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _i64, _i64,
                                           ctypes.c_int, _vp, _vp, _vp, _vp, _vp])


class TrainCfg(ctypes.Structure):
    """ndf_train_cfg (see include/ndf.h); fill with ndf_train_cfg_default()."""

    _fields_ = [("res", ctypes.c_int * 4), ("n_triples", _i64), ("batch", _i64),
                ("refs_per_group", _i64), ("queries_per_group", _i64), ("max_passes", ctypes.c_int),
                ("patience", ctypes.c_int), ("max_decays", ctypes.c_int), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("time_budget_s", ctypes.c_double),
                ("continuous", ctypes.c_int32), ("hash_tf32", ctypes.c_int32)]


class ModelInfo(ctypes.Structure):
    """ndf_model_info_t (see include/ndf.h)."""

    _fields_ = [("measure", ctypes.c_int), ("res", ctypes.c_int * 4), ("X", _i64), ("Y", _i64),
                ("Z", _i64), ("param_count", _i64), ("grid_params", _i64),
                ("network_bytes", _i64), ("training_bytes", _i64), ("adam_steps", _i64),
                ("passes", ctypes.c_int), ("last_loss", ctypes.c_double), ("n_triples", _i64),
                ("gen_seconds", ctypes.c_double), ("train_seconds", ctypes.c_double)]

    def as_dict(self):
        d = {n: getattr(self, n) for n, _ in self._fields_}
        d["res"] = list(self.res)
        return d


_sig("ndf_train_cfg_default", None, [ctypes.POINTER(TrainCfg)])
_sig("ndf_train", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(TrainCfg), ctypes.POINTER(_vp)])
_sig("ndf_infer", ctypes.c_int, [_vp, _i64, _vp])
_sig("ndf_infer_batch", ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp])
_sig("ndf_model_save", ctypes.c_int, [_vp, ctypes.c_char_p])
_sig("ndf_model_load", ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.POINTER(_vp)])
_sig("ndf_model_free", None, [_vp])
_sig("ndf_model_info", ctypes.c_int, [_vp, ctypes.POINTER(ModelInfo)])
_sig("ndf_model_create", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                        ctypes.c_uint64, _i64, _i64, _i64, ctypes.POINTER(_vp)])
_sig("ndf_model_param_count", _i64, [_vp])
_sig("ndf_model_get_params", ctypes.c_int, [_vp, _vp])
_sig("ndf_model_set_params", ctypes.c_int, [_vp, _vp])
_sig("ndf_model_step", ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, ctypes.c_float, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_double), _vp])
_sig("ndf_model_forward", ctypes.c_int, [_vp, _vp, _vp, _i64, _vp])


def _addr(x):
    """Address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):  # torch.Tensor
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):  # numpy
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _check(ctx, st, where):
    if st != NDF_OK:
        detail = _lib.ndf_last_error(ctx).decode() if ctx else ""
        raise NdfError(st, where, detail)


def ndf_status_str(status: int) -> str:
    return _lib.ndf_status_str(status).decode()


def ndf_last_error(ctx) -> str:
    return _lib.ndf_last_error(ctx).decode()


def ndf_create(device: int = 0, cuda_stream=None):
    """Returns an opaque context handle; ``cuda_stream`` is a raw cudaStream_t (int) or None."""
    h = _vp()
    st = _lib.ndf_create(ctypes.byref(h), int(device), cuda_stream)
    if st != NDF_OK:
        raise NdfError(st, "ndf_create", "no usable sm_103 device" if st == NDF_ERR_CUDA else "")
    return h


def ndf_destroy(ctx) -> None:
    _lib.ndf_destroy(ctx)


def ndf_set_stream(ctx, cuda_stream=None) -> None:
    _check(ctx, _lib.ndf_set_stream(ctx, cuda_stream), "ndf_set_stream")


def ndf_synchronize(ctx) -> None:
    _check(ctx, _lib.ndf_synchronize(ctx), "ndf_synchronize")


def ndf_launch_count(ctx) -> int:
    return int(_lib.ndf_launch_count(ctx))


def ndf_index(x, y, z, X, Y, Z) -> int:
    return int(_lib.ndf_index(x, y, z, X, Y, Z))


def ndf_load_ensemble(ctx, field, M, Z, Y, X) -> int:
    fid = ctypes.c_int(-1)
    _check(ctx, _lib.ndf_load_ensemble(ctx, _addr(field), M, Z, Y, X, ctypes.byref(fid)),
           "ndf_load_ensemble")
    return fid.value


def ndf_load_and_compute(ctx, field, M, Z, Y, X, ref_idx: int, k: int, pearson_out=None,
                         mi_out=None) -> int:
    """Load + Pearson + KSG-MI of one reference, the upload pipelined with the search."""
    fid = ctypes.c_int(-1)
    _check(ctx, _lib.ndf_load_and_compute(ctx, _addr(field), M, Z, Y, X, ref_idx, k,
                                          None if pearson_out is None else _addr(pearson_out),
                                          None if mi_out is None else _addr(mi_out),
                                          ctypes.byref(fid)), "ndf_load_and_compute")
    return fid.value


def ndf_free_ensemble(ctx, field_id: int) -> None:
    _check(ctx, _lib.ndf_free_ensemble(ctx, field_id), "ndf_free_ensemble")


def ndf_selftest_timeout(ctx) -> int:
    """Status of the bounded-wait self-test (NDF_ERR_TIMEOUT when the path works)."""
    return int(_lib.ndf_selftest_timeout(ctx))


def ndf_trim_cache(ctx) -> None:
    _check(ctx, _lib.ndf_trim_cache(ctx), "ndf_trim_cache")


def ndf_field_shape(ctx, field_id: int):
    v = [_i64() for _ in range(4)]
    _check(ctx, _lib.ndf_field_shape(ctx, field_id, *[ctypes.byref(t) for t in v]),
           "ndf_field_shape")
    return tuple(t.value for t in v)  # (M, Z, Y, X)


def ndf_field_stats(ctx, field_id: int, mean_out, inv_norm_out) -> None:
    _check(ctx, _lib.ndf_field_stats(ctx, field_id, _addr(mean_out), _addr(inv_norm_out)),
           "ndf_field_stats")


def ndf_field_sorted_columns(ctx, field_id: int, v_begin: int, v_end: int, out) -> None:
    """out: [M][v_end - v_begin] floats (host or device), each vertex's members ascending."""
    _check(ctx, _lib.ndf_field_sorted_columns(ctx, field_id, v_begin, v_end, _addr(out)),
           "ndf_field_sorted_columns")


def ndf_pearson(ctx, ref_field: int, query_field: int, ref_idx: int, out) -> None:
    _check(ctx, _lib.ndf_pearson(ctx, ref_field, query_field, ref_idx, _addr(out)), "ndf_pearson")


def ndf_pearson_batch(ctx, ref_field: int, query_field: int, ref_idx, prec: int, out) -> None:
    """ref_idx: sequence of flat vertex indices (host); out: [R][N] floats."""
    import numpy as _np

    refs = _np.ascontiguousarray(_np.asarray(ref_idx, dtype=_np.int64))
    _check(ctx, _lib.ndf_pearson_batch(ctx, ref_field, query_field, refs.ctypes.data,
                                       int(refs.shape[0]), int(prec), _addr(out)),
           "ndf_pearson_batch")


def ndf_mi_ksg(ctx, ref_field: int, query_field: int, ref_idx: int, k: int, out) -> None:
    _check(ctx, _lib.ndf_mi_ksg(ctx, ref_field, query_field, ref_idx, k, _addr(out)),
           "ndf_mi_ksg")


def ndf_mi_ksg2(ctx, ref_field: int, query_field: int, ref_idx: int, k: int, out) -> None:
    _check(ctx, _lib.ndf_mi_ksg2(ctx, ref_field, query_field, ref_idx, k, _addr(out)),
           "ndf_mi_ksg2")


def ndf_set_ksg_algorithm(ctx, algorithm: int, count_evals: bool = False) -> None:
    _check(ctx, _lib.ndf_set_ksg_algorithm(ctx, int(algorithm), int(bool(count_evals))),
           "ndf_set_ksg_algorithm")


def ndf_ksg_set_schedule(ctx, switch_min: int, every: int = 1) -> None:
    _check(ctx, _lib.ndf_ksg_set_schedule(ctx, int(switch_min), int(every)), "ndf_ksg_set_schedule")


def ndf_ksg_take_eval_count(ctx) -> int:
    v = ctypes.c_uint64(0)
    _check(ctx, _lib.ndf_ksg_take_eval_count(ctx, ctypes.byref(v)), "ndf_ksg_take_eval_count")
    return int(v.value)


def ndf_mi_ksg_batch(ctx, ref_field: int, query_field: int, ref_idx, k: int, out) -> None:
    """ref_idx: a sequence of host indices, or an int64 CUDA tensor (device-resident
    indices: the call then enqueues no host copy and can be graph-captured)."""
    import numpy as _np

    if hasattr(ref_idx, "is_cuda") and ref_idx.is_cuda:
        if str(ref_idx.dtype) != "torch.int64":
            raise TypeError("device reference indices must be int64")
        ptr, R = _addr(ref_idx), int(ref_idx.numel())
    else:
        refs = _np.ascontiguousarray(_np.asarray(ref_idx, dtype=_np.int64))
        ptr, R = refs.ctypes.data, int(refs.shape[0])
    _check(ctx, _lib.ndf_mi_ksg_batch(ctx, ref_field, query_field, ptr, R, int(k), _addr(out)),
           "ndf_mi_ksg_batch")


def ndf_ksg_autotune_search(ctx, ref_field: int, query_field: int, k: int):
    """Sets the fastest exact search and lane schedule; returns (algorithm, switch_min, every)."""
    a, sw, ev = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(ctx, _lib.ndf_ksg_autotune_search(ctx, ref_field, query_field, k, ctypes.byref(a),
                                             ctypes.byref(sw), ctypes.byref(ev)),
           "ndf_ksg_autotune_search")
    return a.value, sw.value, ev.value


def ndf_ksg_autotune(ctx, ref_field: int, query_field: int, k: int):
    g = ctypes.c_int(0)
    t = ctypes.c_int(0)
    _check(ctx, _lib.ndf_ksg_autotune(ctx, ref_field, query_field, k, ctypes.byref(g),
                                      ctypes.byref(t)), "ndf_ksg_autotune")
    return g.value, t.value


def ndf_ksg_debug_pair(ctx, ref_field, query_field, ref_idx, query_idx, k, eps, nx, ny, mi) -> None:
    _check(ctx, _lib.ndf_ksg_debug_pair(ctx, ref_field, query_field, ref_idx, query_idx, k,
                                        _addr(eps), _addr(nx), _addr(ny), _addr(mi)),
           "ndf_ksg_debug_pair")


def ndf_ksg2_debug_pair(ctx, ref_field, query_field, ref_idx, query_idx, k, ex, ey, nx, ny,
                        mi) -> None:
    _check(ctx, _lib.ndf_ksg2_debug_pair(ctx, ref_field, query_field, ref_idx, query_idx, k,
                                         _addr(ex), _addr(ey), _addr(nx), _addr(ny), _addr(mi)),
           "ndf_ksg2_debug_pair")


def ndf_render_volume(ctx, vol_a, vol_b, X: int, Y: int, Z: int, out, *, eye, target, up,
                      fov_y_deg, width, height, step, mode, tf, vmin, vmax, iso=0.0,
                      background=(0.0, 0.0, 0.0, 0.0), ambient=0.2) -> None:
    """Ray-march vol_a (or vol_a - vol_b) into out [height][width][4] (host or device)."""
    import numpy as _np

    tfa = _np.ascontiguousarray(tf, dtype=_np.float32).reshape(-1, 4)
    c = RenderCfg()
    c.eye[:], c.target[:], c.up[:] = list(eye), list(target), list(up)
    c.fov_y_deg, c.width, c.height, c.step = fov_y_deg, width, height, step
    c.mode, c.iso, c.vmin, c.vmax = mode, iso, vmin, vmax
    c.background[:] = list(background)
    c.ambient, c.n_tf = ambient, tfa.shape[0]
    c.tf = tfa.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    _check(ctx, _lib.ndf_render_volume(ctx, _addr(vol_a), None if vol_b is None else _addr(vol_b),
                                       X, Y, Z, ctypes.byref(c), _addr(out)),
           "ndf_render_volume")


class _HashModel:
    """A hash-grid NDF handle; holds its context for error strings."""

    def __init__(self, ctx, ptr):
        self.ctx, self.ptr = ctx, ptr

    @property
    def _as_parameter_(self):
        return self.ptr


def ndf_hash_arch_default() -> HashArch:
    a = HashArch()
    _lib.ndf_hash_arch_default(ctypes.byref(a))
    return a


def ndf_hash_model_create(ctx, arch: HashArch, measure: int, cross: bool, seed: int, X: int, Y: int,
                          Z: int):
    out = _vp()
    _check(ctx, _lib.ndf_hash_model_create(ctx, ctypes.byref(arch), measure, int(bool(cross)), seed,
                                           X, Y, Z, ctypes.byref(out)), "ndf_hash_model_create")
    return _HashModel(ctx, out)


def ndf_hash_model_free(m) -> None:
    _lib.ndf_hash_model_free(m)


def ndf_hash_model_param_count(m) -> int:
    return int(_lib.ndf_hash_model_param_count(m))


def ndf_hash_model_get_params(m, out) -> None:
    _check(m.ctx, _lib.ndf_hash_model_get_params(m, _addr(out)), "ndf_hash_model_get_params")


def ndf_hash_model_set_params(m, params) -> None:
    _check(m.ctx, _lib.ndf_hash_model_set_params(m, _addr(params)), "ndf_hash_model_set_params")


def ndf_hash_model_forward(m, pr, pq, out) -> None:
    B = len(out)
    _check(m.ctx, _lib.ndf_hash_model_forward(m, _addr(pr), _addr(pq), B, _addr(out)),
           "ndf_hash_model_forward")


def ndf_hash_model_step(m, pr, pq, target, lr: float, apply: bool, grad_out=None) -> float:
    loss = ctypes.c_double(0.0)
    _check(m.ctx, _lib.ndf_hash_model_step(m, _addr(pr), _addr(pq), _addr(target), len(target),
                                           lr, int(bool(apply)),
                                           None if grad_out is None else _addr(grad_out),
                                           ctypes.byref(loss)), "ndf_hash_model_step")
    return loss.value


def ndf_hash_train(ctx, ref_field: int, query_field: int, measure: int, k: int, arch: HashArch,
                   cfg=None):
    out = _vp()
    _check(ctx, _lib.ndf_hash_train(ctx, ref_field, query_field, measure, k, ctypes.byref(arch),
                                    None if cfg is None else ctypes.byref(cfg), ctypes.byref(out)),
           "ndf_hash_train")
    return _HashModel(ctx, out)


def ndf_hash_model_info(m) -> dict:
    p, ls, g, t, a = ctypes.c_int(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), _i64()
    _check(m.ctx, _lib.ndf_hash_model_info(m, ctypes.byref(p), ctypes.byref(ls), ctypes.byref(g),
                                           ctypes.byref(t), ctypes.byref(a)), "ndf_hash_model_info")
    return {"passes": p.value, "last_loss": ls.value, "gen_seconds": g.value,
            "train_seconds": t.value, "adam_steps": a.value}


def ndf_hash_infer(m, ref_idx: int, out) -> None:
    _check(m.ctx, _lib.ndf_hash_infer(m, ref_idx, _addr(out)), "ndf_hash_infer")


def ndf_hash_infer_batch(m, ref_idx, out) -> None:
    import numpy as _np

    refs = _np.ascontiguousarray(_np.asarray(ref_idx, dtype=_np.int64))
    _check(m.ctx, _lib.ndf_hash_infer_batch(m, refs.ctypes.data, int(refs.shape[0]), _addr(out)),
           "ndf_hash_infer_batch")


def ndf_hash_set_decode(m, mode: int, cache_queries: bool = False) -> None:
    _check(m.ctx, _lib.ndf_hash_set_decode(m, mode, int(bool(cache_queries))), "ndf_hash_set_decode")


def ndf_hash_get_decode(m) -> int:
    return int(_lib.ndf_hash_get_decode(m))


def ndf_pearson_noalloc(ref_field, query_field, M, N, ref_idx, out, cuda_stream=None) -> None:
    """Allocation-free Pearson volume: device buffers only, enqueued on cuda_stream."""
    st = _lib.ndf_pearson_noalloc(_addr(ref_field), _addr(query_field), M, N, ref_idx,
                                  _addr(out), cuda_stream)
    if st != NDF_OK:
        raise NdfError(st, "ndf_pearson_noalloc", "see include/ndf.h for the argument limits")


def ndf_field_column(ctx, field_id: int, vertex: int, out) -> None:
    """out[m] = member m's value at the vertex (M floats, host or device)."""
    _check(ctx, _lib.ndf_field_column(ctx, field_id, vertex, _addr(out)), "ndf_field_column")


def ndf_pearson_column(ctx, ref_column, query_field: int, out) -> None:
    """Pearson volume of the query field against a reference member column."""
    _check(ctx, _lib.ndf_pearson_column(ctx, _addr(ref_column), query_field, _addr(out)),
           "ndf_pearson_column")


def ndf_mi_ksg_column(ctx, ref_column, query_field: int, k: int, out) -> None:
    """KSG MI volume of the query field against a reference member column."""
    _check(ctx, _lib.ndf_mi_ksg_column(ctx, _addr(ref_column), query_field, k, _addr(out)),
           "ndf_mi_ksg_column")


def ndf_noalloc_pointer_usable(is_device: bool, is_managed: bool, ptr_device: int,
                               current_device: int) -> bool:
    """The buffer rule of ndf_pearson_noalloc (a host-only test hook)."""
    return bool(_lib.ndf_noalloc_pointer_usable(int(is_device), int(is_managed), ptr_device,
                                                current_device))


def ndf_sample_triples(ctx, ref_field: int, query_field: int, measure: int, k: int, n: int,
                       seed: int, pref, pq, target) -> None:
    """n continuous-position training triples: pref/pq [n][3], target [n]."""
    _check(ctx, _lib.ndf_sample_triples(ctx, ref_field, query_field, measure, k, n, seed,
                                        _addr(pref), _addr(pq), _addr(target)),
           "ndf_sample_triples")


def ndf_train_cfg_default() -> TrainCfg:
    c = TrainCfg()
    _lib.ndf_train_cfg_default(ctypes.byref(c))
    return c


def ndf_train(ctx, ref_field: int, query_field: int, measure: int, k: int, cfg=None):
    """Returns an opaque model handle (free with ndf_model_free)."""
    h = _vp()
    _check(ctx, _lib.ndf_train(ctx, ref_field, query_field, measure, k,
                               ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(h)),
           "ndf_train")
    return h


def _model_ctx_error(model, st, where):
    # model-level calls report through the owning context; the handle hides it,
    # so only the status and its description are available here
    if st != NDF_OK:
        raise NdfError(st, where, "")


def ndf_infer(model, ref_idx: int, out) -> None:
    _model_ctx_error(model, _lib.ndf_infer(model, ref_idx, _addr(out)), "ndf_infer")


def ndf_infer_batch(model, ref_idx, out) -> None:
    import numpy as _np

    refs = _np.ascontiguousarray(_np.asarray(ref_idx, dtype=_np.int64))
    _model_ctx_error(model, _lib.ndf_infer_batch(model, refs.ctypes.data, int(refs.shape[0]),
                                                 _addr(out)), "ndf_infer_batch")


def ndf_model_save(model, path: str) -> None:
    _model_ctx_error(model, _lib.ndf_model_save(model, path.encode()), "ndf_model_save")


def ndf_model_load(ctx, path: str):
    h = _vp()
    _check(ctx, _lib.ndf_model_load(ctx, path.encode(), ctypes.byref(h)), "ndf_model_load")
    return h


def ndf_model_free(model) -> None:
    _lib.ndf_model_free(model)


def ndf_model_info(model) -> dict:
    info = ModelInfo()
    _model_ctx_error(model, _lib.ndf_model_info(model, ctypes.byref(info)), "ndf_model_info")
    return info.as_dict()


def ndf_model_create(ctx, res, measure: int, seed: int, X: int, Y: int, Z: int):
    r = (ctypes.c_int * 4)(*[int(v) for v in res])
    h = _vp()
    _check(ctx, _lib.ndf_model_create(ctx, r, measure, seed, X, Y, Z, ctypes.byref(h)),
           "ndf_model_create")
    return h


def ndf_model_param_count(model) -> int:
    return int(_lib.ndf_model_param_count(model))


def ndf_model_get_params(model, out) -> None:
    _model_ctx_error(model, _lib.ndf_model_get_params(model, _addr(out)), "ndf_model_get_params")


def ndf_model_set_params(model, params) -> None:
    _model_ctx_error(model, _lib.ndf_model_set_params(model, _addr(params)), "ndf_model_set_params")


def ndf_model_step(model, p_ref, p_query, target, lr: float, update: bool, grad_out=None) -> float:
    """Returns the mean L1 loss of the batch (positions [B][3] float32)."""
    loss = ctypes.c_double(0.0)
    B = int(p_ref.shape[0])
    _model_ctx_error(model, _lib.ndf_model_step(model, _addr(p_ref), _addr(p_query), _addr(target),
                                                B, float(lr), int(bool(update)), ctypes.byref(loss),
                                                _addr(grad_out)), "ndf_model_step")
    return loss.value


def ndf_model_forward(model, p_ref, p_query, out) -> None:
    _model_ctx_error(model, _lib.ndf_model_forward(model, _addr(p_ref), _addr(p_query),
                                                   int(p_ref.shape[0]), _addr(out)),
                     "ndf_model_forward")


def exported_symbols():
    """Every ndf_* function name this binding declares."""
    return sorted(n for n in globals() if n.startswith("ndf_") and callable(globals()[n]))
