"""GPU parity of the exact estimators against the CPU oracle (same seeded bytes).

Bars (element by element):
  Pearson            |r_gpu - r_oracle(FP64)| <= 1e-5
  KSG eps, nx, ny    bit-exact (FP32 max-norm distances are computed identically)
  KSG MI             |mi_gpu - mi_oracle| <= 1e-6 |mi_oracle| + 1e-9
                     (the FP32 volume adds at most 2^-24 relative rounding)
"""
import numpy as np
import pytest
import torch

import oracle
from golden_io import ksg2_hand_cases
import synth

pytestmark = pytest.mark.gpu

PEARSON_TOL = 1e-5


def mi_close(gpu, ref):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    bad = np.abs(gpu - ref) > 1e-6 * np.abs(ref) + 1e-9
    return not bad.any(), np.flatnonzero(bad)[:10]


def load(ndf, ctx, field):
    f = np.ascontiguousarray(field, dtype=np.float32)
    M, Z, Y, X = f.shape
    return ndf.ndf_load_ensemble(ctx, f, M, Z, Y, X)


def rand_field(shape, seed, kind="normal"):
    rng = np.random.default_rng(seed)
    f = rng.normal(size=shape)
    if kind == "ties":
        f = np.round(f * 2.0) / 2.0
    return f.astype(np.float32)


# ---------------------------------------------------------------- statistics (load)
def test_load_statistics(ndf_mod, ctx, tiny_field):
    fid = load(ndf_mod, ctx, tiny_field)
    M = tiny_field.shape[0]
    N = tiny_field[0].size
    mean = np.empty(N)
    inv = np.empty(N)
    ndf_mod.ndf_field_stats(ctx, fid, mean, inv)
    f64 = tiny_field.reshape(M, N).astype(np.float64)
    mu = f64.mean(axis=0)
    S = ((f64 - mu) ** 2).sum(axis=0)
    np.testing.assert_allclose(mean, mu, rtol=0, atol=1e-5 * np.abs(f64).max())
    np.testing.assert_allclose(inv, 1.0 / np.sqrt(S), rtol=1e-5)
    assert ndf_mod.ndf_field_shape(ctx, fid) == tiny_field.shape
    ndf_mod.ndf_free_ensemble(ctx, fid)


def test_chunked_upload_statistics_and_sorted_columns(ndf_mod, ctx):
    """M = 4096 uploads in ranges that double from 16384 vertices: 16384, 32768
    and a ragged tail of 77.  Statistics and KSG counts (which search the sorted
    columns) must hold at the range boundaries."""
    M, N = 4096, 16384 + 32768 + 77
    rng = np.random.default_rng(99)
    f = rng.normal(size=(M, 1, 1, N)).astype(np.float32)
    f[:, 0, 0, 16383:16386] += 2.0 * f[:, 0, 0, 5:8]  # dependence across a boundary
    f[:, 0, 0, 49150:49153] += 2.0 * f[:, 0, 0, 9:12]
    fid = load(ndf_mod, ctx, f)
    mean = np.empty(N)
    inv = np.empty(N)
    ndf_mod.ndf_field_stats(ctx, fid, mean, inv)
    cols = [0, 16383, 16384, 49151, 49152, N - 1]
    f64 = f.reshape(M, N)[:, cols].astype(np.float64)
    mu = f64.mean(axis=0)
    np.testing.assert_allclose(mean[cols], mu, rtol=0, atol=1e-5 * np.abs(f64).max())
    np.testing.assert_allclose(inv[cols], 1.0 / np.sqrt(((f64 - mu) ** 2).sum(axis=0)), rtol=1e-5)
    check_pairs_bit_exact(ndf_mod, ctx, fid, fid, f, f, 6, cols, 4)
    ndf_mod.ndf_free_ensemble(ctx, fid)


@pytest.mark.parametrize("M,N", [(1000, 640), (1000, 643), (20, 70), (64, 33), (100, 37),
                                 (300, 52), (513, 96), (3000, 41)])
def test_sorted_columns_bit_equal(ndf_mod, ctx, M, N):
    """Every loaded column ascending, bit for bit as numpy sorts it: tiles of 16 vertices
    read as 16-byte quads (N % 4 == 0) or one float at a time (ragged N), each lane count
    of the register network (R = 1, 2, 4, 16, 32), and the shared-memory network above
    1024 members; a column with ties and a constant column included."""
    rng = np.random.default_rng(M * 7 + N)
    f = rng.normal(size=(M, N)).astype(np.float32)
    f[:, 1] = np.round(f[:, 1] * 2.0) / 2.0
    f[:, 2] = 0.75
    f = f + np.float32(0.0)  # no negative zeros: equal keys may leave in either order
    fid = load(ndf_mod, ctx, f.reshape(M, 1, 1, N))
    out = np.empty((M, N), dtype=np.float32)
    ndf_mod.ndf_field_sorted_columns(ctx, fid, 0, N, out)
    assert np.array_equal(out.view(np.uint32), np.sort(f, axis=0).view(np.uint32))
    v0, v1 = 3, N - 2  # a sub-range, into device memory
    dev = torch.empty((M, v1 - v0), dtype=torch.float32, device="cuda")
    ndf_mod.ndf_field_sorted_columns(ctx, fid, v0, v1, dev)
    assert np.array_equal(dev.cpu().numpy().view(np.uint32), out[:, v0:v1].view(np.uint32))
    for a, b in ((-1, 2), (2, 1), (0, N + 1)):
        with pytest.raises(ndf_mod.NdfError) as ei:
            ndf_mod.ndf_field_sorted_columns(ctx, fid, a, b, out)
        assert ei.value.status == ndf_mod.NDF_ERR_ARG
    ndf_mod.ndf_free_ensemble(ctx, fid)


def test_sorted_columns_absent_above_4096_members(ndf_mod, ctx):
    f = rand_field((4097, 1, 1, 8), 5)
    fid = load(ndf_mod, ctx, f)
    out = np.empty((4097, 8), dtype=np.float32)
    with pytest.raises(ndf_mod.NdfError) as ei:
        ndf_mod.ndf_field_sorted_columns(ctx, fid, 0, 8, out)
    assert ei.value.status == ndf_mod.NDF_ERR_STATE
    ndf_mod.ndf_free_ensemble(ctx, fid)


@pytest.mark.parametrize("M,offset", [(1000, 0), (1000, 1), (1100, 0)])
def test_device_source_load_matches_host_load(ndf_mod, ctx, M, offset):
    """A device-resident field is read in place: up to 1024 members the sort kernel
    writes the copy as it reads (16-byte quads from an aligned source, single floats
    from one shifted by a float), above that a contiguous copy comes first.  The
    statistics, sorted columns and both volumes equal those of the same field loaded
    from host memory, bit for bit, for ndf_load_ensemble and ndf_load_and_compute."""
    Z, Y, X = 1, 3, 100  # N = 300: 18 whole 16-vertex tiles and a ragged one
    N, ref = Z * Y * X, 17
    f = rand_field((M, Z, Y, X), 21)
    fh = load(ndf_mod, ctx, f)
    buf = torch.empty(M * N + offset, dtype=torch.float32, device="cuda")
    buf[offset:] = torch.from_numpy(f.reshape(-1)).cuda()
    src = buf[offset:]

    def state(fid):
        mean, inv = np.empty(N), np.empty(N)
        ndf_mod.ndf_field_stats(ctx, fid, mean, inv)
        cols = np.empty((M, N), dtype=np.float32)
        ndf_mod.ndf_field_sorted_columns(ctx, fid, 0, N, cols)
        r, mi = np.empty(N, dtype=np.float32), np.empty(N, dtype=np.float32)
        ndf_mod.ndf_pearson(ctx, fid, fid, ref, r)
        ndf_mod.ndf_mi_ksg(ctx, fid, fid, ref, 4, mi)
        return [mean.view(np.uint64), inv.view(np.uint64), cols.view(np.uint32),
                r.view(np.uint32), mi.view(np.uint32)]

    want = state(fh)
    fd = ndf_mod.ndf_load_ensemble(ctx, src, M, Z, Y, X)
    for a, b in zip(state(fd), want):
        assert np.array_equal(a, b)
    r, mi = np.empty(N, dtype=np.float32), np.empty(N, dtype=np.float32)
    fc = ndf_mod.ndf_load_and_compute(ctx, src, M, Z, Y, X, ref, 4, r, mi)
    assert np.array_equal(r.view(np.uint32), want[3]) and np.array_equal(mi.view(np.uint32), want[4])
    for a, b in zip(state(fc), want):
        assert np.array_equal(a, b)
    r2 = np.empty(N, dtype=np.float32)  # Pearson only, from host memory
    fp = ndf_mod.ndf_load_and_compute(ctx, f, M, Z, Y, X, ref, 4, r2, None)
    assert np.array_equal(r2.view(np.uint32), want[3])
    for a, b in zip(state(fp), want):
        assert np.array_equal(a, b)
    for fid in (fh, fd, fc, fp):
        ndf_mod.ndf_free_ensemble(ctx, fid)


def test_reload_reuses_buffers_without_stale_data(ndf_mod, ctx, tiny_field, tiny_ref):
    """A freed field's buffers are reused by the next load of the same size; the
    new field's statistics, sorted columns and volumes must be its own."""
    N = tiny_field[0].size
    other = (tiny_field[::-1] * 1.5 + 0.25).copy()
    fa = load(ndf_mod, ctx, tiny_field)
    ndf_mod.ndf_free_ensemble(ctx, fa)
    fb = load(ndf_mod, ctx, other)
    out = np.empty(N, dtype=np.float32)
    ndf_mod.ndf_mi_ksg(ctx, fb, fb, tiny_ref, 4, out)
    ok, where = mi_close(out, oracle.ksg_volume(other, other, tiny_ref, 4))
    assert ok, where
    ndf_mod.ndf_pearson(ctx, fb, fb, tiny_ref, out)
    assert np.abs(out - oracle.pearson_volume(other, other, tiny_ref)).max() <= PEARSON_TOL
    ndf_mod.ndf_free_ensemble(ctx, fb)
    ndf_mod.ndf_trim_cache(ctx)


def test_load_from_device_memory(ndf_mod, ctx, tiny_field, tiny_ref):
    t = torch.from_numpy(tiny_field).cuda()
    fid = ndf_mod.ndf_load_ensemble(ctx, t, *tiny_field.shape)
    out = np.empty(tiny_field[0].size, dtype=np.float32)
    ndf_mod.ndf_pearson(ctx, fid, fid, tiny_ref, out)
    ref = oracle.pearson_volume(tiny_field, tiny_field, tiny_ref)
    assert np.abs(out - ref).max() <= PEARSON_TOL
    ndf_mod.ndf_free_ensemble(ctx, fid)


# ---------------------------------------------------------------- Pearson (Eq. 1)
def test_pearson_tiny_host_and_device_outputs(ndf_mod, ctx, tiny_field, tiny_ref):
    fid = load(ndf_mod, ctx, tiny_field)
    N = tiny_field[0].size
    ref = oracle.pearson_volume(tiny_field, tiny_field, tiny_ref)
    host = np.empty(N, dtype=np.float32)
    ndf_mod.ndf_pearson(ctx, fid, fid, tiny_ref, host)
    dev = torch.empty(N, dtype=torch.float32, device="cuda")
    ndf_mod.ndf_pearson(ctx, fid, fid, tiny_ref, dev)
    ndf_mod.ndf_synchronize(ctx)
    assert np.abs(host - ref).max() <= PEARSON_TOL
    np.testing.assert_array_equal(dev.cpu().numpy(), host)
    assert host[tiny_ref] == pytest.approx(1.0, abs=1e-6)
    ndf_mod.ndf_free_ensemble(ctx, fid)


@pytest.mark.parametrize("shape", [(1000, 4, 10, 25),   # N % 4 == 0: vector path, many CTAs
                                   (37, 3, 5, 7),        # N odd: scalar path, ragged tail
                                   (2, 1, 1, 3),         # smallest M
                                   (2500, 2, 4, 9),      # more members than one staged chunk
                                   (64, 1, 1, 1)])       # a single vertex
def test_pearson_shapes(ndf_mod, ctx, shape):
    f = rand_field(shape, seed=sum(shape))
    f[:, 0, 0, 0] += 3.0 * f[:, -1, -1, -1]  # some real dependence
    fid = load(ndf_mod, ctx, f)
    N = f[0].size
    for r in sorted({0, N // 2, N - 1}):
        out = np.empty(N, dtype=np.float32)
        ndf_mod.ndf_pearson(ctx, fid, fid, r, out)
        ref = oracle.pearson_volume(f, f, r)
        assert np.abs(out - ref).max() <= PEARSON_TOL, (shape, r)
    ndf_mod.ndf_free_ensemble(ctx, fid)


def test_pearson_cross_field_and_degenerate(ndf_mod, ctx):
    shape = (200, 2, 6, 10)
    a = rand_field(shape, 11)
    b = (0.6 * a + 0.8 * rand_field(shape, 12)).astype(np.float32)
    b[:, 1, 2, 3] = 7.0  # constant query column: r = 0
    fa, fb = load(ndf_mod, ctx, a), load(ndf_mod, ctx, b)
    out = np.empty(a[0].size, dtype=np.float32)
    ndf_mod.ndf_pearson(ctx, fa, fb, 17, out)
    ref = oracle.pearson_volume(a, b, 17)
    assert np.abs(out - ref).max() <= PEARSON_TOL
    assert out[(1 * 6 + 2) * 10 + 3] == 0.0
    ndf_mod.ndf_free_ensemble(ctx, fa)
    ndf_mod.ndf_free_ensemble(ctx, fb)


# ---------------------------------------------------------------- KSG algorithm 1
@pytest.fixture(params=["brute", "pruned", "block", "lanes"])
def algo(request, ndf_mod, ctx):
    """Every search must give the same bit-exact eps / counts."""
    code = {"brute": ndf_mod.NDF_KSG_BRUTE, "pruned": ndf_mod.NDF_KSG_PRUNED,
            "block": ndf_mod.NDF_KSG_BLOCK, "lanes": ndf_mod.NDF_KSG_LANES}[request.param]
    ndf_mod.ndf_set_ksg_algorithm(ctx, code)
    yield request.param
    ndf_mod.ndf_set_ksg_algorithm(ctx, ndf_mod.NDF_KSG_LANES)  # the default


def ksg_debug(ndf, ctx, fa, fb, r, v, k, M):
    eps = np.empty(M, dtype=np.float32)
    nx = np.empty(M, dtype=np.int32)
    ny = np.empty(M, dtype=np.int32)
    mi = np.empty(1, dtype=np.float64)
    ndf.ndf_ksg_debug_pair(ctx, fa, fb, r, v, k, eps, nx, ny, mi)
    return mi[0], eps, nx, ny


def check_pairs_bit_exact(ndf, ctx, fa, fb, a, b, r, verts, k):
    M = a.shape[0]
    a2 = a.reshape(M, -1)
    b2 = b.reshape(M, -1)
    for v in verts:
        g = ksg_debug(ndf, ctx, fa, fb, r, int(v), k, M)
        o = oracle.ksg_pair(a2[:, r], b2[:, v], k)
        np.testing.assert_array_equal(g[1], o[1], err_msg=f"eps v={v}")
        np.testing.assert_array_equal(g[2], o[2], err_msg=f"nx v={v}")
        np.testing.assert_array_equal(g[3], o[3], err_msg=f"ny v={v}")
        assert abs(g[0] - o[0]) <= 1e-6 * abs(o[0]) + 1e-9, (v, g[0], o[0])


def test_ksg_tiny_every_pair_bit_exact(ndf_mod, ctx, algo, tiny_field, tiny_ref):
    fid = load(ndf_mod, ctx, tiny_field)
    N = tiny_field[0].size
    check_pairs_bit_exact(ndf_mod, ctx, fid, fid, tiny_field, tiny_field, tiny_ref, range(N), 4)
    ndf_mod.ndf_free_ensemble(ctx, fid)


def test_ksg_tiny_volume(ndf_mod, ctx, algo, tiny_field, tiny_ref):
    fid = load(ndf_mod, ctx, tiny_field)
    N = tiny_field[0].size
    out = np.empty(N, dtype=np.float32)
    ndf_mod.ndf_mi_ksg(ctx, fid, fid, tiny_ref, 4, out)
    ref = oracle.ksg_volume(tiny_field, tiny_field, tiny_ref, 4)
    ok, where = mi_close(out, ref)
    assert ok, where
    dev = torch.empty(N, dtype=torch.float32, device="cuda")
    ndf_mod.ndf_mi_ksg(ctx, fid, fid, tiny_ref, 4, dev)
    ndf_mod.ndf_synchronize(ctx)
    np.testing.assert_array_equal(dev.cpu().numpy(), out)  # deterministic
    ndf_mod.ndf_free_ensemble(ctx, fid)


@pytest.mark.parametrize("shape,k,kind", [
    ((1000, 2, 8, 25), 8, "normal"),   # paper-scale M, several tiles + ragged tail
    ((1000, 1, 3, 7), 8, "ties"),      # heavy ties: eps = 0 and equal distances
    ((2500, 1, 2, 9), 8, "normal"),    # M > 2048: threads own two point blocks
    ((4096, 1, 1, 3), 16, "normal"),   # largest M and k
    ((3000, 1, 1, 4), 8, "normal"),    # M > 2048, not a power of two
    ((2, 1, 2, 2), 1, "normal"),       # smallest M
    ((17, 1, 3, 3), 16, "normal"),     # k = M - 1 = 16 (largest supported k)
    ((100, 2, 3, 5), 3, "ties"),
    ((333, 1, 1, 13), 5, "normal"),    # M not a multiple of 4
])
def test_ksg_shapes(ndf_mod, ctx, algo, shape, k, kind):
    f = rand_field(shape, seed=shape[0] + k, kind=kind)
    f[:, 0, 0, 0] = f[:, -1, -1, -1] ** 2 + 0.1 * f[:, 0, 0, 0]
    fid = load(ndf_mod, ctx, f)
    N = f[0].size
    r = N - 1
    out = np.empty(N, dtype=np.float32)
    ndf_mod.ndf_mi_ksg(ctx, fid, fid, r, k, out)
    ref = oracle.ksg_volume(f, f, r, k)
    ok, where = mi_close(out, ref)
    assert ok, (where, out[where], ref[where])
    check_pairs_bit_exact(ndf_mod, ctx, fid, fid, f, f, r, sorted({0, 1, N // 2, N - 1}), k)
    ndf_mod.ndf_free_ensemble(ctx, fid)


def test_ksg_cross_field(ndf_mod, ctx, algo):
    shape = (300, 2, 4, 6)
    a = rand_field(shape, 21)
    b = (np.tanh(a) + 0.5 * rand_field(shape, 22)).astype(np.float32)
    fa, fb = load(ndf_mod, ctx, a), load(ndf_mod, ctx, b)
    N = a[0].size
    out = np.empty(N, dtype=np.float32)
    ndf_mod.ndf_mi_ksg(ctx, fa, fb, 5, 8, out)
    ok, where = mi_close(out, oracle.ksg_volume(a, b, 5, 8))
    assert ok, where
    check_pairs_bit_exact(ndf_mod, ctx, fa, fb, a, b, 5, [0, 5, N - 1], 8)
    ndf_mod.ndf_free_ensemble(ctx, fa)
    ndf_mod.ndf_free_ensemble(ctx, fb)


# ---------------------------------------------------------------- KSG algorithm 2
def ksg2_debug(ndf, ctx, fa, fb, r, v, k, M):
    ex = np.empty(M, dtype=np.float32)
    ey = np.empty(M, dtype=np.float32)
    nx = np.empty(M, dtype=np.int32)
    ny = np.empty(M, dtype=np.int32)
    mi = np.empty(1, dtype=np.float64)
    ndf.ndf_ksg2_debug_pair(ctx, fa, fb, r, v, k, ex, ey, nx, ny, mi)
    return float(mi[0]), ex, ey, nx, ny


def check_pairs2_bit_exact(ndf, ctx, fa, fb, a, b, r, verts, k):
    M = a.shape[0]
    a2 = a.reshape(M, -1)
    b2 = b.reshape(M, -1)
    for v in verts:
        g = ksg2_debug(ndf, ctx, fa, fb, r, int(v), k, M)
        o = oracle.ksg2_pair(a2[:, r], b2[:, v], k)
        for idx, name in ((1, "ex"), (2, "ey"), (3, "nx"), (4, "ny")):
            np.testing.assert_array_equal(g[idx], o[idx], err_msg=f"{name} v={v}")
        assert abs(g[0] - o[0]) <= 1e-6 * abs(o[0]) + 1e-9, (v, g[0], o[0])


@pytest.mark.parametrize("case", ksg2_hand_cases(), ids=lambda c: c["name"])
def test_ksg2_hand_cases(ndf_mod, ctx, algo, case):
    """The hand-enumerated algorithm-2 cases as a two-vertex field (x at vertex 0,
    y at vertex 1): extents, counts and the exact rational MI."""
    f = np.stack([case["x"], case["y"]], axis=1).astype(np.float32).reshape(-1, 1, 1, 2)
    fid = load(ndf_mod, ctx, f)
    M = f.shape[0]
    mi, ex, ey, nx, ny = ksg2_debug(ndf_mod, ctx, fid, fid, 0, 1, case["k"], M)
    np.testing.assert_array_equal(ex, np.array(case["ex"], dtype=np.float32))
    np.testing.assert_array_equal(ey, np.array(case["ey"], dtype=np.float32))
    np.testing.assert_array_equal(nx, case["nx"])
    np.testing.assert_array_equal(ny, case["ny"])
    assert mi == pytest.approx(float(case["mi"]), abs=1e-12)
    out = np.empty(2, dtype=np.float32)
    ndf_mod.ndf_mi_ksg2(ctx, fid, fid, 0, case["k"], out)
    assert out[1] == np.float32(float(case["mi"]))
    ndf_mod.ndf_free_ensemble(ctx, fid)


@pytest.mark.parametrize("shape,k,kind", [
    ((1000, 2, 4, 9), 8, "normal"),
    ((300, 1, 3, 7), 4, "ties"),
    ((17, 1, 3, 3), 16, "normal"),     # k = M - 1
    ((2, 1, 2, 2), 1, "normal"),
    ((3000, 1, 1, 3), 8, "normal"),
])
def test_ksg2_volume_and_pairs(ndf_mod, ctx, algo, shape, k, kind):
    f = rand_field(shape, seed=7 * shape[0] + k, kind=kind)
    fid = load(ndf_mod, ctx, f)
    N = f[0].size
    r = N // 2
    out = np.empty(N, dtype=np.float32)
    ndf_mod.ndf_mi_ksg2(ctx, fid, fid, r, k, out)
    ok, where = mi_close(out, oracle.ksg2_volume(f, f, r, k))
    assert ok, (where, out[where])
    check_pairs2_bit_exact(ndf_mod, ctx, fid, fid, f, f, r, sorted({0, r, N - 1}), k)
    ndf_mod.ndf_free_ensemble(ctx, fid)


# ---------------------------------------------------------------- batched KSG
def test_ksg_batch_matches_oracle_and_single(ndf_mod, ctx, algo):
    ndf = ndf_mod
    shape = (1000, 2, 6, 11)
    f = rand_field(shape, seed=77)
    f[:, 1] = np.tanh(f[:, 0]) + 0.3 * f[:, 1]
    fid = load(ndf, ctx, f)
    N = f[0].size
    refs = [0, 5, 131, N - 1, 64]
    out = np.empty((len(refs), N), dtype=np.float32)
    ndf.ndf_mi_ksg_batch(ctx, fid, fid, refs, 8, out)
    for i, r in enumerate(refs):
        ok, where = mi_close(out[i], oracle.ksg_volume(f, f, r, 8))
        assert ok, (r, where)
        single = np.empty(N, dtype=np.float32)
        ndf.ndf_mi_ksg(ctx, fid, fid, r, 8, single)
        np.testing.assert_array_equal(out[i], single)
    g, t = ndf.ndf_ksg_autotune(ctx, fid, fid, 8)
    assert g in (1, 2, 4, 8) and t in (4, 8)
    dev = torch.empty((len(refs), N), dtype=torch.float32, device="cuda")
    ndf.ndf_mi_ksg_batch(ctx, fid, fid, refs, 8, dev)
    ndf.ndf_synchronize(ctx)
    np.testing.assert_array_equal(dev.cpu().numpy(), out)
    ndf.ndf_free_ensemble(ctx, fid)


def test_ksg_eval_counter(ndf_mod, ctx, tiny_field, tiny_ref):
    ndf = ndf_mod
    fid = load(ndf, ctx, tiny_field)
    M = tiny_field.shape[0]
    N = tiny_field[0].size
    out = np.empty(N, dtype=np.float32)
    counts = {}
    for name in ("NDF_KSG_PRUNED", "NDF_KSG_BLOCK", "NDF_KSG_LANES", "NDF_KSG_BRUTE"):
        ndf.ndf_set_ksg_algorithm(ctx, getattr(ndf, name), True)
        ndf.ndf_mi_ksg(ctx, fid, fid, tiny_ref, 4, out)
        counts[name] = ndf.ndf_ksg_take_eval_count(ctx)
        assert ndf.ndf_ksg_take_eval_count(ctx) == 0
    ndf.ndf_set_ksg_algorithm(ctx, ndf.NDF_KSG_LANES, False)
    # brute force evaluates every candidate; the exact searches strict subsets, the
    # block search fewer than the x-strip scan
    assert counts["NDF_KSG_BRUTE"] == N * M * (M - 1)
    assert 0 < counts["NDF_KSG_BLOCK"] < counts["NDF_KSG_PRUNED"] < N * M * (M - 1)
    # the lane schedule visits the same kind of windows (another side order)
    assert 0 < counts["NDF_KSG_LANES"] < counts["NDF_KSG_PRUNED"]
    ndf.ndf_free_ensemble(ctx, fid)


# ---------------------------------------------------------------- argument errors
def test_argument_errors(ndf_mod, ctx, tiny_field, tiny_ref):
    ndf = ndf_mod
    fid = load(ndf, ctx, tiny_field)
    N = tiny_field[0].size
    out = np.empty(N, dtype=np.float32)
    cases = [
        lambda: ndf.ndf_mi_ksg(ctx, fid, fid, tiny_ref, 0, out),
        lambda: ndf.ndf_mi_ksg(ctx, fid, fid, tiny_ref, 100, out),
        lambda: ndf.ndf_mi_ksg(ctx, fid, fid, tiny_ref, 17, out),
        lambda: ndf.ndf_pearson(ctx, fid, fid, N, out),
        lambda: ndf.ndf_pearson(ctx, fid, fid, -1, out),
        lambda: ndf.ndf_pearson(ctx, fid, 1 << 20, 0, out),  # an id never issued
        lambda: ndf.ndf_pearson(ctx, fid, fid, 0, None),
    ]
    for c in cases:
        with pytest.raises(ndf.NdfError) as ei:
            c()
        assert ei.value.status == ndf.NDF_ERR_ARG
    other = load(ndf, ctx, tiny_field[:, :2])
    with pytest.raises(ndf.NdfError) as ei:
        ndf.ndf_pearson(ctx, fid, other, 0, out)
    assert ei.value.status == ndf.NDF_ERR_ARG
    for value, where in ((np.nan, (3, 0, 0, 0)), (np.inf, (0, 0, 1, 5)), (-np.inf, (7, 0, 0, 15))):
        bad = tiny_field.copy()
        bad[where] = value
        with pytest.raises(ndf.NdfError) as ei:
            load(ndf, ctx, bad)
        assert ei.value.status == ndf.NDF_ERR_ARG
        with pytest.raises(ndf.NdfError) as ei:  # read in place from device memory
            ndf.ndf_load_ensemble(ctx, torch.from_numpy(bad).cuda(), *bad.shape)
        assert ei.value.status == ndf.NDF_ERR_ARG
    with pytest.raises(ndf.NdfError) as ei:
        ndf.ndf_load_ensemble(ctx, tiny_field, 1, 4, 16, 16)
    assert ei.value.status == ndf.NDF_ERR_ARG
    ndf.ndf_free_ensemble(ctx, other)
    with pytest.raises(ndf.NdfError) as ei:
        ndf.ndf_pearson(ctx, other, other, 0, out)
    assert ei.value.status == ndf.NDF_ERR_STATE
    ndf.ndf_free_ensemble(ctx, fid)
    assert ndf.ndf_launch_count(ctx) > 0


# ---------------------------------------------------------------- pipelined load + volumes
def test_load_and_compute_matches_separate_calls(ndf_mod, ctx):
    """The pipelined entry point runs the same kernels range by range (three ranges at
    M = 2048, the reference's middle range first): bit-equal volumes, host and device
    outputs, a skipped measure, and the field stays loaded."""
    ndf = ndf_mod
    shape = (2048, 17, 63, 64)  # 68,544 vertices: ranges of 32,768 + 32,768 + 3,008
    f = rand_field(shape, 31)
    f[:, :, :, ::2] = np.tanh(f[:, :, :, ::2] + 0.3 * f[:, :, :, 1::2])
    f = np.ascontiguousarray(f)
    M, Z, Y, X = shape
    N = Z * Y * X
    ref = 40000
    fid = load(ndf, ctx, f)
    p1 = np.empty(N, np.float32)
    m1 = np.empty(N, np.float32)
    ndf.ndf_pearson(ctx, fid, fid, ref, p1)
    ndf.ndf_mi_ksg(ctx, fid, fid, ref, 8, m1)
    ndf.ndf_free_ensemble(ctx, fid)
    p2 = np.empty(N, np.float32)
    m2 = torch.empty(N, dtype=torch.float32, device="cuda")
    fid2 = ndf.ndf_load_and_compute(ctx, f, M, Z, Y, X, ref, 8, p2, m2)
    ndf.ndf_synchronize(ctx)
    np.testing.assert_array_equal(p2, p1)
    np.testing.assert_array_equal(m2.cpu().numpy(), m1)
    p3 = np.empty(N, np.float32)
    ndf.ndf_pearson(ctx, fid2, fid2, ref, p3)  # the field stays loaded
    np.testing.assert_array_equal(p3, p1)
    # the x-strip search on the same loaded field: the same eps and counts, its FP64
    # digamma sum accumulated in another member order (MI within 1e-6 relative)
    ndf.ndf_set_ksg_algorithm(ctx, ndf.NDF_KSG_PRUNED)
    m3 = np.empty(N, np.float32)
    ndf.ndf_mi_ksg(ctx, fid2, fid2, ref, 8, m3)
    ndf.ndf_set_ksg_algorithm(ctx, ndf.NDF_KSG_LANES)
    np.testing.assert_allclose(m3, m1, rtol=1e-6, atol=1e-9)
    ndf.ndf_free_ensemble(ctx, fid2)
    p4 = np.empty(N, np.float32)
    fid3 = ndf.ndf_load_and_compute(ctx, f, M, Z, Y, X, ref, 8, p4, None)  # Pearson only
    np.testing.assert_array_equal(p4, p1)
    ndf.ndf_free_ensemble(ctx, fid3)


def test_load_and_compute_growing_ranges(ndf_mod, ctx):
    """Ranges that double after the reference's: at M = 1024 (base range 65,536
    vertices) and 458,752 vertices with the reference in the fourth base range, the
    call uploads [196,608, 262,144), then 131,072 and 65,536 vertices above it and
    196,608 below; the volumes must be bit-equal to a plain load and the separate
    calls."""
    ndf = ndf_mod
    shape = (1024, 7, 256, 256)
    f = rand_field(shape, 33)
    M, Z, Y, X = shape
    N = Z * Y * X
    ref = 3 * 65536 + 1234
    fid = load(ndf, ctx, f)
    p1 = torch.empty(N, dtype=torch.float32, device="cuda")
    m1 = torch.empty(N, dtype=torch.float32, device="cuda")
    ndf.ndf_pearson(ctx, fid, fid, ref, p1)
    ndf.ndf_mi_ksg(ctx, fid, fid, ref, 8, m1)
    ndf.ndf_free_ensemble(ctx, fid)
    p2 = torch.empty(N, dtype=torch.float32, device="cuda")
    m2 = torch.empty(N, dtype=torch.float32, device="cuda")
    fid2 = ndf.ndf_load_and_compute(ctx, f, M, Z, Y, X, ref, 8, p2, m2)
    ndf.ndf_synchronize(ctx)
    assert torch.equal(p1, p2)
    assert torch.equal(m1, m2)
    ndf.ndf_free_ensemble(ctx, fid2)


def test_load_and_compute_rejects_bad_input(ndf_mod, ctx, tiny_field, tiny_ref):
    ndf = ndf_mod
    f = tiny_field.copy()
    M, Z, Y, X = f.shape
    out = np.empty(Z * Y * X, np.float32)
    with pytest.raises(ndf.NdfError):
        ndf.ndf_load_and_compute(ctx, f, M, Z, Y, X, Z * Y * X, 4, out, out)  # ref out of range
    with pytest.raises(ndf.NdfError):
        ndf.ndf_load_and_compute(ctx, f, M, Z, Y, X, tiny_ref, M, out, out)  # k >= M
    f[3, 0, 0, 5] = np.nan
    with pytest.raises(ndf.NdfError):
        ndf.ndf_load_and_compute(ctx, f, M, Z, Y, X, tiny_ref, 4, out, out)
    # the context stays usable
    fid = ndf.ndf_load_and_compute(ctx, tiny_field, M, Z, Y, X, tiny_ref, 4, out, None)
    ndf.ndf_free_ensemble(ctx, fid)
