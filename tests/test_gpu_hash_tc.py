"""The tensor-core decoder of the paper's NDF architecture (hash grid + Fourier
features + Snake-family encoders, merge, decoder; Sec. 4.1-4.2) against the
oracle.

The decoder multiplies BF16 operands with FP32 accumulation, so it is held to
two references on the same FP32 parameters and vertex positions:
  oracle.hash_forward_bf16 (the same BF16 operands, FP64 sums).  Where no
    operand's BF16 rounding flips between the FP32-accumulated and the FP64
    value, the two agree to FP32 accumulation error (~1e-7; most vertices of most
    volumes).  A flip moves one operand by one BF16 ulp (2^-8 relative) and the
    rest of the network amplifies it: up to 1.5e-2 at a vertex over 11 layers
    (NumPy emulation of these random networks), and a flip inside the reference's
    own latent shifts every vertex of its volume (measured: median 4e-3 on one of
    the networks below).  Bounds: median and mean 1e-2, max 0.1.
  oracle.hash_forward (FP64): every operand carries 2^-9 relative rounding;
    emulated: mean 8e-3, max 5.4e-2 for 11 layers.  Bounds: mean 3e-2, max 0.2.
A wrong layout, swizzle, bias or merge moves every vertex by about the output's
spread (std 0.2-0.8 here), 20-80 times the median bound.
Exact properties: the cached-query decode equals the uncached one bit for bit
(the same FP32 latent enters the merge), and a self field is symmetric."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

PAPER_SMALL_TABLE = dict(log2_table=14)  # the paper's architecture with 2^14-entry tables


def arch(ndf_mod, **kw):
    a = ndf_mod.ndf_hash_arch_default()
    for k, v in dict(PAPER_SMALL_TABLE, **kw).items():
        setattr(a, k, v)
    return a


def oshape(a, cross, measure):
    return oracle.hash_shape(levels=a.levels, base_res=a.base_res, log2_table=a.log2_table,
                             feat=a.feat, n_freq=a.n_freq, width=a.width, enc_layers=a.enc_layers,
                             dec_layers=a.dec_layers, n_enc=2 if cross else 1, measure=measure,
                             act=a.act, merge=a.merge)


def layout(a, n_enc):
    """Parameter blocks (offset, n_out, n_in) of the flat layout, tables first."""
    din = 3 + 6 * a.n_freq + a.levels * a.feat
    ent = [min((a.base_res << l) ** 3, 2 ** a.log2_table) for l in range(a.levels)]
    tables = sum(ent) * a.feat
    o, enc = 0, []
    for e in range(n_enc):
        t0 = o
        o += tables
        layers = []
        for k in range(a.enc_layers):
            cin = din if k == 0 else a.width
            layers.append((o, a.width, cin))
            o += cin * a.width + a.width
        enc.append((t0, tables, layers))
    dec = []
    for k in range(a.dec_layers):
        out = 1 if k == a.dec_layers - 1 else a.width
        cin = (a.width if a.enc_layers else din) if k == 0 else a.width
        dec.append((o, out, cin))
        o += cin * out + out
    return enc, dec, o


def make_params(a, n_enc, seed, gain=0.9):
    """Tables U(-1, 1); weights gain x He-uniform; biases N(0, 0.1)."""
    rng = np.random.default_rng(seed)
    enc, dec, total = layout(a, n_enc)
    p = np.zeros(total, np.float32)
    for t0, nt, layers in enc:
        p[t0:t0 + nt] = rng.uniform(-1, 1, nt)
    for (o, out, cin) in [l for _, _, ls in enc for l in ls] + dec:
        p[o:o + out * cin] = rng.uniform(-1, 1, out * cin) * np.sqrt(6 / cin) * gain
        p[o + out * cin:o + out * cin + out] = rng.normal(0, 0.1, out)
    return p


def positions(X, Y, Z):
    v = np.arange(X * Y * Z)
    return np.stack([-1 + 2 * (v % X) / (X - 1), -1 + 2 * ((v // X) % Y) / (Y - 1),
                     -1 + 2 * (v // (X * Y)) / (Z - 1)], axis=1).astype(np.float32)


def check(got, want_bf16, want_fp64, what):
    """The kernel does the BF16-operand oracle's roundings; it differs from it only by
    its FP32 summation order and by the BF16 rounding flips that order causes, each
    an error of the same kind and size as the format's own rounding (a flip in the
    reference latent shifts a whole volume).  So the deviation is gated against the
    format's own error on the same vertices, |BF16-operand oracle - FP64 oracle|: at
    most half of it on average and no larger than its largest value, plus the FP32
    summation-order noise where no flip occurs (1e-6 on the mean, 1e-5 at a vertex;
    measured ~1e-7).  Against the FP64 oracle the kernel is then within 1.5x the mean
    and 2x the largest BF16 error by the triangle inequality."""
    e1 = np.abs(got - want_bf16)
    e2 = np.abs(got - want_fp64)
    ebf = np.abs(want_bf16 - want_fp64)
    print(f"{what}: vs bf16 oracle median {np.median(e1):.2e} mean {e1.mean():.2e} max "
          f"{e1.max():.2e} (within 1e-5: {(e1 <= 1e-5).mean():.0%}); vs fp64 mean {e2.mean():.2e} "
          f"max {e2.max():.2e}; bf16 oracle vs fp64 mean {ebf.mean():.2e} max {ebf.max():.2e}; "
          f"output std {want_fp64.std():.3f}")
    assert e1.mean() <= 0.5 * ebf.mean() + 1e-6
    assert e1.max() <= ebf.max() + 1e-5


def oracle_pair(s, p, pos, r, idx):
    pr = np.repeat(pos[r:r + 1].astype(np.float64), len(idx), 0)
    pq = pos[idx].astype(np.float64)
    p64 = p.astype(np.float64)
    return oracle.hash_forward_bf16(s, p64, pr, pq), oracle.hash_forward(s, p64, pr, pq)


@pytest.mark.parametrize("measure", [0, 1])
def test_paper_architecture_vs_oracle(ndf_mod, ctx, measure):
    X, Y, Z = 37, 23, 5  # 4255 vertices: 33 full tiles and a ragged one
    N = X * Y * Z
    a = arch(ndf_mod)
    m = ndf_mod.ndf_hash_model_create(ctx, a, measure, False, 1, X, Y, Z)
    assert ndf_mod.ndf_hash_get_decode(m) == ndf_mod.NDF_HASH_DECODE_TC
    p = make_params(a, 1, 10 + measure)
    ndf_mod.ndf_hash_model_set_params(m, p)
    refs = [0, 1234, N - 1]
    vol = torch.empty((3, N), dtype=torch.float32, device="cuda")
    ndf_mod.ndf_hash_infer_batch(m, refs, vol)
    ndf_mod.ndf_synchronize(ctx)
    got = vol.cpu().numpy()
    pos = positions(X, Y, Z)
    s = oshape(a, False, measure)
    bf, fp_all = oracle_pair(s, p, pos, refs[1], np.arange(N))
    check(got[1], bf, fp_all, f"measure {measure} ref {refs[1]} (all vertices)")
    rng = np.random.default_rng(3)
    for i in (0, 2):
        idx = np.sort(rng.choice(N, 400, replace=False))
        bf, fp = oracle_pair(s, p, pos, refs[i], idx)
        check(got[i][idx], bf, fp, f"measure {measure} ref {refs[i]} (400 vertices)")
    # one reference per call gives the same volume
    single = np.empty(N, np.float32)
    ndf_mod.ndf_hash_infer(m, refs[1], single)
    np.testing.assert_array_equal(single, got[1])
    # the FP32 path on the same model, for scale
    ndf_mod.ndf_hash_set_decode(m, ndf_mod.NDF_HASH_DECODE_FP32)
    f32 = np.empty(N, np.float32)
    ndf_mod.ndf_hash_infer(m, refs[1], f32)
    e32 = np.abs(f32 - fp_all)
    assert np.median(e32) <= 1e-4 and e32.max() <= 5e-3  # FP32 rounding, amplified likewise
    print(f"TC vs FP32 path: mean {np.abs(got[1] - f32).mean():.2e} max {np.abs(got[1] - f32).max():.2e}")
    ndf_mod.ndf_hash_model_free(m)


def test_symmetry_and_cache(ndf_mod, ctx):
    """Self field: R(a, b) == R(b, a) exactly.  Cached query latents: the same
    volumes bit for bit, also after the parameters change."""
    X, Y, Z = 21, 13, 6
    N = X * Y * Z
    a = arch(ndf_mod)
    m = ndf_mod.ndf_hash_model_create(ctx, a, 0, False, 2, X, Y, Z)
    p = make_params(a, 1, 21)
    ndf_mod.ndf_hash_model_set_params(m, p)
    refs = list(range(0, N, 97))
    vol = torch.empty((len(refs), N), dtype=torch.float32, device="cuda")
    ndf_mod.ndf_hash_infer_batch(m, refs, vol)
    ndf_mod.ndf_synchronize(ctx)
    v = vol.cpu().numpy()
    sub = v[:, refs]
    np.testing.assert_array_equal(sub, sub.T)
    ndf_mod.ndf_hash_set_decode(m, ndf_mod.NDF_HASH_DECODE_TC, True)
    cached = torch.empty_like(vol)
    ndf_mod.ndf_hash_infer_batch(m, refs, cached)
    ndf_mod.ndf_synchronize(ctx)
    np.testing.assert_array_equal(cached.cpu().numpy(), v)
    # new parameters: the cache is rebuilt
    p2 = make_params(a, 1, 22)
    ndf_mod.ndf_hash_model_set_params(m, p2)
    ndf_mod.ndf_hash_infer_batch(m, refs, cached)
    ndf_mod.ndf_hash_set_decode(m, ndf_mod.NDF_HASH_DECODE_TC, False)
    fresh = torch.empty_like(vol)
    ndf_mod.ndf_hash_infer_batch(m, refs, fresh)
    ndf_mod.ndf_synchronize(ctx)
    np.testing.assert_array_equal(cached.cpu().numpy(), fresh.cpu().numpy())
    assert not np.array_equal(fresh.cpu().numpy(), v)
    ndf_mod.ndf_hash_model_free(m)


def test_cross_field(ndf_mod, ctx):
    X, Y, Z = 17, 11, 4
    N = X * Y * Z
    a = arch(ndf_mod)
    m = ndf_mod.ndf_hash_model_create(ctx, a, 1, True, 3, X, Y, Z)
    p = make_params(a, 2, 31)
    ndf_mod.ndf_hash_model_set_params(m, p)
    out = np.empty(N, np.float32)
    r = 400
    ndf_mod.ndf_hash_infer(m, r, out)
    bf, fp = oracle_pair(oshape(a, True, 1), p, positions(X, Y, Z), r, np.arange(N))
    check(out, bf, fp, "cross field, MI")
    ndf_mod.ndf_hash_model_free(m)


@pytest.mark.parametrize("act,merge,enc_layers,dec_layers", [
    (0, 0, 2, 2),   # ReLU
    (1, 1, 2, 3),   # Snake, sum merge
    (2, 2, 3, 2),   # SnakeAlt, |difference| merge
    (2, 0, 0, 3),   # grid-only ablation: the merged embedding enters the decoder
    (2, 0, 2, 1),   # no decoder hidden layer: output layer on the merged latent
])
def test_ablations_vs_oracle(ndf_mod, ctx, act, merge, enc_layers, dec_layers):
    X, Y, Z = 19, 9, 7
    N = X * Y * Z
    a = arch(ndf_mod, act=act, merge=merge, enc_layers=enc_layers, dec_layers=dec_layers)
    m = ndf_mod.ndf_hash_model_create(ctx, a, 0, False, 4, X, Y, Z)
    assert ndf_mod.ndf_hash_get_decode(m) == ndf_mod.NDF_HASH_DECODE_TC
    p = make_params(a, 1, 40 + act + 3 * merge + enc_layers)
    ndf_mod.ndf_hash_model_set_params(m, p)
    out = np.empty(N, np.float32)
    r = 77
    ndf_mod.ndf_hash_infer(m, r, out)
    bf, fp = oracle_pair(oshape(a, False, 0), p, positions(X, Y, Z), r, np.arange(N))
    check(out, bf, fp, f"act {act} merge {merge} layers {enc_layers}+{dec_layers}")
    ndf_mod.ndf_hash_model_free(m)


@pytest.mark.parametrize("n_freq,levels,feat", [(3, 5, 1), (0, 6, 2), (5, 3, 4), (12, 6, 2)])
def test_embedding_layouts(ndf_mod, ctx, n_freq, levels, feat):
    """The embedding enters the first layer in operand order: Fourier blocks padded to
    16-byte chunks per axis, then position and grid features.  Frequencies whose
    2 L is not a multiple of 8, no Fourier features, odd feature counts."""
    X, Y, Z = 23, 7, 6
    N = X * Y * Z
    a = arch(ndf_mod, n_freq=n_freq, levels=levels, feat=feat, enc_layers=2, dec_layers=2)
    m = ndf_mod.ndf_hash_model_create(ctx, a, 0, False, 8, X, Y, Z)
    assert ndf_mod.ndf_hash_get_decode(m) == ndf_mod.NDF_HASH_DECODE_TC
    p = make_params(a, 1, 60 + n_freq + levels)
    ndf_mod.ndf_hash_model_set_params(m, p)
    out = np.empty(N, np.float32)
    r = 300
    ndf_mod.ndf_hash_infer(m, r, out)
    bf, fp = oracle_pair(oshape(a, False, 0), p, positions(X, Y, Z), r, np.arange(N))
    check(out, bf, fp, f"L {n_freq} levels {levels} F {feat}")
    ndf_mod.ndf_hash_model_free(m)


def test_small_grids_many_references(ndf_mod, ctx):
    """Fewer vertices than one tile; 70 references (two launches of at most 64)."""
    X, Y, Z = 5, 4, 3
    N = X * Y * Z
    a = arch(ndf_mod, enc_layers=2, dec_layers=2)
    m = ndf_mod.ndf_hash_model_create(ctx, a, 1, False, 5, X, Y, Z)
    p = make_params(a, 1, 51)
    ndf_mod.ndf_hash_model_set_params(m, p)
    refs = [i % N for i in range(70)]
    out = np.empty((70, N), np.float32)  # host output
    ndf_mod.ndf_hash_infer_batch(m, refs, out)
    pos = positions(X, Y, Z)
    s = oshape(a, False, 1)
    for i in (0, 63, 64, 69):
        bf, fp = oracle_pair(s, p, pos, refs[i], np.arange(N))
        check(out[i], bf, fp, f"ref {refs[i]} of 70")
    np.testing.assert_array_equal(out[5], out[65])  # same reference in both launches
    ndf_mod.ndf_hash_model_free(m)


def test_decode_mode_rules(ndf_mod, ctx):
    a = arch(ndf_mod, width=16)
    m = ndf_mod.ndf_hash_model_create(ctx, a, 0, False, 6, 4, 4, 4)
    assert ndf_mod.ndf_hash_get_decode(m) == ndf_mod.NDF_HASH_DECODE_FP32
    with pytest.raises(ndf_mod.NdfError):
        ndf_mod.ndf_hash_set_decode(m, ndf_mod.NDF_HASH_DECODE_TC)
    ndf_mod.ndf_hash_model_free(m)
    a = arch(ndf_mod, dec_layers=1)
    m = ndf_mod.ndf_hash_model_create(ctx, a, 0, False, 6, 4, 4, 4)
    with pytest.raises(ndf_mod.NdfError):
        ndf_mod.ndf_hash_set_decode(m, ndf_mod.NDF_HASH_DECODE_TC, True)  # no layer after the latent
    with pytest.raises(ndf_mod.NdfError):
        ndf_mod.ndf_hash_infer_batch(m, [0, 64], np.empty((2, 64), np.float32))  # 64 out of range
    ndf_mod.ndf_hash_model_free(m)
    a = arch(ndf_mod, merge=3)
    m = ndf_mod.ndf_hash_model_create(ctx, a, 0, False, 6, 4, 4, 4)
    assert ndf_mod.ndf_hash_get_decode(m) == ndf_mod.NDF_HASH_DECODE_FP32  # concatenation
    ndf_mod.ndf_hash_model_free(m)
