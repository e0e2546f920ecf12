"""Pins for the oracle of the paper's NDF architecture (Sec. 4.1-4.2): hash-grid
and Fourier input embedding, Snake-family MLP encoders, product merge, decoder.

The backward is pinned against FP64 central differences (independent of the
hand-written chain rule), symmetry of the shared-encoder field is exact, and a
one-channel network isolates single Fourier features and activations, which
must follow their closed forms."""
import math

import numpy as np
import pytest

import oracle


def shape(**kw):
    base = dict(levels=3, base_res=2, log2_table=5, feat=2, n_freq=2, width=6, enc_layers=2,
                dec_layers=2, n_enc=1, measure=0, act=2)
    base.update(kw)
    return oracle.hash_shape(**base)


@pytest.mark.parametrize("act", [1, 2])
@pytest.mark.parametrize("n_enc,measure", [(1, 0), (2, 1)])
def test_gradient_vs_central_differences(act, n_enc, measure):
    # levels: R = 2, 4, 8 -> 8 and 64, 512 entries against 2^5: one dense, two hashed
    s = shape(act=act, n_enc=n_enc, measure=measure, enc_layers=3, dec_layers=3)
    n = oracle.hash_param_count(s)
    rng = np.random.default_rng(act + 10 * n_enc)
    p = rng.normal(0, 0.6, n)
    pr, pq = rng.uniform(-1, 1, (5, 3)), rng.uniform(-1, 1, (5, 3))
    t = rng.uniform(-0.5, 0.5, 5) if measure == 0 else rng.uniform(0.0, 1.5, 5)
    _, g = oracle.hash_loss_grad(s, p, pr, pq, t)
    h = 1e-6
    idx = rng.choice(n, size=min(n, 120), replace=False)
    for i in idx:
        d = np.zeros(n)
        d[i] = h
        num = (oracle.hash_loss_grad(s, p + d, pr, pq, t)[0] -
               oracle.hash_loss_grad(s, p - d, pr, pq, t)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-7 + 1e-6 * abs(g[i]), (i, num, g[i])


def test_shared_encoder_is_symmetric():
    s = shape()
    rng = np.random.default_rng(4)
    p = rng.normal(0, 0.7, oracle.hash_param_count(s))
    a, b = rng.uniform(-1, 1, (50, 3)), rng.uniform(-1, 1, (50, 3))
    np.testing.assert_array_equal(oracle.hash_forward(s, p, a, b), oracle.hash_forward(s, p, b, a))


def one_channel(n_freq, act, enc_layers):
    s = shape(width=1, n_freq=n_freq, act=act, enc_layers=enc_layers, dec_layers=1)
    return s, np.zeros(oracle.hash_param_count(s))


def test_single_fourier_feature_closed_form():
    # width 1, one linear encoder layer selecting feature sin(2^i pi p_j) and a
    # decoder of weight 1: y = tanh(sin(w p_ref,j) * sin(w p_q,j)), w = 2^i pi
    L, levels, F = 4, 3, 2
    s, p = one_channel(L, 2, 1)
    tables = sum(min(2 ** 5, (2 << l) ** 3) * F for l in range(levels))
    din = 3 + 6 * L + levels * F
    j, i = 1, 3
    p[tables + 3 + (j * L + i) * 2] = 1.0      # encoder W[0][sin feature]
    p[tables + din + 1] = 1.0                  # decoder W (after encoder bias)
    rng = np.random.default_rng(5)
    a, b = rng.uniform(-1, 1, (20, 3)), rng.uniform(-1, 1, (20, 3))
    w = (2 ** i) * math.pi
    want = np.tanh(np.sin(w * a[:, j]) * np.sin(w * b[:, j]))
    np.testing.assert_allclose(oracle.hash_forward(s, p, a, b), want, atol=1e-14)
    p[tables + 3 + (j * L + i) * 2] = 0.0
    p[tables + 3 + (j * L + i) * 2 + 1] = 1.0  # the cosine feature instead
    want = np.tanh(np.cos(w * a[:, j]) * np.cos(w * b[:, j]))
    np.testing.assert_allclose(oracle.hash_forward(s, p, a, b), want, atol=1e-14)


@pytest.mark.parametrize("act,f", [(0, lambda x: np.maximum(x, 0.0)),
                                   (1, lambda x: x + np.sin(x) ** 2),
                                   (2, lambda x: 0.5 * x + np.sin(x) ** 2)])
def test_activation_closed_forms(act, f):
    # width 1, two encoder layers: latent = act(p_x); the product merge and a
    # unit decoder give y = tanh(act(p_ref,x) * act(p_q,x))
    s, p = one_channel(0, act, 2)
    tables = sum(min(2 ** 5, (2 << l) ** 3) * 2 for l in range(3))
    din = 3 + 3 * 2
    p[tables + 0] = 1.0            # layer 0: W[0][p_x]
    p[tables + din + 1] = 1.0      # layer 1: W = 1 (after layer-0 bias)
    p[tables + din + 3] = 1.0      # decoder W
    a = np.stack([np.linspace(-1, 1, 11), np.zeros(11), np.zeros(11)], axis=1)
    b = np.stack([np.full(11, 0.7), np.zeros(11), np.zeros(11)], axis=1)
    np.testing.assert_allclose(oracle.hash_forward(s, p, a, b), np.tanh(f(a[:, 0]) * f(b[:, 0])),
                               atol=1e-14)


def test_dense_level_reads_its_vertex_entry():
    # at a vertex of a dense level the trilinear feature is that vertex's entry:
    # fill level 1 (R = 4, 64 entries) with entry = index, read it through a
    # one-channel linear encoder
    s = shape(width=1, n_freq=0, act=2, enc_layers=1, dec_layers=1, log2_table=6, measure=1)
    p = np.zeros(oracle.hash_param_count(s))
    off1 = 8 * 2
    p[off1:off1 + 64 * 2:2] = np.arange(64)   # feature 0 of level 1
    tables = sum(min(2 ** 6, (2 << l) ** 3) * 2 for l in range(3))
    p[tables + 3 + 1 * 2] = 1.0                # encoder picks level 1, feature 0
    p[tables + 3 + 3 * 2 + 1 + 0] = 1.0        # decoder weight
    for x, y, z in [(0, 0, 0), (3, 1, 2), (1, 3, 3)]:
        pos = np.array([[-1 + 2 * x / 3, -1 + 2 * y / 3, -1 + 2 * z / 3]])
        # the same position twice: softplus(entry^2) with entry = x + 4 y + 16 z
        e2 = float(x + 4 * y + 16 * z) ** 2
        want = math.log1p(math.exp(-e2)) + e2
        assert oracle.hash_forward(s, p, pos, pos)[0] == pytest.approx(want, rel=1e-12)


def test_hashed_level_reads_one_entry_per_vertex():
    # level 2 (R = 8, 512 vertices) over a 64-entry table is hashed.  With entry =
    # index, a vertex must read exactly one entry (trilinear weight 1), and along
    # x the index must change as index(0, y, z) XOR x: the x coordinate enters the
    # spatial hash with multiplier 1 and the coordinates combine by XOR, so the 8
    # vertices of an x-row fill one aligned block of 8 entries (an additive
    # combination, or another x multiplier, breaks this)
    s = shape(width=1, n_freq=0, act=2, enc_layers=1, dec_layers=1, log2_table=6, measure=1)
    p = np.zeros(oracle.hash_param_count(s))
    off2 = 8 * 2 + 64 * 2
    p[off2:off2 + 64 * 2:2] = np.arange(64)   # feature 0 of level 2
    tables = sum(min(2 ** 6, (2 << l) ** 3) * 2 for l in range(3))
    p[tables + 3 + 2 * 2] = 1.0                # encoder picks level 2, feature 0
    p[tables + 3 + 3 * 2 + 1 + 0] = 1.0        # decoder weight
    g = np.arange(8)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([-1 + 2 * X / 7, -1 + 2 * Y / 7, -1 + 2 * Z / 7], axis=-1).reshape(-1, 3)
    out = oracle.hash_forward(s, p, pos, pos)
    cand = np.arange(64, dtype=np.float64) ** 2
    cand = np.log1p(np.exp(-cand)) + cand      # softplus(entry^2), as for the dense level
    diff = np.abs(out[:, None] - cand[None, :])
    e = diff.argmin(axis=1)
    assert (diff[np.arange(len(e)), e] <= 1e-9 * cand[e]).all()
    e = e.reshape(8, 8, 8)
    for y in range(8):
        for z in range(8):
            np.testing.assert_array_equal(e[:, y, z] ^ e[0, y, z], g)
    assert len(np.unique(e)) > 32  # the hash spreads the 512 vertices over the table


@pytest.mark.parametrize("merge,enc_layers", [(1, 2), (2, 2), (3, 2), (0, 0), (3, 0)])
def test_ablations_gradient_vs_central_differences(merge, enc_layers):
    # merge: 1 sum, 2 |difference|, 3 concatenation; enc_layers = 0: grid only
    s = shape(merge=merge, enc_layers=enc_layers, n_enc=2 if merge == 3 else 1)
    n = oracle.hash_param_count(s)
    rng = np.random.default_rng(merge * 10 + enc_layers)
    p = rng.normal(0, 0.6, n)
    pr, pq = rng.uniform(-1, 1, (4, 3)), rng.uniform(-1, 1, (4, 3))
    t = rng.uniform(-0.5, 0.5, 4)
    _, g = oracle.hash_loss_grad(s, p, pr, pq, t)
    h = 1e-6
    for i in rng.choice(n, size=min(n, 100), replace=False):
        d = np.zeros(n)
        d[i] = h
        num = (oracle.hash_loss_grad(s, p + d, pr, pq, t)[0] -
               oracle.hash_loss_grad(s, p - d, pr, pq, t)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-7 + 1e-6 * abs(g[i]), (i, num, g[i])


def test_merge_symmetry():
    # with one shared encoder, sum and |difference| are symmetric, concatenation is not
    rng = np.random.default_rng(8)
    a, b = rng.uniform(-1, 1, (30, 3)), rng.uniform(-1, 1, (30, 3))
    for merge, sym in ((1, True), (2, True), (3, False)):
        s = shape(merge=merge)
        p = rng.normal(0, 0.7, oracle.hash_param_count(s))
        fa, fb = oracle.hash_forward(s, p, a, b), oracle.hash_forward(s, p, b, a)
        assert np.array_equal(fa, fb) == sym


def test_grid_only_latent_is_the_embedding():
    # enc_layers = 0: with a one-layer linear decoder of weight e_j and product
    # merge, y = tanh(x0_j(p_ref) * x0_j(p_q)); x0_0 is p_x
    s = shape(enc_layers=0, dec_layers=1, n_freq=1)
    p = np.zeros(oracle.hash_param_count(s))
    tables = sum(min(2 ** 5, (2 << l) ** 3) * 2 for l in range(3))
    p[tables + 0] = 1.0  # decoder W[0][0]: coordinate x
    rng = np.random.default_rng(9)
    a, b = rng.uniform(-1, 1, (10, 3)), rng.uniform(-1, 1, (10, 3))
    np.testing.assert_allclose(oracle.hash_forward(s, p, a, b), np.tanh(a[:, 0] * b[:, 0]),
                               atol=1e-15)


# ---- the BF16-operand forward (the arithmetic of the tensor-core decoder)

def test_bf16_round_values():
    """Round to nearest BF16 (8 significant bits), ties to even."""
    r = oracle.bf16_round
    assert r(1.0) == 1.0 and r(-2.5) == -2.5 and r(0.0) == 0.0
    assert r(1 + 2 ** -8) == 1.0                      # tie, 1.0000000 is even
    assert r(1 + 3 * 2 ** -8) == 1 + 2 ** -6          # tie, 1.0000001 is odd: up
    assert r(1 + 2 ** -8 + 2 ** -20) == 1 + 2 ** -7   # above the tie: up
    assert r(0.1) == 0.10009765625                    # 1.1001101 x 2^-4
    assert r(-(1 + 2 ** -9)) == -1.0                  # below the tie: down
    assert math.isinf(r(1e39)) and math.isnan(r(float("nan")))


def _offsets(s):
    """Offsets of the flat parameter layout of the header: tables, encoder layers, decoder layers."""
    din = 3 + 6 * s.n_freq + s.levels * s.feat
    ent = [min((s.base_res << l) ** 3, 2 ** s.log2_table) for l in range(s.levels)]
    o = sum(ent) * s.feat
    enc = []
    for k in range(s.enc_layers):
        cin = din if k == 0 else s.width
        enc.append((o, s.width, cin, o + cin * s.width))
        o += cin * s.width + s.width
    o *= s.n_enc
    dec = []
    for k in range(s.dec_layers):
        out = 1 if k == s.dec_layers - 1 else s.width
        cin = (s.width if s.enc_layers else din) if k == 0 else s.width
        dec.append((o, out, cin, o + cin * out))
        o += cin * out + out
    assert o == oracle.hash_param_count(s)
    return dict(din=din, ent=ent, enc=enc, dec=dec)


def _constant_tables(s, p, values):
    """Every entry of level l, feature f holds values[l][f] (BF16-exact), so that
    the trilinear feature of any position is that value."""
    o = 0
    for l, e in enumerate(_offsets(s)["ent"]):
        for f in range(s.feat):
            p[o + f:o + e * s.feat:s.feat] = values[l][f]
        o += e * s.feat


def _rounded(p, layers):
    q = p.copy()
    for (w, out, cin, _) in layers:
        q[w:w + out * cin] = [oracle.bf16_round(x) for x in p[w:w + out * cin]]
    return q


VALS = [[0.75, -1.25], [0.5, 1.5]]  # BF16-exact, and so are their squares


def test_bf16_forward_rounds_encoder_weights_only():
    """One encoder layer, output layer on the merged latent.  At p = 0 the embedding
    [0, 0, 0, sin 0, cos 0, table values] is BF16-exact, so the BF16 forward must
    equal the FP64 forward with the encoder weights rounded and everything else
    (latent, merge, output layer) untouched."""
    s = shape(levels=2, base_res=2, log2_table=5, n_freq=1, width=8, enc_layers=1, dec_layers=1,
              act=0)
    off = _offsets(s)
    p = np.random.default_rng(5).normal(0, 0.7, oracle.hash_param_count(s))
    _constant_tables(s, p, VALS)
    z = np.zeros((1, 3))
    got = oracle.hash_forward_bf16(s, p, z, z)
    want = oracle.hash_forward(s, _rounded(p, off["enc"]), z, z)
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=0)
    assert abs(got[0] - oracle.hash_forward(s, p, z, z)[0]) > 1e-6  # the rounding mattered


def test_bf16_forward_rounds_hidden_decoder_weights_only():
    """Grid-only network (no encoder layer), one hidden decoder layer.  At p = 0 the
    merged latent x0 * x0 = [0, 0, 0, 0, 1, values^2] is BF16-exact: the BF16 forward
    equals the FP64 forward with the hidden layer's weights rounded; the output layer
    (weights and inputs) is not rounded."""
    s = shape(levels=2, base_res=2, log2_table=5, n_freq=1, width=8, enc_layers=0, dec_layers=2,
              act=0)
    off = _offsets(s)
    p = np.random.default_rng(6).normal(0, 0.7, oracle.hash_param_count(s))
    _constant_tables(s, p, VALS)
    z = np.zeros((1, 3))
    got = oracle.hash_forward_bf16(s, p, z, z)
    want = oracle.hash_forward(s, _rounded(p, off["dec"][:1]), z, z)
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=0)
    assert abs(got[0] - oracle.hash_forward(s, _rounded(p, off["dec"]), z, z)[0]) > 1e-6


def test_bf16_forward_rounds_layer_inputs():
    """No Fourier features, constant tables, one encoder layer with BF16-exact weights:
    the BF16 forward is out(w . (h(p_r) * h(p_q)) + b) with h(p) = W [bf16(p), values] + b1,
    i.e. the positions enter the product rounded."""
    s = shape(levels=2, base_res=2, log2_table=5, n_freq=0, width=8, enc_layers=1, dec_layers=1,
              act=0, measure=1)
    off = _offsets(s)
    p = np.random.default_rng(7).normal(0, 0.7, oracle.hash_param_count(s))
    _constant_tables(s, p, VALS)
    p = _rounded(p, off["enc"])
    (w1, c, din, b1), = off["enc"]
    (wo, _, _, bo), = off["dec"]
    W, b, wout = p[w1:w1 + c * din].reshape(c, din), p[b1:b1 + c], p[wo:wo + c]
    pr, pq = np.array([[1 / 3, -0.7, 0.1]]), np.array([[0.3, 0.45, -0.9]])

    def h(pos, rnd):
        x = np.concatenate([[rnd(v) for v in pos[0]], [VALS[0][0], VALS[0][1], VALS[1][0], VALS[1][1]]])
        return W @ x + b

    def soft(x):
        return math.log1p(math.exp(-abs(x))) + max(x, 0.0)

    got = oracle.hash_forward_bf16(s, p, pr, pq)[0]
    want = soft(wout @ (h(pr, oracle.bf16_round) * h(pq, oracle.bf16_round)) + p[bo])
    assert got == pytest.approx(want, rel=1e-12, abs=1e-14)
    plain = soft(wout @ (h(pr, float) * h(pq, float)) + p[bo])
    assert abs(got - plain) > 1e-6
