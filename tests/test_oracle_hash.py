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
