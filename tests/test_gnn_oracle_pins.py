"""Pins of the FP64 graph-network oracle (oracle/gnn_oracle.py) against facts
that do not come from the oracle itself: central finite differences of the
loss, a dense-matrix construction of the propagation, permutation
equivariance, closed-form features and a network whose output is derived by
hand. None of these needs a GPU."""

import math

import numpy as np
import pytest

import synth
from oracle import gnn_oracle as go


def _small(seed, n=14, p=0.3):
    g = synth.random_small_graph(n, p, seed, weights="int8", duplicates=3)
    rng = np.random.default_rng(seed + 100)
    s = rng.choice(np.array([-1, 1], np.int8), size=n)
    y = rng.choice(np.array([-1.0, 1.0]), size=n)
    return g, s, y


def test_param_layout_size():
    assert go.NUM_PARAMS == 16 * 64 + 64 + 2 * (128 * 64 + 64) + 64 + 1 == 17665
    assert synth.GNN_NUM_PARAMS == go.NUM_PARAMS
    p = synth.gnn_init_params(3).astype(np.float64)
    assert np.array_equal(go.pack(go.unpack(p)), p)


def test_propagation_equals_dense_matrix_product():
    # Dense route: accumulate the raw (unmerged, duplicated) edge list into a
    # symmetric matrix, normalise by (row sums of |W| + 1)^-1/2 on both sides.
    g = synth.random_small_graph(30, 0.2, 5, weights="int8", duplicates=20)
    W = np.zeros((g.n, g.n))
    np.add.at(W, (g.src, g.dst), g.w)
    np.add.at(W, (g.dst, g.src), g.w)
    c = 1.0 / np.sqrt(np.abs(W).sum(axis=1) + 1.0)
    A = c[:, None] * W * c[None, :]
    h = np.random.default_rng(1).normal(size=(g.n, 7))
    G = go.Graph(g.n, g.src, g.dst, g.w)
    assert np.allclose(G.propagate(h), A @ h, rtol=1e-13, atol=1e-13)


def test_features_closed_form_on_a_unit_torus():
    # 6 x 6 torus, unit weights, all spins +1: deg 4, d 4, f 4, sum w 4.
    g = synth.torus_graph(6, 0, weights="one")
    G = go.Graph(g.n, g.src, g.dst, g.w)
    x = go.features(G, np.ones(g.n, np.int8))
    want = np.array([1, 4 / 5, 4 / 5, math.log(5) / 8, 4 / 5, 1, 0, 0])
    assert np.allclose(x, want[None, :], rtol=0, atol=1e-15)
    # flipping every other spin (checkerboard): f = -4 s_i, s_i f_i = -4
    s = np.array([1 if (i % 6 + i // 6) % 2 == 0 else -1 for i in range(g.n)], np.int8)
    x = go.features(G, s)
    assert np.allclose(x[:, 1], -4 / 5 * s) and np.allclose(x[:, 2], -4 / 5)


def test_hand_derived_two_vertex_network():
    # Vertices 0, 1 joined by one edge of weight 1; spins (+1, -1).
    # d = (1, 1), c = 2^-1/2, A_hat = [[0, 1/2], [1/2, 0]].
    # Layer 0 routes h's feature 0 (the spin) to unit 0 and a's feature 0 to
    # unit 1, bias 2 on both; layers 1 and 2 copy units 0 and 1 from h (their
    # a-half has zero weights); w_o = (1, -1, 0, ...). Then
    # z_i = (s_i + 2) - (a_i + 2) = s_i - s_j / 2: z = (1.5, -1.5).
    p = {name: np.zeros(shape) for name, shape in go.SHAPES}
    p["W0"][0, 0] = 1.0
    p["W0"][8, 1] = 1.0
    p["b0"][:2] = 2.0
    for l in (1, 2):
        p[f"W{l}"][0, 0] = 1.0
        p[f"W{l}"][1, 1] = 1.0
    p["wo"][0], p["wo"][1] = 1.0, -1.0
    G = go.Graph(2, np.array([0]), np.array([1]), np.array([1]))
    x = go.features(G, np.array([1, -1], np.int8))
    z, _ = go.forward(G, x, go.pack(p))
    assert np.allclose(z, [1.5, -1.5], rtol=0, atol=1e-15)


def test_permutation_equivariance():
    g, s, _ = _small(7, n=40, p=0.15)
    params = synth.gnn_init_params(11).astype(np.float64)
    G = go.Graph(g.n, g.src, g.dst, g.w)
    z, _ = go.forward(G, go.features(G, s), params)
    perm = np.random.default_rng(2).permutation(g.n)        # new id of old vertex i
    G2 = go.Graph(g.n, perm[g.src], perm[g.dst], g.w)
    s2 = np.empty_like(s)
    s2[perm] = s
    z2, _ = go.forward(G2, go.features(G2, s2), params)
    assert np.allclose(z2[perm], z, rtol=1e-12, atol=1e-12)


def test_loss_at_zero_logits_and_its_gradient():
    z = np.zeros(10)
    y = np.array([1, -1] * 5, np.float64)
    assert go.loss(z, y) == pytest.approx(math.log(2.0), abs=1e-15)


@pytest.mark.parametrize("seed", [1, 2])
def test_gradient_matches_central_finite_differences(seed):
    g, s, y = _small(seed)
    G = go.Graph(g.n, g.src, g.dst, g.w)
    x = go.features(G, s)
    params = synth.gnn_init_params(seed).astype(np.float64)
    # larger biases keep pre-activations away from the relu kink
    params += np.random.default_rng(seed).normal(scale=0.05, size=params.shape)
    z, cache = go.forward(G, x, params)
    grad = go.backward(G, params, cache, z, y)
    rng = np.random.default_rng(seed + 1)
    idx = np.concatenate([rng.choice(go.NUM_PARAMS, size=300, replace=False),
                          np.arange(go.NUM_PARAMS - 65, go.NUM_PARAMS)])
    eps = 1e-6
    checked = 0
    for k in idx:
        pp, pm = params.copy(), params.copy()
        pp[k] += eps
        pm[k] -= eps
        zp, cp = go.forward(G, x, pp)
        zm, cm = go.forward(G, x, pm)
        if any(np.any((a > 0) != (b > 0)) for a, b in zip(cp["U"], cm["U"])):
            continue                      # the step crossed a relu kink
        fd = (go.loss(zp, y) - go.loss(zm, y)) / (2 * eps)
        assert abs(fd - grad[k]) <= 1e-7 + 1e-5 * abs(fd), (k, fd, grad[k])
        checked += 1
    assert checked > 300


def test_warm_start_and_flip_bias():
    z = np.array([2.0, -0.5, 0.0, 1e-9, -30.0])
    s = np.array([-1, 1, -1, -1, 1], np.int8)
    assert list(go.warm_start(z, s)) == [1, -1, -1, 1, -1]
    q = go.flip_bias(z)
    # sigmoid(-|z|) * 512: 0.1192*512 = 61.0, 0.3775*512 = 193.3, 256 -> 255
    assert list(q) == [61, 193, 255, 255, 0]


def test_bf16_rounding_against_the_library_and_hand_ties():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    v = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-30, 30, 5000),
                        rng.normal(size=2000).astype(np.float32).astype(np.float64)])
    want = torch.tensor(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(go.to_bf16(v), want)
    # bf16 keeps 7 fraction bits: halfway cases go to the even neighbour
    e = 2.0 ** -8
    assert go.to_bf16(1 + e) == 1.0
    assert go.to_bf16(1 + 3 * e) == 1 + 4 * e
    assert go.to_bf16(-(1 + 3 * e)) == -(1 + 4 * e)
    assert go.to_bf16(1 + e + 2.0 ** -20) == 1 + 2 * e
    assert go.to_bf16(0.0) == 0.0 and go.to_bf16(3.0) == 3.0


def test_storage_rounding_rounds_every_stored_operand():
    g, s, y = _small(5, n=40, p=0.2)
    G = go.Graph(g.n, g.src, g.dst, g.w)
    x = go.features(G, s)
    params = synth.gnn_init_params(5).astype(np.float64)
    z, cache = go.forward(G, x, params)
    zr, cr = go.forward(G, x, params, storage="bf16")
    # every tensor-core operand of the rounded form is a bf16 value, the
    # plain form's are not
    for X in cr["X"] + [cr["h3"]]:
        assert np.array_equal(go.to_bf16(X), X)
    assert not all(np.array_equal(go.to_bf16(X), X) for X in cache["X"][1:])
    # rounding moves the result, by about the rounding's relative size
    rel = np.linalg.norm(zr - z) / np.linalg.norm(z)
    assert 0 < rel < 2.0 ** -5
    gp = go.backward(G, params, cache, z, y)
    gr = go.backward(G, params, cr, zr, y, storage="bf16")
    relg = np.linalg.norm(gr - gp) / np.linalg.norm(gp)
    assert 0 < relg < 2.0 ** -4
    with pytest.raises(ValueError):
        go.forward(G, x, params, storage="fp8")
