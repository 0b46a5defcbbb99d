"""GPU parity of the flip bias (bit-exact against the oracle) and of the
warm-start network (logits and gradients against the FP64 oracle).

The network's arithmetic is bf16 operands with fp32 accumulation: the GPU
uses bf16-rounded weights W_0..W_2 (the oracle is given the same rounded
values) and keeps every activation in bf16 between kernels. Two oracle forms
are compared:

* the plain FP64 network (no activation rounding). Logits agree within the
  stated 1e-2 relative tolerance in norm; element-wise the activation
  rounding alone (relative 2^-9 per stored value) moves a logit by up to
  2 % of |z| plus the rms logit, the bar used there.
* the FP64 network with the same storage rounding (oracle `storage="bf16"`:
  every value the GPU stores as bf16 is rounded at the same point, all sums
  stay in float64). Against it every logit must agree to 1e-2 relative,
  with a floor for logits that cancel their terms: |z - z_ref| <= 1e-2 *
  max(|z_ref|, t / 2), t = sum_k |h3_k w_o,k| + |b_o| the size of the
  logit's terms. At init a logit is a sum of 64 terms of either sign, so
  |z| is often a tenth of t; there the error is set by the terms' rounding,
  which fp32 and float64 resolve differently at about 1e-4 of the stored
  values (a value whose fp32 and float64 results fall on either side of a
  bf16 rounding boundary). An fp32 emulation of the network puts the
  largest |dz| / t at 2.6e-3.

Gradients are compared per parameter block at 1e-2 in norm against both
forms, and element by element against the rounded form with the same
floor rule (t the sum of the absolute terms of the element's sum, t / 4 as
the floor). One relu whose pre-activation is within fp32 rounding of zero
can switch sides between fp32 and float64 and move whole gradient entries,
so the element-wise bar holds for all but 1 in 1000 entries and every entry
stays within 1e-1. The labels agree with the input spins on 80 % of the
vertices (as annealer labels do); with labels independent of the input the
gradient is a sum that almost cancels and its relative error is not bounded
by the arithmetic, so that case is not used. The 64 x 64 torus with +-1
weights is left out of the element-wise gradient check: its vertices share
a handful of feature vectors, so one pre-activation near zero is shared by
thousands of vertices.
"""

import numpy as np
import pytest

import synth
import oracle
from oracle import gnn_oracle as go

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1807_10750_gb300")


def bf16_round(x):
    """Round float32 values to the nearest bf16 (ties to even)."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def effective_params(params):
    """The parameters the GPU computes with: W_0..W_2 in bf16, the rest fp32."""
    d = go.unpack(np.asarray(params, np.float32).astype(np.float64))
    for l in range(3):
        d[f"W{l}"] = bf16_round(d[f"W{l}"]).astype(np.float64)
    return go.pack(d)


GRAPHS = {
    "er_int8": lambda: synth.random_small_graph(3000, 0.004, 3, weights="int8", duplicates=50),
    "torus_pm1": lambda: synth.torus_graph(64, 1, weights="pm1"),
    "zipf_hubs": lambda: synth.zipf_config_graph(20011, 2.1, 4, 3000, 5),
    "int32_weights": lambda: synth.Graph(
        *(lambda g: (g.n, g.src, g.dst, (g.w * 300).astype(np.int32)))(
            synth.random_small_graph(1500, 0.01, 9, weights="int8"))),
}


def _spins(n, seed):
    return np.random.default_rng(seed).choice(np.array([-1, 1], np.int8), size=n)


def _norm_rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("pseed", [1, 2])
def test_logits_match_fp64_oracle(name, pseed):
    g = GRAPHS[name]()
    s = _spins(g.n, 7)
    params = synth.gnn_init_params(pseed)
    with P.ising_create(g.n, g.src, g.dst, g.w) as h, P.ising_gnn_create(params) as net:
        P.ising_set_spins(h, s)
        z = P.ising_gnn_forward(net, h)
    G = go.Graph(g.n, g.src, g.dst, g.w)
    pe = effective_params(params)
    x = go.features(G, s)
    # the plain FP64 network
    z_or, _ = go.forward(G, x, pe)
    assert _norm_rel(z, z_or) <= 1e-2
    scale = np.abs(z_or) + np.sqrt(np.mean(z_or ** 2))
    assert np.all(np.abs(z - z_or) <= 5e-2 * scale)
    # the FP64 network with the GPU's storage rounding: 1e-2 element-wise
    z_rd, cache = go.forward(G, x, pe, storage="bf16")
    d = go.unpack(pe)
    t = np.abs(cache["h3"]) @ np.abs(d["wo"]) + abs(d["bo"][0])
    err = np.abs(z.astype(np.float64) - z_rd)
    ratio = err / np.maximum(np.abs(z_rd), t / 2)
    print(f"{name} seed {pseed}: max |dz| / max(|z|, t/2) = {ratio.max():.2e}, max |dz| / t = "
          f"{(err / t).max():.2e}, logits at the floor {np.mean(np.abs(z_rd) < t / 2):.2f}")
    assert np.all(ratio <= 1e-2), (int(np.argmax(ratio)), float(ratio.max()))


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_tcgen05_and_mma_sync_layers_agree_and_match_the_oracle(name):
    # the forward layers' products on the fifth-generation tensor cores
    # (tcgen05, accumulator in tensor memory) and on mma.sync: the same bf16
    # operands, fp32 sums in a different order
    g = GRAPHS[name]()
    s = _spins(g.n, 5)
    params = synth.gnn_init_params(2)
    out = {}
    with P.ising_create(g.n, g.src, g.dst, g.w) as h, P.ising_gnn_create(params) as net:
        P.ising_set_spins(h, s)
        for path in (P.ISING_GNN_DENSE_TCGEN05, P.ISING_GNN_DENSE_MMA_SYNC):
            P.ising_gnn_set_dense_path(net, path)
            out[path] = P.ising_gnn_forward(net, h).astype(np.float64)
        with pytest.raises(P.IsingError):
            P.ising_gnn_set_dense_path(net, 7)
    G = go.Graph(g.n, g.src, g.dst, g.w)
    pe = effective_params(params)
    d = go.unpack(pe)
    z_rd, cache = go.forward(G, go.features(G, s), pe, storage="bf16")
    t = np.abs(cache["h3"]) @ np.abs(d["wo"]) + abs(d["bo"][0])
    for path, z in out.items():
        ratio = np.abs(z - z_rd) / np.maximum(np.abs(z_rd), t / 2)
        assert np.all(ratio <= 1e-2), (path, float(ratio.max()))
    a, b = out[P.ISING_GNN_DENSE_TCGEN05], out[P.ISING_GNN_DENSE_MMA_SYNC]
    assert np.all(np.abs(a - b) <= 1e-2 * np.maximum(np.abs(b), t / 2))
    assert _norm_rel(a, b) <= 1e-3


def test_tcgen05_pipeline_wraps_its_ring_on_a_large_graph():
    # 150,001 vertices: 1,172 tiles of 128 rows (the last one 113 rows) over
    # one persistent block per SM, so every block passes through its ring of
    # shared-memory stages and its two accumulators several times
    g = synth.er_graph(150_001, 10.0 / 150_000, 12, weights="int8")
    s = _spins(g.n, 6)
    params = synth.gnn_init_params(3)
    out = {}
    with P.ising_create(g.n, g.src, g.dst, g.w) as h, P.ising_gnn_create(params) as net:
        P.ising_set_spins(h, s)
        for path in (P.ISING_GNN_DENSE_TCGEN05, P.ISING_GNN_DENSE_MMA_SYNC):
            P.ising_gnn_set_dense_path(net, path)
            out[path] = P.ising_gnn_forward(net, h).astype(np.float64)
    G = go.Graph(g.n, g.src, g.dst, g.w)
    pe = effective_params(params)
    d = go.unpack(pe)
    z_rd, cache = go.forward(G, go.features(G, s), pe, storage="bf16")
    t = np.abs(cache["h3"]) @ np.abs(d["wo"]) + abs(d["bo"][0])
    for path, z in out.items():
        ratio = np.abs(z - z_rd) / np.maximum(np.abs(z_rd), t / 2)
        assert np.all(ratio <= 1e-2), (path, int(np.argmax(ratio)), float(ratio.max()))
    a, b = out[P.ISING_GNN_DENSE_TCGEN05], out[P.ISING_GNN_DENSE_MMA_SYNC]
    assert _norm_rel(a, b) <= 1e-3


def test_logits_of_edgeless_and_single_vertex_graphs():
    params = synth.gnn_init_params(4)
    e = np.zeros(0, np.int32)
    for n in (1, 100):
        s = _spins(n, 3)
        with P.ising_create(n, e, e, e) as h, P.ising_gnn_create(params) as net:
            P.ising_set_spins(h, s)
            z = P.ising_gnn_forward(net, h)
        G = go.Graph(n, e, e, e)
        pe = effective_params(params)
        z_or, cache = go.forward(G, go.features(G, s), pe)
        # a logit is a dot product that may nearly cancel: bound its error by
        # the magnitude of its terms
        d = go.unpack(pe)
        terms = np.abs(cache["h3"]) @ np.abs(d["wo"]) + abs(d["bo"][0])
        assert np.all(np.abs(z - z_or) <= 1e-2 * terms)


def _gradient_terms(G, params, cache, z, y):
    """Per parameter, the sum of the absolute terms of its gradient sum in the
    rounded oracle form (the same chain rule with every product taken in
    absolute value at the last step)."""
    p = go.unpack(params)
    n = z.shape[0]
    dz = -y / (1.0 + np.exp(y * z)) / n
    T = {"wo": np.abs(cache["h3"]).T @ np.abs(dz), "bo": np.array([np.abs(dz).sum()])}
    dh = dz[:, None] * p["wo"][None, :]
    for l in reversed(range(3)):
        dU = dh * (cache["U"][l] > 0.0)
        dUr = go.to_bf16(dU)
        T[f"W{l}"] = np.abs(cache["X"][l]).T @ np.abs(dUr)
        T[f"b{l}"] = np.abs(dU).sum(axis=0)
        if l > 0:
            dX = dUr @ p[f"W{l}"].T
            dh = dX[:, :64] + G.propagate(go.to_bf16(dX[:, 64:]))
    return go.pack(T)


@pytest.mark.parametrize("name", ["er_int8", "zipf_hubs", "torus_pm1", "int32_weights"])
def test_gradients_match_fp64_oracle(name):
    g = GRAPHS[name]()
    s = _spins(g.n, 11)
    rng = np.random.default_rng(12)
    y = np.where(rng.random(g.n) < 0.8, s, -s).astype(np.int8)
    params = synth.gnn_init_params(3)
    with P.ising_create(g.n, g.src, g.dst, g.w) as h, P.ising_gnn_create(params) as net:
        P.ising_set_spins(h, s)
        loss, grad = P.ising_gnn_gradients(net, h, y)
    G = go.Graph(g.n, g.src, g.dst, g.w)
    pe = effective_params(params)
    x = go.features(G, s)
    yf = y.astype(np.float64)
    z_or, cache = go.forward(G, x, pe)
    assert loss == pytest.approx(go.loss(z_or, yf), rel=1e-3)
    g_or = go.backward(G, pe, cache, z_or, yf)
    z_rd, cache_rd = go.forward(G, x, pe, storage="bf16")
    g_rd = go.backward(G, pe, cache_rd, z_rd, yf, storage="bf16")
    t = _gradient_terms(G, pe, cache_rd, z_rd, yf)
    k = 0
    elementwise = name != "torus_pm1"
    report = []
    for blk, shape in go.SHAPES:
        size = int(np.prod(shape))
        sl = slice(k, k + size)
        assert _norm_rel(grad[sl], g_or[sl]) <= 1e-2, blk
        assert _norm_rel(grad[sl], g_rd[sl]) <= 1e-2, blk
        err = np.abs(grad[sl].astype(np.float64) - g_rd[sl])
        tt = t[sl]
        ratio = err / np.maximum(np.abs(g_rd[sl]), np.maximum(tt, 1e-300) / 4)
        ratio[tt == 0] = 0.0
        report.append(f"{blk} {ratio.max():.1e} ({int(np.sum(ratio > 1e-2))} > 1e-2)")
        if elementwise:
            # an entry whose terms are all zero (a unit that never fires) is
            # an exact zero on both sides
            assert np.all(err[tt == 0] == 0), blk
            assert np.all(ratio <= 1e-1), (blk, int(np.argmax(ratio)), float(ratio.max()))
            assert np.sum(ratio > 1e-2) <= size // 1000, (blk, int(np.sum(ratio > 1e-2)))
        k += size
    print(name, "; ".join(report))


def test_warm_start_and_bias_follow_the_logits():
    g = GRAPHS["zipf_hubs"]()
    s = _spins(g.n, 5)
    params = synth.gnn_init_params(6)
    with P.ising_create(g.n, g.src, g.dst, g.w) as h, P.ising_gnn_create(params) as net:
        P.ising_set_spins(h, s)
        z = P.ising_gnn_forward(net, h)
        P.ising_gnn_warm_start(net, h, set_bias=True)
        s2 = P.ising_get_spins(h)
        q = P.ising_get_flip_bias(h)
    # the warm start ran its own forward pass, which sums every aggregate in
    # a fixed order: the same logits, so the same decisions everywhere
    assert np.array_equal(s2, go.warm_start(z, s))
    qw = go.flip_bias(z.astype(np.float32))
    assert np.max(np.abs(q.astype(int) - qw.astype(int))) <= 1


def test_forward_is_deterministic():
    g = GRAPHS["zipf_hubs"]()
    s = _spins(g.n, 9)
    with P.ising_create(g.n, g.src, g.dst, g.w) as h, P.ising_gnn_create(synth.gnn_init_params(8)) as net:
        P.ising_set_spins(h, s)
        z1 = P.ising_gnn_forward(net, h)
        P.ising_gnn_gradients(net, h, s)   # reuses the workspace in between
        z2 = P.ising_gnn_forward(net, h)
    assert np.array_equal(z1.view(np.uint32), z2.view(np.uint32))


def _batch_graphs():
    """Instances of uneven sizes; one has hubs (rows summed by chunks), one
    no edges at all."""
    gs = [synth.er_graph(n, 10.0 / (n - 1), 40 + k, weights="pm1") for k, n in enumerate((700, 3100, 1500))]
    gs.append(synth.zipf_config_graph(6000, 2.0, 3, 1500, 44, weights="pm1"))
    gs.append(synth.Graph(300, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32)))
    gs.append(synth.er_graph(2200, 10.0 / 2199, 46, weights="pm1"))
    return gs


def test_batch_forward_matches_the_oracle_per_instance():
    gs = _batch_graphs()
    params = synth.gnn_init_params(3)
    pe = effective_params(params)
    d = go.unpack(pe)
    with P.ising_batch_create([(g.n, g.src, g.dst, g.w) for g in gs], replicas=3) as b, \
            P.ising_gnn_create(params) as net:
        P.ising_batch_init_random(b, 5)
        for r in (0, 2):
            z = P.ising_gnn_batch_forward(net, b, replica=r)
            off = 0
            for k, g in enumerate(gs):
                s = P.ising_batch_get_spins(b, k, r)
                G = go.Graph(g.n, g.src, g.dst, g.w)
                z_rd, cache = go.forward(G, go.features(G, s), pe, storage="bf16")
                zk = z[off:off + g.n].astype(np.float64)
                t = np.abs(cache["h3"]) @ np.abs(d["wo"]) + abs(d["bo"][0])
                ratio = np.abs(zk - z_rd) / np.maximum(np.abs(z_rd), t / 2)
                assert np.all(ratio <= 1e-2), (r, k, float(ratio.max()))
                # an instance alone gives the same logits as inside the batch
                with P.ising_create(g.n, g.src, g.dst, g.w) as h:
                    P.ising_set_spins(h, s)
                    assert np.array_equal(P.ising_gnn_forward(net, h), z[off:off + g.n])
                off += g.n
        with pytest.raises(P.IsingError) as e:
            P.ising_gnn_batch_forward(net, b, replica=3)
        assert e.value.code == P.ISING_EINVAL


def test_batch_warm_start_sets_each_replica_from_its_own_logits():
    gs = _batch_graphs()
    with P.ising_batch_create([(g.n, g.src, g.dst, g.w) for g in gs], replicas=4) as b, \
            P.ising_gnn_create(synth.gnn_init_params(4)) as net:
        P.ising_batch_init_random(b, 8)
        before = [[P.ising_batch_get_spins(b, k, r) for k in range(len(gs))] for r in range(4)]
        zs = [P.ising_gnn_batch_forward(net, b, replica=r) for r in range(4)]
        P.ising_gnn_batch_warm_start(net, b, replica=1)
        mid = [[P.ising_batch_get_spins(b, k, r) for k in range(len(gs))] for r in range(4)]
        P.ising_gnn_batch_warm_start(net, b)   # every replica
        after = [[P.ising_batch_get_spins(b, k, r) for k in range(len(gs))] for r in range(4)]
    for r in range(4):
        off = 0
        for k, g in enumerate(gs):
            want = go.warm_start(zs[r][off:off + g.n], before[r][k])
            assert np.array_equal(mid[r][k], want if r == 1 else before[r][k]), (r, k)
            if r != 1:
                assert np.array_equal(after[r][k], want), (r, k)
            off += g.n


def _union(gs):
    """The disjoint union of the instances, vertex ids offset instance by
    instance (the layout of the batched logits and labels)."""
    off = np.cumsum([0] + [g.n for g in gs])
    src = np.concatenate([g.src.astype(np.int64) + o for g, o in zip(gs, off)])
    dst = np.concatenate([g.dst.astype(np.int64) + o for g, o in zip(gs, off)])
    w = np.concatenate([g.w for g in gs])
    return go.Graph(int(off[-1]), src, dst, w)


def test_batch_gradients_match_the_oracle_on_the_union():
    gs = _batch_graphs()
    params = synth.gnn_init_params(3)
    pe = effective_params(params)
    with P.ising_batch_create([(g.n, g.src, g.dst, g.w) for g in gs], replicas=2) as b, \
            P.ising_gnn_create(params) as net:
        P.ising_batch_init_random(b, 12)
        s = np.concatenate([P.ising_batch_get_spins(b, k, 1) for k in range(len(gs))])
        y = np.where(np.random.default_rng(13).random(s.size) < 0.8, s, -s).astype(np.int8)
        loss, grad = P.ising_gnn_batch_gradients(net, b, y, replica=1)
        # the train step's loss is the loss before its update
        assert P.ising_gnn_batch_train_step(net, b, y, lr=1e-3, replica=1, want_loss=True) == pytest.approx(loss, rel=1e-6)
    G = _union(gs)
    x = go.features(G, s)
    yf = y.astype(np.float64)
    z_rd, cache = go.forward(G, x, pe, storage="bf16")
    assert loss == pytest.approx(go.loss(z_rd, yf), rel=1e-3)
    g_rd = go.backward(G, pe, cache, z_rd, yf, storage="bf16")
    t = _gradient_terms(G, pe, cache, z_rd, yf)
    k = 0
    for blk, shape in go.SHAPES:
        size = int(np.prod(shape))
        sl = slice(k, k + size)
        assert _norm_rel(grad[sl], g_rd[sl]) <= 1e-2, blk
        err = np.abs(grad[sl].astype(np.float64) - g_rd[sl])
        ratio = err / np.maximum(np.abs(g_rd[sl]), np.maximum(t[sl], 1e-300) / 4)
        ratio[t[sl] == 0] = 0.0
        assert np.all(ratio <= 1e-1), blk
        assert np.sum(ratio > 1e-2) <= size // 1000, blk
        k += size


@pytest.mark.parametrize("engine", ["phase", "persistent", "dataflow"])
@pytest.mark.parametrize("mode", ["det", "racy"])
def test_flip_bias_anneal_matches_oracle(engine, mode):
    g = synth.random_small_graph(700, 0.02, 17, weights="int8")
    q = np.random.default_rng(3).integers(0, 256, size=g.n).astype(np.uint8)
    eng = {"phase": P.ISING_ENGINE_PHASE, "persistent": P.ISING_ENGINE_PERSISTENT,
           "dataflow": P.ISING_ENGINE_DATAFLOW}[engine]
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        P.ising_set_engine(h, eng)
        P.ising_init_random(h, 4)
        s0 = P.ising_get_spins(h)
        P.ising_set_flip_bias(h, q)
        assert np.array_equal(P.ising_get_flip_bias(h), q)
        md = P.ISING_MODE_DET if mode == "det" else P.ISING_MODE_RACY
        P.ising_anneal(h, p0=0.3, t_total=60, seed=8, mode=md)
        s1 = P.ising_get_spins(h)
        cut = P.ising_cut(h)
    want = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=8, p0=0.3, T=60, bias=q)
    if mode == "det":
        assert np.array_equal(s1, want)
    else:
        # racy: judged by cut only (a sanity bound against the biased
        # deterministic run; the racy pass's quality is tested elsewhere)
        _, _, cut_det = oracle.energy_cut(g.n, g.src, g.dst, g.w, want)
        assert cut >= 0.9 * cut_det


def test_bias_128_and_removal_reproduce_the_unbiased_anneal():
    g = synth.random_small_graph(500, 0.03, 2, weights="int8")
    out = []
    for q in (None, np.full(g.n, 128, np.uint8), "removed"):
        with P.ising_create(g.n, g.src, g.dst, g.w) as h:
            P.ising_init_random(h, 1)
            if q is not None:
                P.ising_set_flip_bias(h, np.zeros(g.n, np.uint8) if isinstance(q, str) else q)
            if isinstance(q, str):
                P.ising_set_flip_bias(h, None)
            P.ising_anneal(h, p0=0.2, t_total=50, seed=3)
            out.append(P.ising_get_spins(h))
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_gnn_argument_errors():
    g = synth.random_small_graph(50, 0.1, 1)
    params = synth.gnn_init_params(1)
    with P.ising_create(g.n, g.src, g.dst, g.w) as h, P.ising_gnn_create(params) as net:
        with pytest.raises(P.IsingError) as e:
            P.ising_gnn_gradients(net, h, np.zeros(g.n, np.int8))
        assert e.value.code == P.ISING_EINVAL
        with pytest.raises(P.IsingError) as e:
            P.ising_get_flip_bias(h)
        assert e.value.code == P.ISING_ESTATE
        bad = params.copy()
        bad[5] = np.nan
        with pytest.raises(P.IsingError):
            P.ising_gnn_set_params(net, bad)
        with pytest.raises(ValueError):
            P.ising_gnn_create(params[:-1])
        assert np.array_equal(P.ising_gnn_get_params(net), params)


def test_training_on_annealer_labels_lowers_the_loss():
    # a few generated graphs; the input spins are a short hot anneal, the
    # labels the spins a longer cool anneal continues to from there
    graphs = [synth.zipf_config_graph(4000, 2.1, 4, 400, 100 + k, weights="int8") for k in range(4)]
    params = synth.gnn_init_params(5)
    with P.ising_gnn_create(params) as net:
        hs, snaps, labels = [], [], []
        for k, g in enumerate(graphs):
            h = P.ising_create(g.n, g.src, g.dst, g.w)
            P.ising_init_random(h, k)
            P.ising_anneal(h, p0=0.1, t_total=200, seed=k, sweeps=20)
            snap = P.ising_get_spins(h)
            P.ising_anneal(h, p0=0.02, t_total=400, seed=50 + k)
            labels.append(P.ising_get_spins(h))
            P.ising_set_spins(h, snap)
            hs.append(h)
            snaps.append(snap)
        first = [P.ising_gnn_gradients(net, h, y)[0] for h, y in zip(hs, labels)]
        for it in range(150):
            k = it % len(hs)
            P.ising_gnn_train_step(net, hs[k], labels[k], lr=3e-3)
        last = [P.ising_gnn_gradients(net, h, y)[0] for h, y in zip(hs, labels)]
        for h in hs:
            h.close()
    # the labels are only partly predictable from the snapshot; 150 steps
    # took the loss from 0.694 to 0.631 when this test was written
    assert np.mean(last) < np.mean(first) - 0.03


def test_trained_network_gains_over_plain_annealing_and_untrained_network():
    """What the trained network adds: on a held-out power-law graph, a short
    anneal followed by rounds of (network warm start + 10 greedy sweeps)
    reaches a higher cut than a plain anneal that takes longer, and than the
    same procedure with the untrained network. The final cut is checked
    against the oracle's cut of the returned spins."""
    import torch
    rng = np.random.default_rng(21)
    train = []
    for k in range(16):
        n = int(rng.integers(2000, 10000))
        s = int(rng.integers(1 << 30))
        train.append(synth.zipf_config_graph(n, 2.1, 4, n // 4, s) if k % 2 == 0
                     else synth.er_graph(n, 10.0 / (n - 1), s, weights="int8"))
    test = synth.zipf_config_graph(30000, 2.1, 4, 3000, 777)
    params = synth.gnn_init_params(2)

    def learned_cut(net, h, seed):
        P.ising_init_random(h, seed)
        P.ising_anneal(h, p0=0.1, t_total=50, seed=seed)
        for r in range(4):
            P.ising_gnn_warm_start(net, h, set_bias=False)
            P.ising_anneal(h, p0=0.0, t_total=10, seed=1 + r)
        return P.ising_cut(h)

    with P.ising_gnn_create(params) as net, P.ising_gnn_create(params) as untrained:
        ex = []
        for k, g in enumerate(train):
            h = P.ising_create(g.n, g.src, g.dst, g.w)
            P.ising_init_random(h, k)
            P.ising_anneal(h, p0=0.1, t_total=100, seed=k)
            snap = torch.empty(g.n, dtype=torch.int8, device="cuda")
            P.ising_get_spins(h, snap)
            P.ising_anneal(h, p0=0.01, t_total=200, seed=500 + k)
            lab = torch.empty(g.n, dtype=torch.int8, device="cuda")
            P.ising_get_spins(h, lab)
            ex.append((h, snap, lab))
        for it in range(1500):
            h, snap, lab = ex[it % len(ex)]
            P.ising_set_spins(h, snap)
            P.ising_gnn_train_step(net, h, lab, lr=2e-3)
        for h, _, _ in ex:
            h.close()
        with P.ising_create(test.n, test.src, test.dst, test.w) as h:
            trained = [learned_cut(net, h, 40 + k) for k in range(3)]
            final = P.ising_get_spins(h)
            base = [learned_cut(untrained, h, 40 + k) for k in range(3)]
            plain = []
            for k in range(3):
                P.ising_init_random(h, 40 + k)
                P.ising_anneal(h, p0=0.1, t_total=400, seed=40 + k)
                plain.append(P.ising_cut(h))
    assert trained[-1] == oracle.energy_cut(test.n, test.src, test.dst, test.w, final)[2]
    # 50 + 4 x 10 sweeps and four forward passes against a 400-sweep anneal
    assert np.mean(trained) > np.mean(plain)
    assert np.mean(trained) > np.mean(base)
