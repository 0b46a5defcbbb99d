"""The seeded input generators: the shapes the workloads claim, reproducibility,
and that the faster unique step gives numpy's result. No GPU."""

import numpy as np

import synth
from synth import graphs


def test_sorted_unique_equals_numpy_unique():
    rng = np.random.default_rng(3)
    for size, hi in ((0, 10), (1, 10), (1000, 50), (200_000, 10**12)):
        a = rng.integers(0, hi, size=size, dtype=np.int64)
        assert np.array_equal(graphs._sorted_unique(a), np.unique(a))


def test_generators_are_pure_functions_of_their_seed():
    a = synth.zipf_config_graph(5000, 2.1, 4, 1000, 9)
    b = synth.zipf_config_graph(5000, 2.1, 4, 1000, 9)
    c = synth.zipf_config_graph(5000, 2.1, 4, 1000, 10)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst) and np.array_equal(a.w, b.w)
    assert not (a.src.size == c.src.size and np.array_equal(a.src, c.src))
    e = synth.er_graph(3000, 10.0 / 2999, 4, weights="int8")
    f = synth.er_graph(3000, 10.0 / 2999, 4, weights="int8")
    assert np.array_equal(e.src, f.src) and np.array_equal(e.w, f.w)


def test_generated_graphs_have_the_stated_shape():
    # erased configuration model: no self-loops, no repeated pair, src < dst
    g = synth.zipf_config_graph(20000, 2.1, 4, 3000, 5)
    assert np.all(g.src < g.dst)
    key = g.src.astype(np.int64) * g.n + g.dst
    assert np.unique(key).size == key.size
    assert set(np.unique(g.w).tolist()) <= set(range(-8, 9)) - {0}
    deg = np.bincount(np.concatenate([g.src, g.dst]), minlength=g.n)
    assert deg.max() > 256 and np.median(deg) < 16          # hubs and a light bulk
    # G(n, p): mean degree near p (n - 1)
    e = synth.er_graph(20000, 10.0 / 19999, 6, weights="pm1")
    assert abs(2 * e.m / e.n - 10.0) < 0.3
    assert set(np.unique(e.w).tolist()) == {-1, 1}


def test_warmstart_specs_build_the_workload_graphs():
    train, test, spec = synth.warmstart_specs(train_count=6, test_count=1)
    tr, te, spec2 = synth.warmstart_workload(train_count=6, test_count=1)
    assert spec == spec2
    for t, g in zip(train + test, tr + te):
        h = synth.graph_from_spec(t)
        assert h.n == g.n and np.array_equal(h.src, g.src) and np.array_equal(h.w, g.w)
    kinds = [t[0] for t in train]
    assert kinds == ["zipf", "er"] * 3
    big, _, bspec = synth.warmstart_specs(synth.WARMSTART_BATCHED, train_count=400)
    ns = np.array([t[1] for t in big])
    assert bspec["nmin"] == 1000 and bspec["nmax"] == 100000
    assert ns.min() >= 1000 and ns.max() <= 100000 and ns.max() > 50000
