"""Seeded generators for undirected weighted graphs.

Every generator returns a :class:`Graph`: ``n`` vertices and an undirected edge
list ``(src, dst, w)`` of int32 arrays, each edge listed once with
``src != dst``. The generators only draw random structure; merging duplicate
edges, colouring and everything else the annealer does is left to its callers.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Graph:
    n: int
    src: np.ndarray
    dst: np.ndarray
    w: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def arrays(self):
        return (np.ascontiguousarray(self.src, dtype=np.int32),
                np.ascontiguousarray(self.dst, dtype=np.int32),
                np.ascontiguousarray(self.w, dtype=np.int32))


def draw_weights(kind: str, m: int, rng: np.random.Generator) -> np.ndarray:
    """Edge weights: ``one`` (all +1), ``pm1`` (uniform {-1,+1}) or ``int8``
    (uniform over [-8, 8] without 0, the integer range of the paper's large
    irregular workloads as restated for this build)."""
    if kind == "one":
        return np.ones(m, dtype=np.int32)
    if kind == "pm1":
        return (rng.integers(0, 2, size=m, dtype=np.int32) * 2 - 1).astype(np.int32)
    if kind == "int8":
        mag = rng.integers(1, 9, size=m, dtype=np.int32)
        sgn = rng.integers(0, 2, size=m, dtype=np.int32) * 2 - 1
        return (mag * sgn).astype(np.int32)
    raise ValueError(f"unknown weight kind {kind!r}")


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    """np.unique(a) for an integer array, by sorting (the same result; much
    faster than the hash-based path of recent numpy on large arrays)."""
    a = np.sort(a, kind="stable")
    if a.size == 0:
        return a
    keep = np.empty(a.size, dtype=bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def _pairs_from_index(k: np.ndarray):
    """Map a linear index over {(i, j): 0 <= i < j} (ordered by j, then i) to
    the pair (i, j)."""
    k = k.astype(np.int64)
    j = np.floor((1.0 + np.sqrt(1.0 + 8.0 * k.astype(np.float64))) / 2.0).astype(np.int64)
    # fix floating point rounding at the boundaries
    j = np.where(j * (j - 1) // 2 > k, j - 1, j)
    j = np.where((j + 1) * j // 2 <= k, j + 1, j)
    i = k - j * (j - 1) // 2
    return i, j


def er_graph(n: int, p: float, seed: int, weights: str = "one") -> Graph:
    """Erdos-Renyi G(n, p): every unordered pair is an edge independently with
    probability p."""
    rng = np.random.default_rng(seed)
    npairs = n * (n - 1) // 2
    if npairs <= 4_000_000:
        keep = rng.random(npairs) < p
        idx = np.nonzero(keep)[0]
    else:
        # Same law as above without materialising all pairs: draw the edge
        # count, then that many distinct pair indices uniformly.
        m = int(rng.binomial(npairs, p))
        idx = _sorted_unique(rng.integers(0, npairs, size=m, dtype=np.int64))
        while idx.size < m:
            more = rng.integers(0, npairs, size=m - idx.size, dtype=np.int64)
            idx = _sorted_unique(np.concatenate([idx, more]))
        idx = idx[:m]
    i, j = _pairs_from_index(idx)
    w = draw_weights(weights, idx.size, rng)
    return Graph(n, i.astype(np.int32), j.astype(np.int32), w,
                 meta={"kind": "er", "p": p, "seed": seed, "weights": weights})


def torus_graph(L: int, seed: int, weights: str = "pm1", Ly: int | None = None) -> Graph:
    """2-D toroidal grid L x Ly with row-major vertex ids ``y * L + x`` and the
    four nearest neighbours (wrap-around in both directions)."""
    Ly = L if Ly is None else Ly
    if L < 3 or Ly < 3:
        raise ValueError("torus sides must be >= 3 so that no edge repeats")
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(Ly, dtype=np.int64), np.arange(L, dtype=np.int64), indexing="ij")
    v = (y * L + x).ravel()
    right = (y * L + (x + 1) % L).ravel()
    down = (((y + 1) % Ly) * L + x).ravel()
    src = np.concatenate([v, v])
    dst = np.concatenate([right, down])
    w = draw_weights(weights, src.size, rng)
    return Graph(L * Ly, src.astype(np.int32), dst.astype(np.int32), w,
                 meta={"kind": "torus", "L": L, "Ly": Ly, "seed": seed, "weights": weights})


def grid_graph(Lx: int, Ly: int, seed: int = 0, weights: str = "one") -> Graph:
    """Open 2-D grid (no wrap-around), row-major ids."""
    rng = np.random.default_rng(seed)
    src, dst = [], []
    for y in range(Ly):
        for x in range(Lx):
            v = y * Lx + x
            if x + 1 < Lx:
                src.append(v); dst.append(v + 1)
            if y + 1 < Ly:
                src.append(v); dst.append(v + Lx)
    src = np.array(src, dtype=np.int32)
    dst = np.array(dst, dtype=np.int32)
    return Graph(Lx * Ly, src, dst, draw_weights(weights, src.size, rng),
                 meta={"kind": "grid", "Lx": Lx, "Ly": Ly})


def complete_graph(n: int, seed: int = 0, weights: str = "one") -> Graph:
    rng = np.random.default_rng(seed)
    i, j = np.triu_indices(n, k=1)
    return Graph(n, i.astype(np.int32), j.astype(np.int32), draw_weights(weights, i.size, rng),
                 meta={"kind": "complete"})


def cycle_graph(n: int, seed: int = 0, weights: str = "one") -> Graph:
    rng = np.random.default_rng(seed)
    src = np.arange(n, dtype=np.int32)
    dst = ((src + 1) % n).astype(np.int32)
    return Graph(n, src, dst, draw_weights(weights, n, rng), meta={"kind": "cycle"})


def random_small_graph(n: int, p: float, seed: int, weights: str = "int8",
                       duplicates: int = 0) -> Graph:
    """A small G(n, p) graph, optionally with ``duplicates`` extra copies of
    random existing edges listed again (in either orientation) so that callers
    exercise duplicate merging."""
    g = er_graph(n, p, seed, weights)
    if duplicates and g.m:
        rng = np.random.default_rng(seed + 7919)
        pick = rng.integers(0, g.m, size=duplicates)
        flip = rng.integers(0, 2, size=duplicates).astype(bool)
        s = np.where(flip, g.dst[pick], g.src[pick])
        d = np.where(flip, g.src[pick], g.dst[pick])
        w = draw_weights(weights, duplicates, rng)
        g = Graph(g.n, np.concatenate([g.src, s]).astype(np.int32),
                  np.concatenate([g.dst, d]).astype(np.int32),
                  np.concatenate([g.w, w]).astype(np.int32), meta=dict(g.meta, duplicates=duplicates))
    return g


def _powerlaw_degrees(n: int, alpha: float, dmin: int, dmax: int, rng) -> np.ndarray:
    k = np.arange(dmin, dmax + 1, dtype=np.float64)
    pk = k ** (-alpha)
    cdf = np.cumsum(pk)
    cdf /= cdf[-1]
    u = rng.random(n)
    return (np.searchsorted(cdf, u, side="right") + dmin).astype(np.int64)


def zipf_config_graph(n: int, alpha: float, dmin: int, dmax: int, seed: int,
                      weights: str = "int8") -> Graph:
    """Erased configuration model: i.i.d. degrees from a discrete power law
    P(d) ~ d^-alpha on [dmin, dmax], stubs paired by a seeded shuffle, then
    self-loops and repeated pairs removed."""
    rng = np.random.default_rng(seed)
    deg = _powerlaw_degrees(n, alpha, dmin, dmax, rng)
    stubs = np.repeat(np.arange(n, dtype=np.int64), deg)
    if stubs.size % 2:
        stubs = stubs[:-1]
    rng.shuffle(stubs)
    a, b = stubs[0::2], stubs[1::2]
    keep = a != b
    a, b = a[keep], b[keep]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key = _sorted_unique(lo * n + hi)
    src = (key // n).astype(np.int32)
    dst = (key % n).astype(np.int32)
    w = draw_weights(weights, src.size, rng)
    return Graph(n, src, dst, w, meta={"kind": "zipf", "alpha": alpha, "dmin": dmin,
                                       "dmax": dmax, "seed": seed, "weights": weights,
                                       "max_degree_drawn": int(deg.max())})


def batched_er_graphs(count: int, nmin: int, nmax: int, avg_degree: float, seed: int,
                      weights: str = "pm1") -> list[Graph]:
    """``count`` Erdos-Renyi graphs with vertex counts log-uniform in
    [nmin, nmax] and p = avg_degree / (n - 1)."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=count))
    ns = np.clip(np.rint(ns).astype(np.int64), nmin, nmax)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [er_graph(int(n), min(1.0, avg_degree / (n - 1)), int(s), weights) for n, s in zip(ns, seeds)]


# Named workloads with the shapes the benchmark and the parity tests use.
WORKLOADS = {
    # G(800, 0.06), unit weights: the shape of the G-set row G9 (800 vertices,
    # ~19k edges). 1000 sweeps, flip probability linear 0.1 -> 0.
    "er800": dict(gen="er", n=800, p=0.06, weights="one", gen_seed=1,
                  p0=0.1, sweeps=1000, seed=1),
    # 1024 x 1024 torus, +-1 weights: the torus rows of Table III scaled up.
    "torus1024": dict(gen="torus", L=1024, weights="pm1", gen_seed=2,
                      p0=0.1, sweeps=2000, seed=1),
    # 2^20-vertex erased configuration model, power-law degrees (alpha 2.1,
    # max degree 10k), weights in [-8, 8] \ {0}: the large irregular C rows.
    "zipf1m": dict(gen="zipf", n=1 << 20, alpha=2.1, dmin=4, dmax=10000, weights="int8",
                   gen_seed=3, p0=0.1, sweeps=2000, seed=1),
}


# The batched workload: 1024 Erdos-Renyi instances, n log-uniform in
# [500, 20000], mean degree 10, +-1 weights; 8 replicas each, 1000 sweeps.
BATCHED = dict(count=1024, nmin=500, nmax=20000, avg_degree=10.0, gen_seed=4, weights="pm1",
               replicas=8, p0=0.1, sweeps=1000, seed=1)


def batched_workload(**override) -> tuple[list[Graph], dict]:
    spec = dict(BATCHED)
    spec.update(override)
    gs = batched_er_graphs(spec["count"], spec["nmin"], spec["nmax"], spec["avg_degree"],
                           spec["gen_seed"], spec["weights"])
    return gs, {k: spec[k] for k in ("replicas", "p0", "sweeps", "seed")}


def workload(name: str, **override) -> tuple[Graph, dict]:
    """Build a named workload's graph; returns (graph, schedule parameters)."""
    spec = dict(WORKLOADS[name])
    spec.update(override)
    gen = spec["gen"]
    if gen == "er":
        g = er_graph(spec["n"], spec["p"], spec["gen_seed"], spec["weights"])
    elif gen == "torus":
        g = torus_graph(spec["L"], spec["gen_seed"], spec["weights"])
    elif gen == "zipf":
        g = zipf_config_graph(spec["n"], spec["alpha"], spec["dmin"], spec["dmax"],
                              spec["gen_seed"], spec["weights"])
    else:
        raise ValueError(gen)
    sched = {k: spec[k] for k in ("p0", "sweeps", "seed")}
    return g, sched


# The learned warm-start workload: training graphs (Erdos-Renyi with mean
# degree 10 and power-law graphs, alternating; n log-uniform in
# [nmin, nmax]; weights uniform in [-8, 8] without 0) and held-out
# 100k-vertex power-law test graphs. WARMSTART is the small form the tests
# and the single-graph measurements use; WARMSTART_BATCHED the batched form
# (training graphs of 1k-100k vertices).
WARMSTART = dict(train_count=64, nmin=1000, nmax=30000, gen_seed=5, test_count=2, test_n=100000,
                 test_seed=4242, alpha=2.1, dmin=4, dmax=10000)
WARMSTART_BATCHED = dict(WARMSTART, train_count=2048, nmax=100000, test_count=152)


def warmstart_specs(base=None, **override):
    """(train, test, spec): graph specs (kind, n, seed, alpha, dmin, dmax) in
    the order `warmstart_workload` generates them; `graph_from_spec` builds
    one (so that a process pool can build them)."""
    spec = dict(WARMSTART if base is None else base)
    spec.update(override)
    rng = np.random.default_rng(spec["gen_seed"])
    train = []
    for k in range(spec["train_count"]):
        n = int(np.clip(np.rint(np.exp(rng.uniform(math.log(spec["nmin"]), math.log(spec["nmax"])))),
                        spec["nmin"], spec["nmax"]))
        s = int(rng.integers(0, 2 ** 31 - 1))
        if k % 2 == 0:
            train.append(("zipf", n, s, spec["alpha"], spec["dmin"], min(spec["dmax"], n // 4)))
        else:
            train.append(("er", n, s, 0.0, 0, 0))
    test = [("zipf", spec["test_n"], spec["test_seed"] + k, spec["alpha"], spec["dmin"], spec["dmax"])
            for k in range(spec["test_count"])]
    return train, test, spec


def graph_from_spec(t) -> Graph:
    kind, n, s, alpha, dmin, dmax = t
    if kind == "zipf":
        return zipf_config_graph(n, alpha, dmin, dmax, s, weights="int8")
    return er_graph(n, min(1.0, 10.0 / (n - 1)), s, weights="int8")


def warmstart_workload(**override):
    train, test, spec = warmstart_specs(**override)
    return [graph_from_spec(t) for t in train], [graph_from_spec(t) for t in test], spec
