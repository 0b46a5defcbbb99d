"""Host logic of the halo engine, without a device: the recursive
breadth-first bisection and the plan (ising_plan_halo).

The partition must be balanced (every part n / P or n / P + 1 vertices),
deterministic and compact on a lattice; the plan's largest work ratio is
recomputed here from the partition and the colouring by breadth-first layers
(phase j of an epoch of D = S * K phases updates the class-(j - 1) mod K
vertices at most D - j hops from the part)."""

import numpy as np
import pytest
import scipy.sparse as sp

import synth


@pytest.fixture(scope="module")
def P():
    from paper_1807_10750_gb300 import _build
    _build.build()
    import paper_1807_10750_gb300 as P
    return P


def _adjacency(g):
    a = sp.coo_matrix((np.ones(g.src.size), (g.src, g.dst)), shape=(g.n, g.n)).tocsr()
    return ((a + a.T) > 0).astype(np.int8).tocsr()


def _work_ratio(g, part, colour, parts, S):
    """Largest rows-updated-per-sweep / rows-owned over the parts."""
    A = _adjacency(g)
    K = int(colour.max()) + 1
    D = S * K
    worst = 0.0
    for p in range(parts):
        hops = np.full(g.n, -1, np.int64)
        front = part == p
        hops[front] = 0
        for h in range(1, D + 1):
            reach = (A @ front.astype(np.int8)) > 0
            front = reach & (hops < 0)
            hops[front] = h
        rows = 0
        for j in range(1, D + 1):
            c = (j - 1) % K
            rows += int(np.count_nonzero((colour == c) & (hops >= 0) & (hops <= D - j)))
        worst = max(worst, rows / (S * np.count_nonzero(part == p)))
    return worst


def test_torus_partition_balanced_compact_and_deterministic(P):
    g = synth.torus_graph(128, 1, weights="pm1")
    part, plan = P.ising_plan_halo(g.n, g.src, g.dst, g.w, 16, 2)
    assert plan is not None
    sizes = np.bincount(part, minlength=16)
    assert sizes.min() >= g.n // 16 and sizes.max() <= g.n // 16 + 1
    cut = np.count_nonzero(part[g.src] != part[g.dst])
    # 16 compact parts of 1024 vertices cut a few percent of the 32768 edges;
    # a random assignment would cut 94 %
    assert cut < 0.06 * g.src.size, cut
    again, _ = P.ising_plan_halo(g.n, g.src, g.dst, g.w, 16, 2)
    assert np.array_equal(part, again)


@pytest.mark.parametrize("S", [1, 2, 3])
@pytest.mark.parametrize("name", ["torus", "torus_odd", "two_tori"])
def test_plan_work_ratio_matches_breadth_first_recount(P, name, S):
    g = {"torus": lambda: synth.torus_graph(48, 3, weights="pm1"),
         "torus_odd": lambda: synth.torus_graph(41, 2, weights="int8", Ly=29),
         "two_tori": lambda: _two_tori()}[name]()
    parts = 12
    K, colour = P.ising_plan_colouring(g.n, g.src, g.dst, g.w)
    part, plan = P.ising_plan_halo(g.n, g.src, g.dst, g.w, parts, S)
    if S * K > 16:
        assert plan is None
        return
    assert plan is not None
    sizes = np.bincount(part, minlength=parts)
    assert sizes.min() >= g.n // parts and sizes.max() <= g.n // parts + 1
    want = _work_ratio(g, part, colour, parts, S)
    assert plan["work_ratio"] == pytest.approx(want, rel=1e-12)
    assert 0 < plan["smem_bytes"] <= 225 * 1024


def _two_tori():
    a = synth.torus_graph(30, 5, weights="int8")
    b = synth.torus_graph(20, 6, weights="pm1", Ly=17)
    return synth.Graph(a.n + b.n, np.concatenate([a.src, b.src + a.n]).astype(np.int32),
                       np.concatenate([a.dst, b.dst + a.n]).astype(np.int32),
                       np.concatenate([a.w, b.w]).astype(np.int32))


def test_graphs_the_engine_does_not_take(P):
    k6 = synth.complete_graph(6, 1, weights="pm1")           # 6 colours
    part, plan = P.ising_plan_halo(k6.n, k6.src, k6.dst, k6.w, 2, 1)
    assert plan is None and sorted(np.bincount(part)) == [3, 3]
    n = 200                                                  # a row of 199 entries
    star = synth.Graph(n, np.zeros(n - 1, np.int32), np.arange(1, n, dtype=np.int32),
                       np.ones(n - 1, np.int32))
    assert P.ising_plan_halo(star.n, star.src, star.dst, star.w, 4, 1)[1] is None
    big = synth.torus_graph(8, 1, weights="pm1")
    big.w = (big.w * 300).astype(np.int32)                   # beyond int8
    assert P.ising_plan_halo(big.n, big.src, big.dst, big.w, 4, 1)[1] is None
    small = synth.torus_graph(4, 1)
    assert P.ising_plan_halo(small.n, small.src, small.dst, small.w, 17, 1)[1] is None  # empty parts


def test_plan_argument_errors(P):
    g = synth.torus_graph(8, 1)
    for parts, S in ((0, 1), (4, 0), (4, 17)):
        with pytest.raises(P.IsingError) as e:
            P.ising_plan_halo(g.n, g.src, g.dst, g.w, parts, S)
        assert e.value.code == P.ISING_EINVAL
    with pytest.raises(P.IsingError) as e:   # a self-loop, as in ising_create
        P.ising_plan_halo(3, np.array([0, 1]), np.array([0, 2]), np.array([1, 1]), 2, 1)
    assert e.value.code == P.ISING_EINVAL
