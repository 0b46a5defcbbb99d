"""Pins for the CPU oracle: each test checks it against something other than
itself -- published known answers, closed forms, brute force over all spin
states, invariants of the zero-temperature dynamics and known max-cut optima.

None of these tests touches a GPU.
"""

import itertools
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# independent helpers (direct definitions, written from the edge list as given,
# duplicates and zero weights included)
# ---------------------------------------------------------------------------
def direct_cut(g, s):
    """Eq. 4 written out: total weight of the listed edges whose ends differ."""
    s = np.asarray(s, dtype=np.int64)
    return int(np.sum(g.w.astype(np.int64) * (s[g.src] != s[g.dst])))


def direct_energy(g, s):
    s = np.asarray(s, dtype=np.int64)
    return int(np.sum(g.w.astype(np.int64) * s[g.src] * s[g.dst]))


def all_states(n):
    bits = (np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1
    return (1 - 2 * bits).astype(np.int8)


def brute_force_max_cut(g):
    S = all_states(g.n).astype(np.int64)
    cuts = ((S[:, g.src] != S[:, g.dst]) * g.w.astype(np.int64)[None, :]).sum(axis=1)
    return int(cuts.max())


def field(g, s):
    """f_i = sum over listed edges touching i of w * s_other."""
    s = np.asarray(s, dtype=np.int64)
    f = np.zeros(g.n, dtype=np.int64)
    np.add.at(f, g.src, g.w.astype(np.int64) * s[g.dst])
    np.add.at(f, g.dst, g.w.astype(np.int64) * s[g.src])
    return f


# ---------------------------------------------------------------------------
# Philox4x32-10
# ---------------------------------------------------------------------------
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_philox_word_uniformity():
    # 2^16 words of the annealer's counter layout: mean and byte histogram.
    xs = np.array([oracle.random_word(12345, 0, i, 7, 0, 0) for i in range(1 << 16)],
                  dtype=np.uint64)
    u = xs.astype(np.float64) / 2.0 ** 32
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)
    counts = np.bincount((xs & 0xFF).astype(np.int64), minlength=256)
    exp = u.size / 256
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 255 + 6 * math.sqrt(2 * 255)
    # top bit (used for initial spins) is balanced
    top = (xs >> 31).astype(np.int64)
    assert abs(top.mean() - 0.5) < 5 * math.sqrt(0.25 / top.size)


def test_random_word_key_layout():
    # seed occupies the key (lo, hi); instance is folded into the high key word.
    seed = (0x01234567 << 32) | 0x89ABCDEF
    a = oracle.random_word(seed, 0, 1, 2, 3, 4)
    b = int(oracle.philox([1, 2, 3, 4], [0x89ABCDEF, 0x01234567])[0])
    assert a == b
    c = oracle.random_word(seed, 5, 1, 2, 3, 4)
    d = int(oracle.philox([1, 2, 3, 4], [0x89ABCDEF, 0x01234567 ^ ((5 * 0x9E3779B9) & 0xFFFFFFFF)])[0])
    assert c == d


# ---------------------------------------------------------------------------
# schedule
# ---------------------------------------------------------------------------
def test_threshold_closed_forms():
    assert [oracle.threshold(0.5, 3, t) for t in range(3)] == [2 ** 31, 2 ** 30, 0]
    assert [oracle.threshold(0.25, 5, t) for t in range(5)] == [2 ** 30, 3 * 2 ** 28, 2 ** 29, 2 ** 28, 0]
    assert all(oracle.threshold(0.0, 100, t) == 0 for t in range(100))
    assert oracle.threshold(1.0, 10, 0) == 2 ** 32 - 1
    assert oracle.threshold(0.9, 1, 0) == 0
    assert oracle.threshold(0.1, 1000, 0) == round(0.1 * 2 ** 32)


@pytest.mark.parametrize("p0,T", [(0.1, 1000), (0.37, 17), (1.0, 2), (0.003, 2000)])
def test_threshold_monotone_and_ends(p0, T):
    thr = [oracle.threshold(p0, T, t) for t in range(T)]
    assert thr[-1] == 0
    assert thr[0] == min(2 ** 32 - 1, math.floor(p0 * 2 ** 32 + 0.5))
    assert all(a >= b for a, b in zip(thr, thr[1:]))
    # linear: thr[t] within 1 of thr[0] * (T-1-t)/(T-1)
    for t in range(0, T, max(1, T // 50)):
        assert abs(thr[t] - thr[0] * (T - 1 - t) / (T - 1)) <= 1.0


# ---------------------------------------------------------------------------
# energy and cut
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(6))
def test_energy_cut_brute_force(seed):
    g = synth.random_small_graph(9, 0.5, seed, weights="int8", duplicates=6)
    for s in all_states(g.n)[:: 3]:
        H, W, cut = oracle.energy_cut(g.n, g.src, g.dst, g.w, s)
        assert H == direct_energy(g, s)
        assert W == int(g.w.sum())
        assert cut == direct_cut(g, s)
        # sign symmetry: s and -s cut the same edges
        assert oracle.energy_cut(g.n, g.src, g.dst, g.w, -s)[2] == cut


def test_duplicates_merge_and_zero_weight_edges_vanish():
    src = np.array([0, 1, 1, 2, 0], dtype=np.int32)
    dst = np.array([1, 0, 2, 1, 2], dtype=np.int32)
    w = np.array([2, 3, 4, -4, 1], dtype=np.int32)
    # (0,1) merges to 5, (1,2) merges to 0 (no edge), (0,2) weight 1
    assert oracle.num_edges(3, src, dst, w) == 2
    C, col = oracle.colouring(3, src, dst, w)
    # 1 and 2 are no longer adjacent: Welsh-Powell gives 0 (deg 2) colour 0,
    # then 1 and 2 (deg 1 each) both colour 1.
    assert C == 2 and list(col) == [0, 1, 1]
    s = np.array([1, -1, -1], dtype=np.int8)
    H, W, cut = oracle.energy_cut(3, src, dst, w, s)
    assert (H, W, cut) == (-6, 6, 6)


@pytest.mark.parametrize("bad", [
    dict(n=3, src=[0], dst=[0], w=[1]),      # self-loop
    dict(n=3, src=[0], dst=[3], w=[1]),      # out of range
    dict(n=3, src=[-1], dst=[1], w=[1]),     # negative id
    dict(n=0, src=[], dst=[], w=[]),         # empty vertex set
])
def test_invalid_graphs_rejected(bad):
    with pytest.raises(ValueError):
        oracle.num_edges(bad["n"], bad["src"], bad["dst"], bad["w"])


# ---------------------------------------------------------------------------
# colouring
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(5))
def test_colouring_is_proper(seed):
    g = synth.random_small_graph(60, 0.2, seed, duplicates=10)
    C, col = oracle.colouring(g.n, g.src, g.dst, g.w)
    assert col.min() == 0 and col.max() == C - 1
    merged_nonzero = {}
    for u, v, w in zip(g.src, g.dst, g.w):
        k = (min(u, v), max(u, v))
        merged_nonzero[k] = merged_nonzero.get(k, 0) + int(w)
    for (u, v), w in merged_nonzero.items():
        if w != 0:
            assert col[u] != col[v]
    # first fit: a vertex of colour c has neighbours of every colour below c
    adj = [set() for _ in range(g.n)]
    for (u, v), w in merged_nonzero.items():
        if w != 0:
            adj[u].add(v); adj[v].add(u)
    for v in range(g.n):
        assert set(range(col[v])) <= {col[u] for u in adj[v]}


def test_colouring_torus_is_checkerboard():
    g = synth.torus_graph(8, 0, weights="pm1")
    C, col = oracle.colouring(g.n, g.src, g.dst, g.w)
    y, x = np.divmod(np.arange(g.n), 8)
    assert C == 2 and np.array_equal(col, (x + y) % 2)


def test_colouring_special_graphs():
    g = synth.complete_graph(7)
    assert oracle.colouring(g.n, g.src, g.dst, g.w)[0] == 7
    g = synth.cycle_graph(10)
    assert oracle.colouring(g.n, g.src, g.dst, g.w)[0] == 2
    # path 0-1-2: the degree-2 middle vertex is coloured first
    C, col = oracle.colouring(3, np.array([0, 1]), np.array([1, 2]), np.array([1, 1]))
    assert list(col) == [1, 0, 1]
    # star: hub 5 coloured 0, leaves 1
    C, col = oracle.colouring(6, np.array([5] * 5), np.arange(5), np.ones(5))
    assert C == 2 and col[5] == 0 and set(col[:5]) == {1}


def _double_star(leaves):
    """Centres 0 and 1 joined to each other, each with `leaves` leaves of its
    own: both centres have degree leaves + 1."""
    src = [0]
    dst = [1]
    nxt = 2
    for c in (0, 1):
        for _ in range(leaves):
            src.append(c)
            dst.append(nxt)
            nxt += 1
    a = lambda x: np.array(x, dtype=np.int32)
    return nxt, a(src), a(dst), a([1] * len(src))


def test_colouring_hub_tier_threshold_is_256_neighbours():
    # R6: a vertex with at least 256 distinct neighbours is a hub; hubs take
    # the low colours among themselves, every other vertex starts above them.
    # Centres of degree 256: hubs 0 and 1 get colours 0 and 1, and every leaf
    # gets colour 2 (plain Welsh-Powell would give the leaves of centre 0
    # colour 1 and those of centre 1 colour 0).
    n, src, dst, w = _double_star(255)
    C, col = oracle.colouring(n, src, dst, w)
    assert C == 3 and col[0] == 0 and col[1] == 1 and set(col[2:]) == {2}
    # Centres of degree 255 are not hubs: plain Welsh-Powell.
    n, src, dst, w = _double_star(254)
    C, col = oracle.colouring(n, src, dst, w)
    assert C == 2 and col[0] == 0 and col[1] == 1
    assert set(col[2:2 + 254]) == {1} and set(col[2 + 254:]) == {0}


def test_colouring_hub_degree_counts_merged_neighbours():
    # 300 edges from vertex 0, but 100 of them repeat a pair and 20 of those
    # cancel to weight 0: vertex 0 has 200 - 20 = 180 distinct neighbours, so
    # it is no hub. Plain Welsh-Powell then gives the 20 vertices left
    # isolated colour 0 (a hub 0 would push them to colour 1).
    src = np.zeros(300, np.int32)
    dst = np.concatenate([np.arange(1, 201), np.arange(1, 101)]).astype(np.int32)
    w = np.ones(300, np.int32)
    w[200:220] = -1
    C, col = oracle.colouring(201, src, dst, w)
    assert C == 2 and col[0] == 0
    assert set(col[1:21]) == {0} and set(col[21:]) == {1}


def _merged_adjacency(g):
    merged = {}
    for u, v, w in zip(g.src, g.dst, g.w):
        k = (min(u, v), max(u, v))
        merged[k] = merged.get(k, 0) + int(w)
    adj = [set() for _ in range(g.n)]
    for (u, v), w in merged.items():
        if w != 0:
            adj[u].add(v); adj[v].add(u)
    return adj


@pytest.mark.parametrize("seed", range(3))
def test_colouring_two_tiers_on_a_graph_with_hubs(seed):
    # A power-law graph whose largest degrees exceed 256: the colouring is
    # proper; hub colours are all below non-hub colours; within each tier it
    # is first fit (a vertex of colour c has, among its own tier's
    # neighbours, every colour of its tier below c); hubs are coloured in
    # Welsh-Powell order, so class 0 holds the largest-degree vertex.
    g = synth.zipf_config_graph(6000, 2.0, 3, 1500, 40 + seed)
    adj = _merged_adjacency(g)
    deg = np.array([len(a) for a in adj])
    hub = deg >= 256
    assert 3 <= hub.sum() < g.n // 10
    C, col = oracle.colouring(g.n, g.src, g.dst, g.w)
    m = int(col[hub].max()) + 1
    assert col[~hub].min() == m and C == col.max() + 1
    for v in range(g.n):
        assert all(col[u] != col[v] for u in adj[v])
        same_tier = {col[u] for u in adj[v] if hub[u] == hub[v]}
        low = 0 if hub[v] else m
        assert set(range(low, col[v])) <= same_tier
    top = int(np.lexsort((np.arange(g.n), -deg))[0])
    assert col[top] == 0


def test_colouring_complete_graph_of_hubs():
    # K_300: every vertex has 299 neighbours, so all are hubs: 300 classes,
    # vertex i in class i (equal degrees, smaller id first).
    g = synth.complete_graph(300)
    C, col = oracle.colouring(g.n, g.src, g.dst, g.w)
    assert C == 300 and np.array_equal(col, np.arange(300))


# ---------------------------------------------------------------------------
# the annealing sweep
# ---------------------------------------------------------------------------
def test_init_spins_balanced_and_seeded():
    s = oracle.init_spins(100000, 9)
    assert set(np.unique(s)) == {-1, 1}
    assert abs(s.mean()) < 5 / math.sqrt(s.size)
    assert not np.array_equal(s, oracle.init_spins(100000, 10))
    assert not np.array_equal(s, oracle.init_spins(100000, 9, replica=1))
    assert np.array_equal(s, oracle.init_spins(100000, 9))


def test_edgeless_graph_tie_keeps_spin_and_flip_rate():
    # No edges: every field is 0, so Eq. 2 leaves the spin (R2) and only the
    # random flip acts. At p0 = 0 nothing changes; at sweep 0 of a 2-sweep
    # schedule the flip probability is exactly thr[0] / 2^32.
    n = 40000
    e = np.zeros(0, dtype=np.int32)
    s0 = oracle.init_spins(n, 3)
    s = oracle.anneal(n, e, e, e, s0, seed=4, p0=0.0, T=50)
    assert np.array_equal(s, s0)
    s = oracle.anneal(n, e, e, e, s0, seed=4, p0=0.3, T=2, sweeps=1)
    frac = float((s != s0).mean())
    p = oracle.threshold(0.3, 2, 0) / 2 ** 32
    assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / n)


def test_flip_follows_update_in_the_same_sweep():
    # p0 = 1 on a 2-sweep schedule: sweep 0 flips (almost surely) every spin
    # right after its update. Unit-weight even torus, all spins +1: colour 0
    # sees f = 4 -> -1, flipped -> +1; colour 1 then sees all +1 -> -1 ->
    # flipped -> +1. Every spin ends at +1, cut 0. (Flipping before the
    # update, or at the end of the sweep, gives a different state.)
    g = synth.torus_graph(6, 0, weights="one")
    s = oracle.anneal(g.n, g.src, g.dst, g.w, np.ones(g.n, np.int8), seed=11, p0=1.0, T=2, sweeps=1)
    assert np.all(s == 1)


@pytest.mark.parametrize("seed", range(4))
def test_zero_temperature_reaches_local_minimum_monotonically(seed):
    g = synth.random_small_graph(200, 0.05, seed, weights="int8", duplicates=20)
    s = oracle.init_spins(g.n, seed)
    prev_cut = direct_cut(g, s)
    for _ in range(200):
        s2 = oracle.anneal(g.n, g.src, g.dst, g.w, s, seed=seed, p0=0.0, T=1)
        cut = direct_cut(g, s2)
        assert cut >= prev_cut
        if np.array_equal(s2, s):
            break
        s, prev_cut = s2, cut
    else:
        pytest.fail("zero-temperature dynamics did not settle")
    f = field(g, s)
    # no single flip improves the cut: s_i f_i <= 0 everywhere
    assert np.all(s.astype(np.int64) * f <= 0)
    for i in range(0, g.n, 7):
        t = s.copy(); t[i] = -t[i]
        assert direct_cut(g, t) <= direct_cut(g, s)


def test_zero_temperature_fixed_points_known():
    # Checkerboard on a positive-weight even torus is the maximum cut (W) and
    # a fixed point of the T=0 dynamics.
    g = synth.torus_graph(8, 0, weights="one")
    y, x = np.divmod(np.arange(g.n), 8)
    s = np.where((x + y) % 2 == 0, 1, -1).astype(np.int8)
    s2 = oracle.anneal(g.n, g.src, g.dst, g.w, s, seed=1, p0=0.0, T=5)
    assert np.array_equal(s, s2)
    assert oracle.energy_cut(g.n, g.src, g.dst, g.w, s2)[2] == int(g.w.sum())
    # K_n, unit weights: a T=0 local minimum has sum(s) in {-1,0,1}, which is
    # the maximum cut floor(n/2) * ceil(n/2).
    for n in (7, 10):
        g = synth.complete_graph(n)
        s = oracle.anneal(g.n, g.src, g.dst, g.w, oracle.init_spins(n, n), seed=2, p0=0.0, T=20)
        assert oracle.energy_cut(g.n, g.src, g.dst, g.w, s)[2] == (n // 2) * ((n + 1) // 2)


@pytest.mark.parametrize("make,optimum", [
    (lambda: synth.torus_graph(12, 0, weights="one"), lambda g: int(g.w.sum())),
    (lambda: synth.grid_graph(9, 7, weights="one"), lambda g: int(g.w.sum())),
    (lambda: synth.cycle_graph(15), lambda g: g.n - 1),
    (lambda: synth.complete_graph(11), lambda g: 5 * 6),
])
def test_anneal_reaches_known_optimum(make, optimum):
    g = make()
    best = 0
    for seed in range(8):
        s = oracle.anneal(g.n, g.src, g.dst, g.w, oracle.init_spins(g.n, seed), seed=seed,
                          p0=0.1, T=400)
        cut = oracle.energy_cut(g.n, g.src, g.dst, g.w, s)[2]
        assert cut <= optimum(g)
        best = max(best, cut)
    assert best == optimum(g)


@pytest.mark.parametrize("seed", range(4))
def test_anneal_vs_brute_force_optimum(seed):
    g = synth.random_small_graph(12, 0.4, seed, weights="int8")
    opt = brute_force_max_cut(g)
    # every run stays at or below the optimum, and a fair share reaches it:
    # the four graphs' hit rates are about 0.39 to 0.98, so 60 runs give at
    # least 23 hits on average and fewer than 10 has probability ~1e-4
    hits = 0
    for r in range(60):
        s = oracle.anneal(g.n, g.src, g.dst, g.w, oracle.init_spins(g.n, 100 + r), seed=r,
                          p0=0.1, T=300)
        cut = direct_cut(g, s)
        assert cut <= opt
        hits += cut == opt
    assert hits >= 10


def test_split_anneal_equals_whole():
    g = synth.random_small_graph(300, 0.03, 5, weights="int8")
    s0 = oracle.init_spins(g.n, 5)
    whole = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=77, p0=0.2, T=60)
    part = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=77, p0=0.2, T=60, sweeps=23)
    part = oracle.anneal(g.n, g.src, g.dst, g.w, part, seed=77, p0=0.2, T=60, t_begin=23)
    assert np.array_equal(whole, part)


def test_anneal_rejects_bad_arguments():
    g = synth.cycle_graph(5)
    s = np.ones(5, np.int8)
    with pytest.raises(ValueError):
        oracle.anneal(g.n, g.src, g.dst, g.w, s, seed=1, p0=1.5, T=10)
    with pytest.raises(ValueError):
        oracle.anneal(g.n, g.src, g.dst, g.w, s, seed=1, p0=0.1, T=10, t_begin=5, sweeps=6)
    bad = s.copy(); bad[2] = 0
    with pytest.raises(ValueError):
        oracle.anneal(g.n, g.src, g.dst, g.w, bad, seed=1, p0=0.1, T=10)


def test_flip_needs_word_strictly_below_threshold():
    # Sec. IV-B: a thread flips if its random number is *below* F_p. Choose p0
    # so that thr[0] equals the word drawn for vertex 0 at sweep 0 exactly: that
    # vertex must not flip, while p0 one step higher flips it.
    seed = 31
    x = oracle.random_word(seed, 0, 0, 0, 0, 0)
    e = np.zeros(0, dtype=np.int32)
    s0 = np.ones(1, dtype=np.int8)
    p_eq = x / 2.0 ** 32
    assert oracle.threshold(p_eq, 2, 0) == x
    assert oracle.anneal(1, e, e, e, s0, seed=seed, p0=p_eq, T=2, sweeps=1)[0] == 1
    p_up = (x + 1) / 2.0 ** 32
    assert oracle.anneal(1, e, e, e, s0, seed=seed, p0=p_up, T=2, sweeps=1)[0] == -1


# ---------------------------------------------------------------------------
# Algorithm 1's N-flip schedule
# ---------------------------------------------------------------------------
def test_nflip_flips_exactly_n_distinct_spins_on_an_edgeless_graph():
    # No edges: Eq. 2 never changes a spin, so after sweep t exactly N_t spins
    # differ from before, N_t = floor(N0 (T-1-t) / (T-1)).
    n, T, N0 = 5000, 6, 1234
    e = np.zeros(0, dtype=np.int32)
    s = oracle.init_spins(n, 1)
    for t in range(T):
        s2 = oracle.anneal_nflip(n, e, e, e, s, seed=3, n0=N0, T=T, t_begin=t, sweeps=1)
        assert int((s2 != s).sum()) == N0 * (T - 1 - t) // (T - 1)
        s = s2


def _nflip_candidates(n, N, seed, t, replica, instance=0):
    """Reading R10 recomputed from the known-answer-pinned Philox: candidate j
    is floor(x_j * n / 2^32), x_j = word 0 of Philox4x32-10 at counter
    (j, t, replica, 2) under the key (lo32 seed, hi32 seed ^ instance *
    0x9E3779B9); the first N distinct candidates are chosen."""
    key = [seed & 0xFFFFFFFF, ((seed >> 32) ^ (instance * 0x9E3779B9)) & 0xFFFFFFFF]
    chosen, seen, j = [], set(), 0
    while len(chosen) < N:
        x = int(oracle.philox([j, t, replica, 2], key)[0])
        c = (x * n) >> 32
        if c not in seen:
            seen.add(c)
            chosen.append(c)
        j += 1
    return set(chosen), j


@pytest.mark.parametrize("n,N0,T,seed,t,replica", [
    (5000, 1234, 6, 3, 0, 0),
    (5000, 1234, 6, 3, 4, 0),
    (5000, 700, 9, 2 ** 33 + 5, 2, 3),   # high key word in use
    (64, 60, 2, 11, 0, 1),               # N close to n: many repeated candidates
    (50, 45, 3, 17, 1, 2),
])
def test_nflip_changes_exactly_the_first_distinct_candidates(n, N0, T, seed, t, replica):
    # On an edgeless graph Eq. 2 leaves every spin as it is, so the spins that
    # change in sweep t are exactly Algorithm 1's N_t random choices. They must
    # be the first N_t distinct values of floor(x_j n / 2^32) (R10). A map
    # x mod n, another output word, another stream or counter layout, or
    # taking N_t candidates without skipping repeats all give another set.
    e = np.zeros(0, dtype=np.int32)
    s = oracle.init_spins(n, 7, replica=replica)
    s2 = oracle.anneal_nflip(n, e, e, e, s, seed=seed, n0=N0, T=T, t_begin=t, sweeps=1,
                             replica=replica)
    Nt = N0 * (T - 1 - t) // (T - 1)
    want, draws = _nflip_candidates(n, Nt, seed, t, replica)
    assert set(np.nonzero(s2 != s)[0].tolist()) == want
    if n <= 64:
        assert draws > Nt  # repeats were skipped in this case


def test_nflip_candidate_map_takes_the_high_bits():
    # For n = 2^k, floor(x n / 2^32) is the top k bits of x: one vertex of
    # an edgeless 2^k-vertex graph flipped at N_t = 1 is x_0 >> (32 - k).
    e = np.zeros(0, dtype=np.int32)
    for k, seed in ((4, 1), (10, 2), (16, 3)):
        n = 1 << k
        s = np.ones(n, np.int8)
        s2 = oracle.anneal_nflip(n, e, e, e, s, seed=seed, n0=1, T=2, sweeps=1)
        x0 = int(oracle.philox([0, 0, 0, 2], [seed, 0])[0])
        assert np.nonzero(s2 != s)[0].tolist() == [x0 >> (32 - k)]


def test_nflip_all_spins_when_n0_equals_n():
    n = 300
    e = np.zeros(0, dtype=np.int32)
    s = oracle.init_spins(n, 2)
    s2 = oracle.anneal_nflip(n, e, e, e, s, seed=5, n0=n, T=2, sweeps=1)
    assert np.array_equal(s2, -s)


def test_nflip_choice_is_uniform():
    # over many sweeps every vertex is chosen about equally often
    n, T, N0 = 64, 401, 16
    e = np.zeros(0, dtype=np.int32)
    counts = np.zeros(n)
    s = np.ones(n, np.int8)
    for t in range(T - 1):
        s2 = oracle.anneal_nflip(n, e, e, e, s, seed=9, n0=N0, T=T, t_begin=t, sweeps=1)
        counts += (s2 != s)
        s = s2
    exp = counts.sum() / n
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < (n - 1) + 6 * math.sqrt(2 * (n - 1))


def test_nflip_zero_is_greedy_and_reaches_local_minimum():
    g = synth.random_small_graph(150, 0.05, 8, weights="int8")
    s = oracle.init_spins(g.n, 8)
    a = oracle.anneal_nflip(g.n, g.src, g.dst, g.w, s, seed=1, n0=0, T=30)
    b = oracle.anneal(g.n, g.src, g.dst, g.w, s, seed=1, p0=0.0, T=30)
    assert np.array_equal(a, b)
    assert np.all(a.astype(np.int64) * field(g, a) <= 0)


def test_nflip_reaches_known_optimum_and_rejects_bad_n0():
    g = synth.torus_graph(10, 0, weights="one")
    best = max(oracle.energy_cut(g.n, g.src, g.dst, g.w,
                                 oracle.anneal_nflip(g.n, g.src, g.dst, g.w, oracle.init_spins(g.n, k),
                                                     seed=k, n0=8, T=300))[2] for k in range(6))
    assert best == int(g.w.sum())
    with pytest.raises(ValueError):
        oracle.anneal_nflip(g.n, g.src, g.dst, g.w, np.ones(g.n, np.int8), seed=1, n0=g.n + 1, T=5)


# --- R11: per-vertex flip bias (project addition; q = 128 is Algorithm 2) ---

def test_bias_128_is_algorithm_2_and_zero_is_greedy():
    g = synth.random_small_graph(300, 0.05, 21, weights="int8")
    s0 = oracle.init_spins(g.n, 5)
    plain = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=9, p0=0.2, T=40)
    q128 = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=9, p0=0.2, T=40,
                         bias=np.full(g.n, 128, np.uint8))
    assert np.array_equal(plain, q128)
    greedy = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=9, p0=0.0, T=40)
    q0 = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=9, p0=0.2, T=40,
                       bias=np.zeros(g.n, np.uint8))
    assert np.array_equal(greedy, q0)


def test_bias_scales_the_flip_rate_per_vertex():
    # Edgeless graph: only the flip acts. Four groups of vertices with
    # q = 32, 64, 200, 255 must flip at rate thr[0] * q / 128 / 2^32.
    n = 4 * 30000
    e = np.zeros(0, dtype=np.int32)
    qs = np.array([32, 64, 200, 255], np.uint8)
    q = np.repeat(qs, n // 4)
    s0 = oracle.init_spins(n, 3)
    s = oracle.anneal(n, e, e, e, s0, seed=8, p0=0.25, T=2, sweeps=1, bias=q)
    thr = oracle.threshold(0.25, 2, 0)
    for k, qk in enumerate(qs):
        part = slice(k * (n // 4), (k + 1) * (n // 4))
        frac = float((s[part] != s0[part]).mean())
        p = (thr * int(qk) >> 7) / 2 ** 32
        assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / (n // 4)), (qk, frac, p)


def test_bias_threshold_clamps_at_the_top():
    # p0 = 1 and q = 255: thr * q / 128 exceeds 2^32 - 1 and clamps there, so
    # sweep 0 flips every spin whose word is not 2^32 - 1 (all of them here).
    n = 5000
    e = np.zeros(0, dtype=np.int32)
    s0 = oracle.init_spins(n, 2)
    s = oracle.anneal(n, e, e, e, s0, seed=6, p0=1.0, T=2, sweeps=1,
                      bias=np.full(n, 255, np.uint8))
    assert np.array_equal(s, -s0)


@pytest.mark.parametrize("replica", range(8))
def test_vertex_draws_share_philox_evaluations(replica):
    # R5: vertex v's initial spin and flip in replica r use word v mod 4 of the
    # counter (v // 4, t, r, stream), computed here with the KAT-pinned Philox.
    n, seed, inst = 301, 0x0123456789ABCDEF, 3
    key = [seed & 0xFFFFFFFF, ((seed >> 32) ^ (inst * 0x9E3779B9)) & 0xFFFFFFFF]
    words = lambda v, t, s: oracle.philox([v // 4, t, replica, s], key)[v % 4]
    s0 = oracle.init_spins(n, seed, instance=inst, replica=replica)
    want0 = np.array([-1 if words(v, 0, 1) >> 31 else 1 for v in range(n)], np.int8)
    assert np.array_equal(s0, want0)
    # edgeless graph, p0 = 1/2, T = 2: sweep 0 flips vertex v iff its word < 2^31
    e = np.zeros(0, dtype=np.int32)
    s1 = oracle.anneal(n, e, e, e, s0, seed=seed, instance=inst, replica=replica, p0=0.5, T=2,
                       sweeps=1)
    flipped = s1 != s0
    want = np.array([words(v, 0, 0) < 2 ** 31 for v in range(n)])
    assert np.array_equal(flipped, want)
