"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Deterministic mode must match the oracle bit for bit in spins, energy and cut.
The racy mode is judged by cut value only.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

ENGINES = ["phase", "persistent", "dataflow", "persistent_grid", "itemflow", "halo", "hub"]


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_1807_10750_gb300 import _build
    _build.build()
    import paper_1807_10750_gb300 as P
    return P


def engine_id(P, name):
    return {"phase": P.ISING_ENGINE_PHASE, "persistent": P.ISING_ENGINE_PERSISTENT,
            "dataflow": P.ISING_ENGINE_DATAFLOW, "auto": P.ISING_ENGINE_AUTO,
            "persistent_grid": P.ISING_ENGINE_PERSISTENT_GRID,
            "itemflow": P.ISING_ENGINE_ITEMFLOW, "halo": P.ISING_ENGINE_HALO,
            "hub": P.ISING_ENGINE_HUB}[name]


def gpu_anneal(P, g, s0, *, seed, p0, T, t_begin=0, sweeps=None, flags=0, engine="auto",
               mode=None, replica=0):
    with P.ising_create(g.n, g.src, g.dst, g.w, flags=flags) as h:
        P.ising_set_engine(h, engine_id(P, engine))
        P.ising_set_spins(h, s0)
        P.ising_anneal(h, p0=p0, t_total=T, t_begin=t_begin, sweeps=sweeps, seed=seed,
                       mode=P.ISING_MODE_DET if mode is None else mode, replica=replica)
        s = P.ising_get_spins(h)
        return s, P.ising_energy(h), P.ising_cut(h)


def check_det(P, g, *, seed, p0, T, t_begin=0, sweeps=None, s0=None, flags=0, engine="auto",
              replica=0):
    if s0 is None:
        s0 = oracle.init_spins(g.n, seed + 1000)
    want = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=seed, p0=p0, T=T, t_begin=t_begin,
                         sweeps=sweeps, replica=replica)
    got, H, cut = gpu_anneal(P, g, s0, seed=seed, p0=p0, T=T, t_begin=t_begin, sweeps=sweeps,
                             flags=flags, engine=engine, replica=replica)
    mism = np.nonzero(got != want)[0]
    assert mism.size == 0, f"{mism.size} spins differ, first at {mism[:8]}"
    Hw, W, cutw = oracle.energy_cut(g.n, g.src, g.dst, g.w, want)
    assert (H, cut) == (Hw, cutw)
    return got


SMALL_GRAPHS = {
    "er_dup_int8": lambda: synth.random_small_graph(300, 0.04, 1, weights="int8", duplicates=60),
    "er_dense_pm1": lambda: synth.random_small_graph(120, 0.5, 2, weights="pm1"),
    "torus_pm1": lambda: synth.torus_graph(16, 3, weights="pm1"),
    "torus_odd": lambda: synth.torus_graph(15, 4, weights="int8", Ly=9),
    "grid_one": lambda: synth.grid_graph(13, 7),
    "complete": lambda: synth.complete_graph(40, 5, weights="int8"),
    "zipf_small": lambda: synth.zipf_config_graph(20000, 2.1, 2, 3000, 6),
    "cycle_odd": lambda: synth.cycle_graph(33),
}


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("name", sorted(SMALL_GRAPHS))
def test_det_bit_exact_small(P, name, engine):
    g = SMALL_GRAPHS[name]()
    check_det(P, g, seed=17, p0=0.15, T=60, engine=engine)


@pytest.mark.parametrize("engine", ENGINES)
def test_det_bit_exact_int32_weights(P, engine):
    g = synth.random_small_graph(500, 0.02, 8, weights="int8")
    g.w = (g.w * 97).astype(np.int32)  # beyond int8
    check_det(P, g, seed=3, p0=0.1, T=40, engine=engine)
    g2 = synth.random_small_graph(500, 0.02, 8, weights="int8")
    check_det(P, g2, seed=3, p0=0.1, T=40, flags=P.ISING_CREATE_WEIGHTS_I32, engine=engine)


@pytest.mark.parametrize("engine", ENGINES)
def test_det_hub_rows_sliced_across_warps(P, engine):
    # A star-heavy graph: two hubs of degree ~n plus sparse noise, so the hubs'
    # rows are split into many slices combined through the partial-sum slots.
    rng = np.random.default_rng(0)
    n = 60000
    hub_a = np.full(n - 2, 0, np.int32); leaf = np.arange(2, n, dtype=np.int32)
    hub_b = np.full(n // 2, 1, np.int32); leaf_b = rng.choice(np.arange(2, n), n // 2, replace=False).astype(np.int32)
    noise = synth.er_graph(n, 3.0 / n, 1, weights="int8")
    src = np.concatenate([hub_a, hub_b, noise.src]); dst = np.concatenate([leaf, leaf_b, noise.dst])
    w = synth.draw_weights("int8", src.size, rng)
    g = synth.Graph(n, src.astype(np.int32), dst.astype(np.int32), w)
    check_det(P, g, seed=5, p0=0.2, T=30, engine=engine)


@pytest.mark.parametrize("engine", ENGINES)
def test_det_edge_cases(P, engine):
    e = np.zeros(0, np.int32)
    for n in (1, 2, 37, 100000):
        g = synth.Graph(n, e, e, e)
        check_det(P, g, seed=n, p0=0.4, T=7, engine=engine)
    # merged-zero edges vanish
    g = synth.Graph(3, np.array([0, 1, 1, 2], np.int32), np.array([1, 0, 2, 1], np.int32),
                    np.array([2, 3, 4, -4], np.int32))
    check_det(P, g, seed=2, p0=0.3, T=9, engine=engine)


@pytest.mark.parametrize("engine", ENGINES)
def test_er800_full_schedule_bit_exact(P, engine):
    # G(800, 0.06), unit weights, 1000 sweeps, p0 = 0.1, seed 1.
    g, sch = synth.workload("er800")
    s0 = oracle.init_spins(g.n, sch["seed"])
    check_det(P, g, seed=sch["seed"], p0=sch["p0"], T=sch["sweeps"], s0=s0, engine=engine)


@pytest.mark.parametrize("engine", ENGINES)
def test_torus1024_full_size_segments_bit_exact(P, engine):
    # The 1024 x 1024 torus of the benchmark: first and last sweeps of the
    # 2000-sweep schedule, each from a shared state.
    g, sch = synth.workload("torus1024")
    T = sch["sweeps"]
    s0 = oracle.init_spins(g.n, sch["seed"])
    s1 = check_det(P, g, seed=sch["seed"], p0=sch["p0"], T=T, sweeps=12, s0=s0, engine=engine)
    check_det(P, g, seed=sch["seed"], p0=sch["p0"], T=T, t_begin=T - 12, s0=s1, engine=engine)


def test_zipf1m_full_size_segment_bit_exact(P):
    g, sch = synth.workload("zipf1m")
    s0 = oracle.init_spins(g.n, sch["seed"])
    for engine in ENGINES:
        check_det(P, g, seed=sch["seed"], p0=sch["p0"], T=sch["sweeps"], sweeps=3, s0=s0,
                  engine=engine)


def test_init_random_matches_oracle(P):
    g = synth.random_small_graph(3000, 0.002, 9)
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        for seed, rep in [(0, 0), (1, 0), (2 ** 40 + 7, 3)]:
            P.ising_init_random(h, seed, rep)
            assert np.array_equal(P.ising_get_spins(h), oracle.init_spins(g.n, seed, replica=rep))


def test_energy_and_cut_match_oracle(P):
    g = synth.random_small_graph(2000, 0.01, 10, weights="int8", duplicates=300)
    rng = np.random.default_rng(1)
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        assert P.ising_num_edges(h) == oracle.num_edges(g.n, g.src, g.dst, g.w)
        for _ in range(4):
            s = (rng.integers(0, 2, g.n) * 2 - 1).astype(np.int8)
            P.ising_set_spins(h, s)
            H, W, cut = oracle.energy_cut(g.n, g.src, g.dst, g.w, s)
            assert P.ising_energy(h) == H
            assert P.ising_cut(h) == cut
            assert P.ising_total_weight(h) == W


@pytest.mark.parametrize("engine", ENGINES)
def test_split_anneal_equals_whole(P, engine):
    g = synth.random_small_graph(5000, 0.002, 11, weights="int8")
    s0 = oracle.init_spins(g.n, 4)
    whole, _, _ = gpu_anneal(P, g, s0, seed=9, p0=0.2, T=50, engine=engine)
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        P.ising_set_engine(h, engine_id(P, engine))
        P.ising_set_spins(h, s0)
        P.ising_anneal(h, p0=0.2, t_total=50, sweeps=17, seed=9)
        P.ising_anneal(h, p0=0.2, t_total=50, t_begin=17, sweeps=0, seed=9)
        P.ising_anneal(h, p0=0.2, t_total=50, t_begin=17, seed=9)
        assert np.array_equal(P.ising_get_spins(h), whole)


def test_spins_roundtrip_host_and_device(P):
    import torch
    g = synth.random_small_graph(1000, 0.01, 12)
    rng = np.random.default_rng(2)
    s = (rng.integers(0, 2, g.n) * 2 - 1).astype(np.int8)
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        P.ising_set_spins(h, s)
        assert np.array_equal(P.ising_get_spins(h), s)
        dev = torch.from_numpy(-s).cuda()
        P.ising_set_spins(h, dev)
        out = torch.zeros(g.n, dtype=torch.int8, device="cuda")
        P.ising_get_spins(h, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), -s)
        bad = s.copy(); bad[5] = 0
        with pytest.raises(P.IsingError):
            P.ising_set_spins(h, bad)
        bad_dev = torch.from_numpy(bad).cuda()
        with pytest.raises(P.IsingError):
            P.ising_set_spins(h, bad_dev)
        assert np.array_equal(P.ising_get_spins(h), -s)  # unchanged by rejected calls


def test_anneal_argument_errors(P):
    g = synth.cycle_graph(10)
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        for kw in (dict(p0=1.5, t_total=10), dict(p0=-0.1, t_total=10),
                   dict(p0=0.1, t_total=10, t_begin=8, sweeps=3), dict(p0=0.1, t_total=2 ** 32)):
            with pytest.raises(P.IsingError) as e:
                P.ising_anneal(h, seed=1, **kw)
            assert e.value.code == P.ISING_EINVAL
        with pytest.raises(P.IsingError):
            P.ising_anneal(h, seed=1, p0=0.1, t_total=10, mode=7)
        with pytest.raises(P.IsingError):
            P.ising_set_engine(h, 9)
        # the handle still works after rejected calls
        P.ising_anneal(h, seed=1, p0=0.1, t_total=10)
        assert P.ising_cut(h) >= 0


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("name", ["torus256", "er800"])
def test_racy_mode_cut_quality(P, name, engine):
    if name == "torus256":
        g, T = synth.torus_graph(256, 7, weights="pm1"), 400
    else:
        g, T = synth.workload("er800")[0], 1000
    det, racy = [], []
    for seed in range(6):
        s0 = oracle.init_spins(g.n, seed)
        det.append(gpu_anneal(P, g, s0, seed=seed, p0=0.1, T=T)[2])
        s, H, cut = gpu_anneal(P, g, s0, seed=seed, p0=0.1, T=T, mode=P.ISING_MODE_RACY,
                               engine=engine)
        assert set(np.unique(s)) <= {-1, 1}
        assert (H, cut) == oracle.energy_cut(g.n, g.src, g.dst, g.w, s)[::2]
        racy.append(cut)
    assert np.mean(racy) >= 0.98 * np.mean(det), (racy, det)


@pytest.mark.parametrize("engine", ENGINES)
def test_energy_trace_matches_oracle_checkpoints(P, engine):
    g = synth.random_small_graph(700, 0.01, 21, weights="int8", duplicates=30)
    s0 = oracle.init_spins(g.n, 3)
    T, every = 50, 7
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        P.ising_set_engine(h, engine_id(P, engine))
        P.ising_set_spins(h, s0)
        trace = P.ising_anneal_trace(h, p0=0.2, t_total=T, seed=4, every=every)
        final = P.ising_energy(h)
    assert trace.size == -(-T // every) and trace[-1] == final
    s = s0.copy()
    for i in range(trace.size):
        k = min(every, T - i * every)
        s = oracle.anneal(g.n, g.src, g.dst, g.w, s, seed=4, p0=0.2, T=T, t_begin=i * every, sweeps=k)
        assert trace[i] == oracle.energy_cut(g.n, g.src, g.dst, g.w, s)[0], i


def test_convergence_region_matches_oracle(P):
    # Fig. 4's region: per seed, random start and anneal with that seed; the
    # library's cut after every chunk, and its min / max over the seeds, equal
    # the oracle's.
    g = synth.torus_graph(32, 5, weights="pm1")
    T, every, seeds = 100, 10, [3, 9, 27, 81]
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        idx, cuts, lo, hi = P.ising_convergence_region(h, seeds=seeds, p0=0.1, t_total=T, every=every)
    assert idx.tolist() == list(range(10, 101, 10))
    want = np.zeros((len(seeds), T // every), np.int64)
    for k, sd in enumerate(seeds):
        s = oracle.init_spins(g.n, sd)
        for i in range(T // every):
            s = oracle.anneal(g.n, g.src, g.dst, g.w, s, seed=sd, p0=0.1, T=T, t_begin=i * every,
                              sweeps=every)
            want[k, i] = oracle.energy_cut(g.n, g.src, g.dst, g.w, s)[2]
    assert np.array_equal(cuts, want)
    assert np.array_equal(lo, want.min(axis=0)) and np.array_equal(hi, want.max(axis=0))
    # annealing improves the cut from early to late checkpoints on average
    assert cuts[:, -1].mean() > cuts[:, 0].mean()


def gpu_anneal_nflip(P, g, s0, *, seed, n0, T, t_begin=0, sweeps=None, engine="auto", mode=None):
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        P.ising_set_engine(h, engine_id(P, engine))
        P.ising_set_spins(h, s0)
        P.ising_anneal(h, kind=P.ISING_SCHED_NFLIP, n0=n0, t_total=T, t_begin=t_begin,
                       sweeps=sweeps, seed=seed, mode=P.ISING_MODE_DET if mode is None else mode)
        return P.ising_get_spins(h), P.ising_cut(h)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("name", ["er_dup_int8", "torus_pm1", "zipf_small", "complete"])
def test_nflip_schedule_bit_exact(P, name, engine):
    g = SMALL_GRAPHS[name]()
    s0 = oracle.init_spins(g.n, 12)
    n0 = min(g.n, 37)
    want = oracle.anneal_nflip(g.n, g.src, g.dst, g.w, s0, seed=6, n0=n0, T=40)
    got, cut = gpu_anneal_nflip(P, g, s0, seed=6, n0=n0, T=40, engine=engine)
    assert np.array_equal(got, want)
    assert cut == oracle.energy_cut(g.n, g.src, g.dst, g.w, want)[2]


@pytest.mark.parametrize("engine", ["phase", "persistent"])
def test_nflip_paper_setting_er800(P, engine):
    # the paper's accuracy runs: 1000 sweeps, 200 random flips decaying linearly
    g, sch = synth.workload("er800")
    s0 = oracle.init_spins(g.n, 1)
    want = oracle.anneal_nflip(g.n, g.src, g.dst, g.w, s0, seed=1, n0=200, T=1000)
    got, _ = gpu_anneal_nflip(P, g, s0, seed=1, n0=200, T=1000, engine=engine)
    assert np.array_equal(got, want)


def test_nflip_edge_cases(P):
    e = np.zeros(0, np.int32)
    g = synth.Graph(3000, e, e, e)
    s0 = oracle.init_spins(g.n, 2)
    for n0 in (g.n, 1, 0):
        want = oracle.anneal_nflip(g.n, e, e, e, s0, seed=4, n0=n0, T=3)
        for engine in ("phase", "persistent"):
            got, _ = gpu_anneal_nflip(P, g, s0, seed=4, n0=n0, T=3, engine=engine)
            assert np.array_equal(got, want), (n0, engine)
    # split equals whole, and n0 > n is rejected
    g = SMALL_GRAPHS["er_dup_int8"]()
    s0 = oracle.init_spins(g.n, 3)
    whole = oracle.anneal_nflip(g.n, g.src, g.dst, g.w, s0, seed=8, n0=50, T=30)
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        P.ising_set_spins(h, s0)
        P.ising_anneal(h, kind=P.ISING_SCHED_NFLIP, n0=50, t_total=30, sweeps=11, seed=8)
        P.ising_anneal(h, kind=P.ISING_SCHED_NFLIP, n0=50, t_total=30, t_begin=11, seed=8)
        assert np.array_equal(P.ising_get_spins(h), whole)
        with pytest.raises(P.IsingError):
            P.ising_anneal(h, kind=P.ISING_SCHED_NFLIP, n0=g.n + 1, t_total=30, seed=8)


# Graphs the persistent engine anneals in one block (int8 weights, at most
# 4095 vertices): dense with repeated edges (29 classes), K_40 (40 classes of
# one vertex), a torus (2 classes), a 4095-vertex random graph (the size
# limit) and a single vertex. The first three keep every packed word in
# shared memory (resident form); the 4095-vertex graph's 168k words stream
# through the ring of bulk copies. Deterministic sweeps, with and without a
# flip bias and Algorithm 1's schedule, must match the grid-barrier form and
# the oracle bit for bit.
BLOCK_GRAPHS = {
    "dense300": lambda: synth.random_small_graph(300, 0.3, 3, weights="int8", duplicates=100),
    "complete40": lambda: synth.complete_graph(40, 1, weights="pm1"),
    "torus32": lambda: synth.torus_graph(32, 1, weights="pm1"),
    "n4095": lambda: synth.random_small_graph(4095, 0.01, 8, weights="int8"),
    "single": lambda: synth.Graph(1, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32)),
}


@pytest.mark.parametrize("name", sorted(BLOCK_GRAPHS))
@pytest.mark.parametrize("biased", [False, True])
def test_block_engine_matches_grid_engine_and_oracle(P, name, biased):
    g = BLOCK_GRAPHS[name]()
    q = np.random.default_rng(9).integers(0, 256, size=g.n).astype(np.uint8) if biased else None
    T = 40
    out = {}
    for engine in ("persistent", "persistent_grid"):
        with P.ising_create(g.n, g.src, g.dst, g.w) as h:
            P.ising_set_engine(h, engine_id(P, engine))
            P.ising_init_random(h, 2)
            s0 = P.ising_get_spins(h)
            if biased:
                P.ising_set_flip_bias(h, q)
            P.ising_anneal(h, p0=0.2, t_total=T, seed=5, sweeps=17)
            P.ising_anneal(h, p0=0.2, t_total=T, seed=5, t_begin=17)
            out[engine] = (P.ising_get_spins(h), P.ising_cut(h))
    assert np.array_equal(out["persistent"][0], out["persistent_grid"][0])
    want = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=5, p0=0.2, T=T, bias=q)
    assert np.array_equal(out["persistent"][0], want)
    assert out["persistent"][1] == oracle.energy_cut(g.n, g.src, g.dst, g.w, want)[2]


@pytest.mark.parametrize("name", ["dense300", "n4095"])
def test_block_engine_nflip_schedule(P, name):
    g = BLOCK_GRAPHS[name]()
    n0, T = min(200, g.n), 60
    with P.ising_create(g.n, g.src, g.dst, g.w) as h:
        P.ising_init_random(h, 6)
        s0 = P.ising_get_spins(h)
        P.ising_anneal(h, t_total=T, seed=7, kind=P.ISING_SCHED_NFLIP, n0=n0)
        got = P.ising_get_spins(h)
    want = oracle.anneal_nflip(g.n, g.src, g.dst, g.w, s0, seed=7, n0=n0, T=T)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("name", ["torus96", "er5k_sparse", "grid_open"])
def test_itemflow_engine_matches_oracle_over_many_sweeps(P, name):
    # graphs whose rows are never sliced across warps, so the item-dataflow
    # engine runs them; many sweeps let items run ahead of one another
    g = {"torus96": lambda: synth.torus_graph(96, 2, weights="pm1"),
         "er5k_sparse": lambda: synth.random_small_graph(5000, 0.002, 3, weights="int8"),
         "grid_open": lambda: synth.grid_graph(70, 53, 1, weights="int8")}[name]()
    s0 = oracle.init_spins(g.n, 3)
    got, _, _ = gpu_anneal(P, g, s0, seed=4, p0=0.15, T=300, engine="itemflow")
    want = oracle.anneal(g.n, g.src, g.dst, g.w, s0, seed=4, p0=0.15, T=300)
    assert np.array_equal(got, want)


def _stars_without_hubs():
    # a sparse random graph plus 20 vertices of about 210 neighbours each:
    # rows long enough to be sliced across warps, but no vertex reaches the
    # hub degree (256)
    rng = np.random.default_rng(9)
    base = synth.random_small_graph(20000, 4e-4, 2)
    centres = np.repeat(np.arange(20, dtype=np.int32), 200)
    leaves = np.concatenate([rng.choice(np.arange(20, 20000), 200, replace=False) for _ in range(20)])
    src = np.concatenate([base.src, centres]).astype(np.int32)
    dst = np.concatenate([base.dst, leaves]).astype(np.int32)
    w = np.concatenate([base.w, synth.draw_weights("int8", centres.size, rng)]).astype(np.int32)
    return synth.Graph(20000, src, dst, w)


def test_auto_engine_choice(P):
    # small graph -> the one-block form; a lattice with about 1000 vertices
    # per SM -> halo; unsliced large graph without a halo plan (or with too
    # much repeated work) -> item dataflow; a graph with hubs -> the hub
    # engine; sliced rows without hubs -> the grid engine; racy and N-flip
    # anneals of an unsliced graph -> the grid engine
    cases = [
        (synth.random_small_graph(400, 0.03, 1, weights="int8"), {}, P.ISING_ENGINE_USED_BLOCK),
        (synth.torus_graph(384, 2, weights="pm1"), {}, P.ISING_ENGINE_HALO),
        (synth.torus_graph(100, 2, weights="pm1"), {}, P.ISING_ENGINE_ITEMFLOW),
        (synth.torus_graph(96, 2, weights="pm1"), {}, P.ISING_ENGINE_ITEMFLOW),
        (synth.random_small_graph(20000, 4e-4, 2), {}, P.ISING_ENGINE_ITEMFLOW),
        (synth.zipf_config_graph(20011, 2.1, 4, 3000, 5), {}, P.ISING_ENGINE_HUB),
        (_stars_without_hubs(), {}, P.ISING_ENGINE_PERSISTENT_GRID),
        (synth.zipf_config_graph(20011, 2.1, 4, 3000, 5), {"mode": P.ISING_MODE_RACY},
         P.ISING_ENGINE_PERSISTENT_GRID),
        (synth.torus_graph(96, 2, weights="pm1"), {"mode": P.ISING_MODE_RACY},
         P.ISING_ENGINE_PERSISTENT_GRID),
        (synth.torus_graph(96, 2, weights="pm1"), {"kind": P.ISING_SCHED_NFLIP, "n0": 50},
         P.ISING_ENGINE_PERSISTENT_GRID),
    ]
    for g, kw, want in cases:
        with P.ising_create(g.n, g.src, g.dst, g.w) as h:
            assert P.ising_engine_used(h) == -1
            P.ising_halo_info(h)  # the halo plan is built by a host thread: wait for it
            P.ising_init_random(h, 1)
            P.ising_anneal(h, p0=0.1, t_total=10, seed=1, **kw)
            assert P.ising_engine_used(h) == want, (g.n, kw)
