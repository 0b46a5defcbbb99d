"""The C-ABI library without a GPU: it builds, loads, exports every entry point
declared in include/ising.h, and its host-side logic (validation, merging,
colouring) behaves as documented. No compute call touches a device here."""

import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_1807_10750_gb300 import _build
    _build.build()
    import paper_1807_10750_gb300 as P
    return P


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ising_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol(P):
    import ctypes
    declared = declared_functions()
    assert "ising_create" in declared and "ising_anneal" in declared
    L = ctypes.CDLL(P.LIB_PATH)
    for name in declared:
        assert hasattr(L, name), name
    assert declared == set(P.EXPORTS)


def test_strerror_names_every_status(P):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert P.strerror(code) != "unknown status"
    assert P.strerror(-99) == "unknown status"


@pytest.mark.parametrize("n,src,dst,w,code", [
    (3, [0], [0], [1], -1),            # self-loop
    (3, [0], [3], [1], -1),            # id out of range
    (3, [-2], [1], [1], -1),           # negative id
    (0, [], [], [], -1),               # no vertices
    (-5, [], [], [], -1),
    (2, [0, 0], [1, 1], [2 ** 31 - 1, 1], -6),  # merged field exceeds int32
])
def test_create_rejects_invalid_input_before_touching_the_device(P, n, src, dst, w, code):
    with pytest.raises(P.IsingError) as e:
        P.ising_create(n, np.array(src, np.int32), np.array(dst, np.int32), np.array(w, np.int32))
    assert e.value.code == code


def test_plan_colouring_rejects_the_same_inputs(P):
    with pytest.raises(P.IsingError):
        P.ising_plan_colouring(3, [0], [0], [1])


@pytest.mark.parametrize("make", [
    lambda: synth.torus_graph(16, 0),
    lambda: synth.torus_graph(10, 1, weights="int8"),
    lambda: synth.random_small_graph(400, 0.03, 3, duplicates=80),
    lambda: synth.random_small_graph(50, 0.5, 4, weights="pm1", duplicates=200),
    lambda: synth.zipf_config_graph(5000, 2.1, 2, 400, 5),
    lambda: synth.complete_graph(9),
    lambda: synth.zipf_config_graph(6000, 2.0, 3, 1500, 41),   # hubs: two colour tiers
    lambda: synth.complete_graph(300),                        # every vertex a hub
])
def test_host_colouring_equals_oracle(P, make):
    g = make()
    C, col = P.ising_plan_colouring(g.n, g.src, g.dst, g.w)
    C2, col2 = oracle.colouring(g.n, g.src, g.dst, g.w)
    assert C == C2
    assert np.array_equal(col, col2)


def _big_duplicates_graph(seed):
    # 600k edge entries (the host build's multi-threaded passes start at
    # 2^19), a fifth of them repeated and some repeats cancelling to zero
    rng = np.random.default_rng(seed)
    n, m = 300_000, 500_000
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n, m)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    w = rng.integers(-8, 9, src.size)
    rep = rng.random(src.size) < 0.2
    w_rep = np.where(rng.random(rep.sum()) < 0.5, -w[rep], rng.integers(-8, 9, rep.sum()))
    return synth.Graph(n, np.concatenate([src, dst[rep]]).astype(np.int32),
                       np.concatenate([dst, src[rep]]).astype(np.int32),
                       np.concatenate([w, w_rep]).astype(np.int32))


@pytest.mark.parametrize("make", [
    lambda: _big_duplicates_graph(1),
    lambda: synth.zipf_config_graph(200_000, 2.1, 4, 5000, 7, weights="int8"),
])
def test_multithreaded_host_colouring_equals_oracle(P, make):
    g = make()
    assert g.src.size >= 1 << 19
    C, col = P.ising_plan_colouring(g.n, g.src, g.dst, g.w)
    C2, col2 = oracle.colouring(g.n, g.src, g.dst, g.w)
    assert C == C2
    assert np.array_equal(col, col2)
    assert P.ising_plan_colouring(g.n, g.src, g.dst, g.w)[1].tobytes() == col.tobytes()


@pytest.mark.parametrize("make", [
    # 8M and more merged entries: the colouring runs level by level on
    # several threads and must still equal the sequential first fit
    lambda: synth.zipf_config_graph(600_000, 2.1, 4, 10000, 3, weights="int8"),
    lambda: synth.er_graph(400_000, 24.0 / 399_999, 5, weights="int8"),
    # every vertex a hub (one tier only)
    lambda: synth.zipf_config_graph(30_000, 1.5, 300, 2000, 7),
])
def test_level_parallel_colouring_equals_oracle(P, make):
    g = make()
    assert 2 * g.m >= 1 << 23
    C, col = P.ising_plan_colouring(g.n, g.src, g.dst, g.w)
    C2, col2 = oracle.colouring(g.n, g.src, g.dst, g.w)
    assert C == C2
    assert np.array_equal(col, col2)


def test_large_build_merges_repeated_and_cancelling_edges(P):
    # more than 2^19 edges, so the directed rows are built by several threads
    # from per-thread edge ranges; edges listed again in either orientation
    # and exact cancellations (an edge plus its negation) must merge as the
    # oracle merges them, which the colouring shows
    g = synth.random_small_graph(300_000, 4.0 / 299_999, 31, weights="int8", duplicates=60_000)
    k = 20_000
    src = np.concatenate([g.src, g.dst[:k]]).astype(np.int32)
    dst = np.concatenate([g.dst, g.src[:k]]).astype(np.int32)
    w = np.concatenate([g.w, -g.w[:k]]).astype(np.int32)
    assert src.size >= 1 << 19
    C, col = P.ising_plan_colouring(g.n, src, dst, w)
    C2, col2 = oracle.colouring(g.n, src, dst, w)
    assert C == C2
    assert np.array_equal(col, col2)
    # the cancellations changed the graph: without them the colouring differs
    C3, col3 = P.ising_plan_colouring(g.n, g.src, g.dst, g.w)
    assert not np.array_equal(col, col3)


def test_host_colouring_edgeless_and_single_vertex(P):
    e = np.zeros(0, np.int32)
    C, col = P.ising_plan_colouring(5, e, e, e)
    assert C == 1 and np.all(col == 0)
    C, col = P.ising_plan_colouring(1, e, e, e)
    assert C == 1 and col[0] == 0


def test_zero_weight_merge_changes_colouring(P):
    src = np.array([0, 1, 1, 2, 0], np.int32)
    dst = np.array([1, 0, 2, 1, 2], np.int32)
    w = np.array([2, 3, 4, -4, 1], np.int32)
    C, col = P.ising_plan_colouring(3, src, dst, w)
    assert C == 2 and list(col) == [0, 1, 1]


def test_static_energy_rejects_bad_arguments_before_any_device_work(P):
    """ising_energy_csr_static checks its scalar arguments and null pointers
    before its first CUDA call, so these run without a GPU: n beyond the
    scratch array's capacity, n <= 0, and a null col or w."""
    import ctypes
    L = P.lib()
    buf = (ctypes.c_int32 * 4)()
    sp = (ctypes.c_int8 * 4)()
    out = (ctypes.c_int64 * 2)()
    a = ctypes.cast(buf, ctypes.c_void_p)
    s = ctypes.cast(sp, ctypes.c_void_p)
    o = ctypes.cast(out, ctypes.c_void_p)
    assert L.ising_energy_csr_static(P.ISING_STATIC_MAX_VERTICES + 1, a, a, a, s, o, None) == P.ISING_ERANGE
    assert L.ising_energy_csr_static(0, a, a, a, s, o, None) == P.ISING_EINVAL
    assert L.ising_energy_csr_static(4, a, None, a, s, o, None) == P.ISING_EINVAL
    assert L.ising_energy_csr_static(4, a, a, None, s, o, None) == P.ISING_EINVAL
    assert L.ising_energy_csr_static(4, None, a, a, s, o, None) == P.ISING_EINVAL


def test_static_energy_wrapper_checks_lengths(P):
    """The Python binding checks every tensor's length before the call (the
    kernels cannot): row_ptr n + 1, spins n, out 2, col and w equal. CPU
    tensors of the right lengths are refused as not on the device."""
    import torch
    n = 5
    good = dict(row_ptr=torch.zeros(n + 1, dtype=torch.int32), col=torch.zeros(8, dtype=torch.int32),
                w=torch.zeros(8, dtype=torch.int32), spins=torch.ones(n, dtype=torch.int8),
                out=torch.zeros(2, dtype=torch.int64))
    bad = [dict(row_ptr=torch.zeros(n, dtype=torch.int32)),
           dict(spins=torch.ones(n + 1, dtype=torch.int8)),
           dict(out=torch.zeros(1, dtype=torch.int64)),
           dict(w=torch.zeros(7, dtype=torch.int32))]
    for change in bad:
        args = dict(good, **change)
        with pytest.raises(ValueError):
            P.ising_energy_csr_static(n, args["row_ptr"], args["col"], args["w"], args["spins"],
                                      args["out"])
    with pytest.raises(TypeError):
        P.ising_energy_csr_static(n, good["row_ptr"], good["col"], good["w"], good["spins"],
                                  good["out"])
