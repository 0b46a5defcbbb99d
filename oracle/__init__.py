"""Python access to the CPU oracle (``ising_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs are the only callers.
The product package never imports this module, and this module imports
nothing from the product package.

Each function below follows one passage of the paper (Cook et al., "GPU Ising
Computing for Combinatorial Optimization Problems in VLSI Physical Design"):

* :func:`anneal` -- Algorithm 2 (update by Eq. 2, then flip with probability
  F_p), swept over greedy colour classes (the checkerboard scheme of
  Sec. IV-B generalised); readings R1-R7 are listed in ``ising_oracle.cpp``.
* :func:`energy_cut` -- Eq. 3/5 energy and the Eq. 4 cut.
* :func:`threshold` -- the linearly decaying flip probability F_p
  (Algorithm 2, "reduce F_p"; Sec. V-A, linear decay).
* :func:`philox` -- Philox4x32-10 (Salmon et al., SC'11), the counter-based
  generator that stands in for the per-thread cuRAND streams of Sec. IV-B.
* :func:`colouring` -- Welsh-Powell greedy colouring (reading R6).
* :func:`anneal` with ``bias`` -- a per-vertex flip bias (R11, a project
  addition used by the learned warm start; not in the paper).
* :func:`anneal_nflip` -- Algorithm 1's schedule: update every spin, then flip
  N_t distinct random spins, N decreasing linearly (reading R10).

Parity of the full spin trajectory is unpinned by the paper (it prints no
worked example); the pins are the properties checked in ``tests/``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ising_oracle.cpp")
_LIB = os.path.join(_HERE, "libising_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libising_oracle.so`` with g++."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i8p = ctypes.POINTER(ctypes.c_int8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.oracle_philox4x32_10.restype = ctypes.c_int
        L.oracle_random_word.argtypes = [ctypes.c_uint64, ctypes.c_uint32] + [ctypes.c_uint32] * 4
        L.oracle_random_word.restype = ctypes.c_uint32
        L.oracle_threshold.argtypes = [ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64]
        L.oracle_threshold.restype = ctypes.c_uint32
        L.oracle_num_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p]
        L.oracle_num_edges.restype = ctypes.c_int64
        L.oracle_colouring.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, i32p]
        L.oracle_colouring.restype = ctypes.c_int32
        L.oracle_init_spins.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_uint32, i8p]
        L.oracle_init_spins.restype = ctypes.c_int
        L.oracle_energy_cut.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, i8p,
                                        i64p, i64p, i64p]
        L.oracle_energy_cut.restype = ctypes.c_int
        L.oracle_anneal.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, i8p,
                                    ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_uint64]
        L.oracle_anneal.restype = ctypes.c_int
        L.oracle_anneal_biased.argtypes = L.oracle_anneal.argtypes + [ctypes.POINTER(ctypes.c_uint8)]
        L.oracle_anneal_biased.restype = ctypes.c_int
        L.oracle_anneal_nflip.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, i8p,
                                          ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.c_uint64]
        L.oracle_anneal_nflip.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _edges(src, dst, w):
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.int32)
    assert src.shape == dst.shape == w.shape
    return src, dst, w


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of a 4-word counter and 2-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def random_word(seed: int, instance: int, c0: int, c1: int, c2: int, c3: int) -> int:
    return int(lib().oracle_random_word(seed, instance, c0, c1, c2, c3))


def threshold(p0: float, T: int, t: int) -> int:
    return int(lib().oracle_threshold(p0, T, t))


def num_edges(n, src, dst, w) -> int:
    src, dst, w = _edges(src, dst, w)
    r = lib().oracle_num_edges(n, src.size, _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32),
                               _p(w, ctypes.c_int32))
    if r < 0:
        raise ValueError("invalid graph")
    return int(r)


def colouring(n, src, dst, w):
    """Returns (number of colours, colour per vertex)."""
    src, dst, w = _edges(src, dst, w)
    col = np.zeros(n, dtype=np.int32)
    C = lib().oracle_colouring(n, src.size, _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32),
                               _p(w, ctypes.c_int32), _p(col, ctypes.c_int32))
    if C < 0:
        raise ValueError("invalid graph")
    return int(C), col


def init_spins(n: int, seed: int, instance: int = 0, replica: int = 0) -> np.ndarray:
    s = np.zeros(n, dtype=np.int8)
    if lib().oracle_init_spins(n, seed, instance, replica, _p(s, ctypes.c_int8)) != 0:
        raise ValueError("invalid n")
    return s


def energy_cut(n, src, dst, w, s):
    """Returns (H, W, cut) as Python ints."""
    src, dst, w = _edges(src, dst, w)
    s = np.ascontiguousarray(s, dtype=np.int8)
    H = ctypes.c_int64()
    W = ctypes.c_int64()
    cut = ctypes.c_int64()
    r = lib().oracle_energy_cut(n, src.size, _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32),
                                _p(w, ctypes.c_int32), _p(s, ctypes.c_int8), ctypes.byref(H),
                                ctypes.byref(W), ctypes.byref(cut))
    if r != 0:
        raise ValueError("invalid graph")
    return H.value, W.value, cut.value


def anneal(n, src, dst, w, s, *, seed: int, p0: float, T: int, t_begin: int = 0,
           sweeps: int | None = None, instance: int = 0, replica: int = 0,
           bias=None) -> np.ndarray:
    """Deterministic anneal; returns the new spin vector (input not modified).
    ``bias``: optional uint8 per-vertex flip bias q (R11; 128 = unbiased)."""
    src, dst, w = _edges(src, dst, w)
    out = np.array(s, dtype=np.int8, copy=True)
    if sweeps is None:
        sweeps = T - t_begin
    if bias is None:
        r = lib().oracle_anneal(n, src.size, _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32),
                                _p(w, ctypes.c_int32), _p(out, ctypes.c_int8), seed, instance,
                                replica, p0, T, t_begin, sweeps)
    else:
        q = np.ascontiguousarray(bias, dtype=np.uint8)
        assert q.shape == (n,)
        r = lib().oracle_anneal_biased(n, src.size, _p(src, ctypes.c_int32),
                                       _p(dst, ctypes.c_int32), _p(w, ctypes.c_int32),
                                       _p(out, ctypes.c_int8), seed, instance, replica, p0, T,
                                       t_begin, sweeps, _p(q, ctypes.c_uint8))
    if r != 0:
        raise ValueError("invalid anneal arguments")
    return out


def anneal_nflip(n, src, dst, w, s, *, seed: int, n0: int, T: int, t_begin: int = 0,
                 sweeps: int | None = None, instance: int = 0, replica: int = 0) -> np.ndarray:
    """Algorithm 1's N-flip schedule; returns the new spins (input unchanged)."""
    src, dst, w = _edges(src, dst, w)
    out = np.array(s, dtype=np.int8, copy=True)
    if sweeps is None:
        sweeps = T - t_begin
    r = lib().oracle_anneal_nflip(n, src.size, _p(src, ctypes.c_int32), _p(dst, ctypes.c_int32),
                                  _p(w, ctypes.c_int32), _p(out, ctypes.c_int8), seed, instance,
                                  replica, n0, T, t_begin, sweeps)
    if r != 0:
        raise ValueError("invalid N-flip anneal arguments")
    return out
