"""GB300 Ising max-cut annealer: thin Python binding of ``include/ising.h``.

Every function here marshals arguments and calls the C ABI of
``libising_gb300.so`` (built in-tree by ``paper_1807_10750_gb300._build``);
all compute runs in the library's CUDA kernels. There is no CPU fallback: if
the library is missing, :func:`lib` raises.

Device buffers may be torch CUDA tensors (their ``data_ptr()`` is passed with
``on_device=1``); streams may be ``torch.cuda.Stream`` objects or raw
``cudaStream_t`` integers.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libising_gb300.so")

ISING_OK = 0
ISING_EINVAL = -1
ISING_ENOMEM = -2
ISING_ECUDA = -3
ISING_ETIMEOUT = -4
ISING_ESTATE = -5
ISING_ERANGE = -6

ISING_MODE_DET = 0
ISING_MODE_RACY = 1
ISING_SCHED_LINEAR = 0
ISING_SCHED_NFLIP = 1
ISING_ENGINE_AUTO = 0
ISING_ENGINE_PHASE = 1
ISING_ENGINE_PERSISTENT = 2
ISING_ENGINE_DATAFLOW = 3
ISING_ENGINE_PERSISTENT_GRID = 4
ISING_ENGINE_ITEMFLOW = 5
ISING_ENGINE_HALO = 7
ISING_ENGINE_HUB = 8
ISING_CREATE_WEIGHTS_I32 = 1
ISING_STATIC_MAX_VERTICES = 1 << 24

# Every entry point declared in include/ising.h.
EXPORTS = (
    "ising_create", "ising_anneal", "ising_energy", "ising_cut", "ising_total_weight",
    "ising_get_spins", "ising_set_spins", "ising_init_random", "ising_num_colours",
    "ising_colouring", "ising_num_edges", "ising_set_engine", "ising_destroy",
    "ising_strerror", "ising_plan_colouring", "ising_launch_count", "ising_energy_csr_static",
    "ising_batch_create", "ising_batch_init_random", "ising_batch_anneal", "ising_batch_cuts",
    "ising_batch_get_spins", "ising_batch_set_spins", "ising_batch_autotune", "ising_batch_set_block",
    "ising_batch_info", "ising_batch_destroy", "ising_anneal_trace",
    "ising_set_flip_bias", "ising_get_flip_bias", "ising_gnn_create", "ising_gnn_set_params",
    "ising_gnn_get_params", "ising_gnn_forward", "ising_gnn_gradients", "ising_gnn_train_step",
    "ising_gnn_warm_start", "ising_gnn_launch_count", "ising_gnn_destroy", "ising_debug_fault",
    "ising_engine_used", "ising_set_halo_sweeps", "ising_halo_info", "ising_plan_halo",
    "ising_convergence_region", "ising_batch_set_tuning", "ising_batch_tuning",
    "ising_gnn_batch_forward", "ising_gnn_batch_warm_start", "ising_gnn_batch_gradients",
    "ising_gnn_batch_train_step", "ising_gnn_set_dense_path",
)
ISING_ENGINE_USED_BLOCK = 6
ISING_FAULT_NONE = 0
ISING_FAULT_SKIP_ARRIVAL = 1
ISING_FAULT_SHORT_COPY = 2
ISING_GNN_NUM_PARAMS = 17665
ISING_ALL_REPLICAS = 0xFFFFFFFF
ISING_GNN_DENSE_TCGEN05 = 0
ISING_GNN_DENSE_MMA_SYNC = 1


class IsingError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


class ising_schedule(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("replica", ctypes.c_uint32), ("p0", ctypes.c_double),
                ("t_begin", ctypes.c_uint64), ("t_total", ctypes.c_uint64), ("n0", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_1807_10750_gb300._build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.ising_create.argtypes = [ctypes.c_int32, ctypes.c_int64, vp, vp, vp, ctypes.c_uint32, vp,
                                   ctypes.POINTER(vp)]
        L.ising_anneal.argtypes = [vp, ctypes.POINTER(ising_schedule), ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_int, vp]
        L.ising_energy.argtypes = [vp, i64p]
        L.ising_cut.argtypes = [vp, i64p]
        L.ising_total_weight.argtypes = [vp, i64p]
        L.ising_get_spins.argtypes = [vp, vp, ctypes.c_int]
        L.ising_set_spins.argtypes = [vp, vp, ctypes.c_int]
        L.ising_init_random.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint32]
        L.ising_num_colours.argtypes = [vp, i32p]
        L.ising_colouring.argtypes = [vp, i32p]
        L.ising_num_edges.argtypes = [vp, i64p]
        L.ising_set_engine.argtypes = [vp, ctypes.c_int]
        L.ising_destroy.argtypes = [vp]
        L.ising_destroy.restype = None
        L.ising_plan_colouring.argtypes = [ctypes.c_int32, ctypes.c_int64, vp, vp, vp, i32p, i32p]
        L.ising_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        L.ising_energy_csr_static.argtypes = [ctypes.c_int32, vp, vp, vp, vp, vp, vp]
        L.ising_anneal_trace.argtypes = [vp, ctypes.POINTER(ising_schedule), ctypes.c_uint32,
                                         ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, vp, vp]
        L.ising_convergence_region.argtypes = [vp, ctypes.POINTER(ising_schedule), ctypes.c_uint32,
                                               vp, ctypes.c_uint32, ctypes.c_int, ctypes.c_uint32,
                                               vp, vp, vp, vp]
        L.ising_batch_create.argtypes = [ctypes.c_int32, vp, vp, vp, vp, vp, ctypes.c_uint32, vp,
                                         ctypes.POINTER(vp)]
        L.ising_batch_init_random.argtypes = [vp, ctypes.c_uint64]
        L.ising_batch_anneal.argtypes = [vp, ctypes.POINTER(ising_schedule), ctypes.c_uint32,
                                         ctypes.c_uint64, vp]
        L.ising_batch_cuts.argtypes = [vp, vp]
        L.ising_batch_get_spins.argtypes = [vp, ctypes.c_int32, ctypes.c_uint32, vp]
        L.ising_batch_set_spins.argtypes = [vp, ctypes.c_int32, ctypes.c_uint32, vp]
        L.ising_batch_autotune.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32)]
        L.ising_batch_set_block.argtypes = [vp, ctypes.c_int32]
        L.ising_batch_set_tuning.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        L.ising_batch_tuning.argtypes = [vp, vp, vp, vp, vp]
        L.ising_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), i64p,
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint64)]
        L.ising_batch_destroy.argtypes = [vp]
        L.ising_batch_destroy.restype = None
        L.ising_set_flip_bias.argtypes = [vp, vp, ctypes.c_int]
        L.ising_get_flip_bias.argtypes = [vp, vp]
        L.ising_gnn_create.argtypes = [vp, ctypes.POINTER(ctypes.c_void_p)]
        L.ising_gnn_set_params.argtypes = [vp, vp]
        L.ising_gnn_get_params.argtypes = [vp, vp]
        L.ising_gnn_forward.argtypes = [vp, vp, vp, ctypes.c_int]
        L.ising_gnn_gradients.argtypes = [vp, vp, vp, ctypes.c_int, vp, vp]
        L.ising_gnn_train_step.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_float, vp]
        L.ising_gnn_warm_start.argtypes = [vp, vp, ctypes.c_int]
        L.ising_gnn_batch_forward.argtypes = [vp, vp, ctypes.c_uint32, vp, ctypes.c_int]
        L.ising_gnn_batch_warm_start.argtypes = [vp, vp, ctypes.c_uint32]
        L.ising_gnn_set_dense_path.argtypes = [vp, ctypes.c_int]
        L.ising_gnn_batch_gradients.argtypes = [vp, vp, ctypes.c_uint32, vp, ctypes.c_int, vp, vp]
        L.ising_gnn_batch_train_step.argtypes = [vp, vp, ctypes.c_uint32, vp, ctypes.c_int, ctypes.c_float, vp]
        L.ising_gnn_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        L.ising_gnn_destroy.argtypes = [vp]
        L.ising_gnn_destroy.restype = None
        L.ising_debug_fault.argtypes = [vp, ctypes.c_int, ctypes.c_uint64]
        L.ising_engine_used.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
        L.ising_set_halo_sweeps.argtypes = [vp, ctypes.c_uint32]
        L.ising_plan_halo.argtypes = [ctypes.c_int32, ctypes.c_int64, vp, vp, vp, ctypes.c_int32,
                                      ctypes.c_uint32, vp, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_double)]
        L.ising_halo_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
        L.ising_strerror.argtypes = [ctypes.c_int]
        L.ising_strerror.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("ising_destroy", "ising_strerror", "ising_batch_destroy"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().ising_strerror(code).decode()


def _check(code: int, what: str):
    if code != ISING_OK:
        raise IsingError(code, what)


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def _buffer(x, dtype, n: int | None, writable: bool):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor."""
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        import torch  # only when a tensor is passed
        want = {np.int8: torch.int8, np.int32: torch.int32, np.int64: torch.int64,
                np.uint8: torch.uint8, np.float32: torch.float32}[dtype]
        if x.dtype != want:
            raise TypeError(f"expected a {want} tensor")
        if not x.is_contiguous() or (n is not None and x.numel() != n):
            raise ValueError("tensor must be contiguous with the expected length")
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda), x
    a = np.asarray(x)
    if a.dtype != dtype or not a.flags.c_contiguous or (writable and not a.flags.writeable):
        if writable:
            raise TypeError(f"expected a writable contiguous {np.dtype(dtype).name} array")
        a = np.ascontiguousarray(a, dtype=dtype)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} elements, got {a.size}")
    return ctypes.c_void_p(a.ctypes.data), 0, a


class IsingGraph:
    """Owning wrapper of an ``ising_graph*`` handle (``ising_destroy`` on close)."""

    def __init__(self, ptr: int, n: int):
        self.ptr = ctypes.c_void_p(ptr)
        self.n = n

    def close(self):
        if self.ptr and self.ptr.value:
            lib().ising_destroy(self.ptr)
            self.ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def ising_create(n: int, src, dst, w, flags: int = 0, stream=None) -> IsingGraph:
    ps, _, ks = _buffer(src, np.int32, None, False)
    m = ks.size if hasattr(ks, "size") else ks.numel()
    pd, _, kd = _buffer(dst, np.int32, m, False)
    pw, _, kw = _buffer(w, np.int32, m, False)
    out = ctypes.c_void_p()
    _check(lib().ising_create(n, m, ps, pd, pw, flags, _stream(stream), ctypes.byref(out)),
           "ising_create")
    return IsingGraph(out.value, n)


def ising_anneal(g: IsingGraph, *, t_total: int, seed: int, p0: float = 0.0,
                 sweeps: int | None = None, mode: int = ISING_MODE_DET, t_begin: int = 0,
                 replica: int = 0, stream=None, kind: int = ISING_SCHED_LINEAR, n0: int = 0) -> None:
    """Linear schedule (kind=ISING_SCHED_LINEAR, p0) or Algorithm 1's N-flip
    schedule (kind=ISING_SCHED_NFLIP, n0)."""
    if sweeps is None:
        sweeps = t_total - t_begin
    sched = ising_schedule(kind, replica, p0, t_begin, t_total, n0, 0)
    _check(lib().ising_anneal(g.ptr, ctypes.byref(sched), sweeps, seed & (2 ** 64 - 1), mode,
                              _stream(stream)), "ising_anneal")


def ising_anneal_trace(g: IsingGraph, *, t_total: int, seed: int, every: int, p0: float = 0.0,
                       sweeps: int | None = None, mode: int = ISING_MODE_DET, t_begin: int = 0,
                       replica: int = 0, stream=None, kind: int = ISING_SCHED_LINEAR,
                       n0: int = 0) -> np.ndarray:
    """Energies after every ``every`` sweeps (int64 array)."""
    if sweeps is None:
        sweeps = t_total - t_begin
    sched = ising_schedule(kind, replica, p0, t_begin, t_total, n0, 0)
    out = np.zeros(max(0, -(-sweeps // every)) if every > 0 else 0, dtype=np.int64)
    _check(lib().ising_anneal_trace(g.ptr, ctypes.byref(sched), sweeps, seed & (2 ** 64 - 1), mode,
                                    every, out.ctypes.data, _stream(stream)), "ising_anneal_trace")
    return out


def ising_convergence_region(g: IsingGraph, *, seeds, p0: float, t_total: int, every: int,
                             sweeps: int | None = None, t_begin: int = 0, replica: int = 0,
                             mode: int = ISING_MODE_DET, stream=None):
    """The Fig. 4 view, computed by the library (include/ising.h): returns
    (sweep reached after each chunk, cuts[seed, chunk], min over seeds, max
    over seeds). Row 0 of cuts is the one-run curve."""
    if sweeps is None:
        sweeps = t_total - t_begin
    sd = np.ascontiguousarray([int(x) & (2 ** 64 - 1) for x in seeds], dtype=np.uint64)
    points = -(-sweeps // every) if every > 0 else 0
    cuts = np.zeros((sd.size, points), dtype=np.int64)
    lo = np.zeros(points, dtype=np.int64)
    hi = np.zeros(points, dtype=np.int64)
    sched = ising_schedule(ISING_SCHED_LINEAR, replica, p0, t_begin, t_total, 0, 0)
    _check(lib().ising_convergence_region(g.ptr, ctypes.byref(sched), sweeps, sd.ctypes.data, sd.size,
                                          mode, every, cuts.ctypes.data, lo.ctypes.data, hi.ctypes.data,
                                          _stream(stream)), "ising_convergence_region")
    idx = t_begin + np.minimum(np.arange(1, points + 1) * every, sweeps)
    return idx, cuts, lo, hi


def ising_energy(g: IsingGraph) -> int:
    v = ctypes.c_int64()
    _check(lib().ising_energy(g.ptr, ctypes.byref(v)), "ising_energy")
    return v.value


def ising_cut(g: IsingGraph) -> int:
    v = ctypes.c_int64()
    _check(lib().ising_cut(g.ptr, ctypes.byref(v)), "ising_cut")
    return v.value


def ising_total_weight(g: IsingGraph) -> int:
    v = ctypes.c_int64()
    _check(lib().ising_total_weight(g.ptr, ctypes.byref(v)), "ising_total_weight")
    return v.value


def ising_num_edges(g: IsingGraph) -> int:
    v = ctypes.c_int64()
    _check(lib().ising_num_edges(g.ptr, ctypes.byref(v)), "ising_num_edges")
    return v.value


def ising_get_spins(g: IsingGraph, out=None):
    """Spins in caller order; into ``out`` (numpy int8 or torch int8 tensor) if
    given, else a new numpy array."""
    if out is None:
        out = np.empty(g.n, dtype=np.int8)
    p, on_dev, keep = _buffer(out, np.int8, g.n, True)
    _check(lib().ising_get_spins(g.ptr, p, on_dev), "ising_get_spins")
    return out


def ising_set_spins(g: IsingGraph, spins) -> None:
    p, on_dev, keep = _buffer(spins, np.int8, g.n, False)
    _check(lib().ising_set_spins(g.ptr, p, on_dev), "ising_set_spins")


def ising_init_random(g: IsingGraph, seed: int, replica: int = 0) -> None:
    _check(lib().ising_init_random(g.ptr, seed & (2 ** 64 - 1), replica), "ising_init_random")


def ising_num_colours(g: IsingGraph) -> int:
    v = ctypes.c_int32()
    _check(lib().ising_num_colours(g.ptr, ctypes.byref(v)), "ising_num_colours")
    return v.value


def ising_colouring(g: IsingGraph) -> np.ndarray:
    out = np.empty(g.n, dtype=np.int32)
    _check(lib().ising_colouring(g.ptr, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
           "ising_colouring")
    return out


def ising_plan_colouring(n: int, src, dst, w):
    """Host-only: (number of colours, colour per vertex) that ising_create would
    use for this edge list. Needs no GPU."""
    ps, _, ks = _buffer(src, np.int32, None, False)
    m = ks.size
    pd, _, kd = _buffer(dst, np.int32, m, False)
    pw, _, kw = _buffer(w, np.int32, m, False)
    out = np.empty(max(n, 0), dtype=np.int32)
    C = ctypes.c_int32()
    _check(lib().ising_plan_colouring(n, m, ps, pd, pw,
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      ctypes.byref(C)), "ising_plan_colouring")
    return C.value, out


def ising_engine_used(g: IsingGraph) -> int:
    """The engine the last anneal call ran (ISING_ENGINE_*, or ISING_ENGINE_USED_BLOCK)."""
    v = ctypes.c_int32()
    _check(lib().ising_engine_used(g.ptr, ctypes.byref(v)), "ising_engine_used")
    return v.value


def ising_debug_fault(g: IsingGraph, kind: int, wait_budget_ns: int = 0) -> None:
    """Failure-detection test hook (see include/ising.h)."""
    _check(lib().ising_debug_fault(g.ptr, kind, wait_budget_ns), "ising_debug_fault")


def ising_set_engine(g: IsingGraph, engine: int) -> None:
    _check(lib().ising_set_engine(g.ptr, engine), "ising_set_engine")


def ising_set_halo_sweeps(g: IsingGraph, sweeps_per_exchange: int) -> None:
    """Sweeps per exchange of the halo engine (0: automatic)."""
    _check(lib().ising_set_halo_sweeps(g.ptr, sweeps_per_exchange), "ising_set_halo_sweeps")


def ising_plan_halo(n: int, src, dst, w, parts: int, sweeps_per_exchange: int):
    """Host only: (part of every vertex, plan dict or None if the graph does not
    qualify) -- the halo engine's partition and plan without a device."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.int32)
    out = np.empty(max(n, 1), np.int32)
    smem, ratio = ctypes.c_int32(), ctypes.c_double()
    rc = lib().ising_plan_halo(n, src.size, src.ctypes.data, dst.ctypes.data, w.ctypes.data, parts,
                               sweeps_per_exchange, out.ctypes.data, ctypes.byref(smem), ctypes.byref(ratio))
    if rc == ISING_ESTATE:
        return out[:n], None
    _check(rc, "ising_plan_halo")
    return out[:n], {"smem_bytes": smem.value, "work_ratio": ratio.value}


def ising_halo_info(g: IsingGraph) -> dict | None:
    """The halo engine's plan (parts, sweeps per exchange, shared memory per
    block, largest work ratio), or None if the graph does not qualify."""
    parts, sweeps, smem = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    ratio = ctypes.c_double()
    rc = lib().ising_halo_info(g.ptr, ctypes.byref(parts), ctypes.byref(sweeps), ctypes.byref(smem),
                               ctypes.byref(ratio))
    if rc == ISING_ESTATE:
        return None
    _check(rc, "ising_halo_info")
    return {"parts": parts.value, "sweeps_per_exchange": sweeps.value, "smem_bytes": smem.value,
            "work_ratio": ratio.value}


def ising_energy_csr_static(n: int, row_ptr, col, w, spins, out, stream=None) -> None:
    """Energy and cut of ``spins`` on a caller-owned device CSR graph into the
    device int64[2] ``out``, allocating nothing (see include/ising.h). All
    arguments are torch CUDA tensors on the current device: row_ptr int32[n+1],
    col and w int32 of equal length, spins int8[n], out int64[2]. Lengths are
    checked here because the kernels cannot check them."""
    if int(n) <= 0:
        raise ValueError("n must be positive")
    lengths = {"row_ptr": (row_ptr, n + 1), "spins": (spins, n), "out": (out, 2)}
    for name, (t, want) in lengths.items():
        if not hasattr(t, "numel") or t.numel() != want:
            raise ValueError(f"{name} must have {want} elements")
    if not hasattr(col, "numel") or not hasattr(w, "numel") or col.numel() != w.numel():
        raise ValueError("col and w must have the same length")

    def ptr(t, dtype):
        p, on_dev, _ = _buffer(t, dtype, None, False)
        if not on_dev:
            raise TypeError("ising_energy_csr_static takes device tensors")
        return p
    ptrs = [ptr(row_ptr, np.int32), ptr(col, np.int32), ptr(w, np.int32), ptr(spins, np.int8),
            ptr(out, np.int64)]
    import torch  # device tensors imply torch
    dev = torch.cuda.current_device()
    for t in (row_ptr, col, w, spins, out):
        if t.device.index != dev:
            raise ValueError("every tensor must be on the current CUDA device")
    _check(lib().ising_energy_csr_static(n, *ptrs, _stream(stream)), "ising_energy_csr_static")


def ising_launch_count(g: IsingGraph) -> int:
    v = ctypes.c_uint64()
    _check(lib().ising_launch_count(g.ptr, ctypes.byref(v)), "ising_launch_count")
    return v.value


def ising_destroy(g: IsingGraph) -> None:
    g.close()


# ---------------------------------------------------------------------------
# batched instances
# ---------------------------------------------------------------------------
class IsingBatch:
    """Owning wrapper of an ``ising_batch*`` handle."""

    def __init__(self, ptr: int, ns, replicas: int):
        self.ptr = ctypes.c_void_p(ptr)
        self.n = [int(x) for x in ns]
        self.replicas = replicas

    def close(self):
        if self.ptr and self.ptr.value:
            lib().ising_batch_destroy(self.ptr)
            self.ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def ising_batch_create(graphs, replicas: int = 8, stream=None) -> IsingBatch:
    """``graphs``: sequence of (n, src, dst, w) host arrays."""
    ns = np.array([g[0] for g in graphs], dtype=np.int32)
    srcs = [np.ascontiguousarray(g[1], dtype=np.int32) for g in graphs]
    ms = np.array([s.size for s in srcs], dtype=np.int64)
    src = np.ascontiguousarray(np.concatenate(srcs) if srcs else np.zeros(0), dtype=np.int32)
    dst = np.ascontiguousarray(np.concatenate([np.asarray(g[2], dtype=np.int32) for g in graphs]), dtype=np.int32)
    w = np.ascontiguousarray(np.concatenate([np.asarray(g[3], dtype=np.int32) for g in graphs]), dtype=np.int32)
    out = ctypes.c_void_p()
    _check(lib().ising_batch_create(len(graphs), ns.ctypes.data, ms.ctypes.data, src.ctypes.data,
                                    dst.ctypes.data, w.ctypes.data, replicas, _stream(stream),
                                    ctypes.byref(out)), "ising_batch_create")
    return IsingBatch(out.value, ns, replicas)


def ising_batch_init_random(b: IsingBatch, seed: int) -> None:
    _check(lib().ising_batch_init_random(b.ptr, seed & (2 ** 64 - 1)), "ising_batch_init_random")


def ising_batch_anneal(b: IsingBatch, *, p0: float, t_total: int, seed: int, sweeps: int | None = None,
                       t_begin: int = 0, stream=None) -> None:
    if sweeps is None:
        sweeps = t_total - t_begin
    sched = ising_schedule(ISING_SCHED_LINEAR, 0, p0, t_begin, t_total, 0, 0)
    _check(lib().ising_batch_anneal(b.ptr, ctypes.byref(sched), sweeps, seed & (2 ** 64 - 1),
                                    _stream(stream)), "ising_batch_anneal")


def ising_batch_cuts(b: IsingBatch) -> np.ndarray:
    """int64 array [num_graphs, replicas]."""
    out = np.zeros((len(b.n), b.replicas), dtype=np.int64)
    _check(lib().ising_batch_cuts(b.ptr, out.ctypes.data), "ising_batch_cuts")
    return out


def ising_batch_get_spins(b: IsingBatch, graph: int, replica: int) -> np.ndarray:
    out = np.empty(b.n[graph], dtype=np.int8)
    _check(lib().ising_batch_get_spins(b.ptr, graph, replica, out.ctypes.data), "ising_batch_get_spins")
    return out


def ising_batch_set_spins(b: IsingBatch, graph: int, replica: int, spins) -> None:
    s = np.ascontiguousarray(spins, dtype=np.int8)
    if s.size != b.n[graph]:
        raise ValueError("wrong length")
    _check(lib().ising_batch_set_spins(b.ptr, graph, replica, s.ctypes.data), "ising_batch_set_spins")


def ising_batch_autotune(b: IsingBatch, probe_sweeps: int = 20) -> int:
    v = ctypes.c_int32()
    _check(lib().ising_batch_autotune(b.ptr, probe_sweeps, ctypes.byref(v)), "ising_batch_autotune")
    return v.value


def ising_batch_set_block(b: IsingBatch, block: int) -> None:
    _check(lib().ising_batch_set_block(b.ptr, block), "ising_batch_set_block")


def ising_batch_set_tuning(b: IsingBatch, block: int, row_split: int, tail: int) -> None:
    _check(lib().ising_batch_set_tuning(b.ptr, block, row_split, tail), "ising_batch_set_tuning")


def ising_batch_tuning(b: IsingBatch) -> dict:
    """The configuration in use and the last autotune's 18 probe times (ms),
    indexed 6 * block_index + 2 * split_index + tail_index."""
    blk, split, tail = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    probe = np.zeros(18, dtype=np.float32)
    _check(lib().ising_batch_tuning(b.ptr, ctypes.byref(blk), ctypes.byref(split), ctypes.byref(tail),
                                    probe.ctypes.data), "ising_batch_tuning")
    return {"block": blk.value, "row_split": split.value, "tail": tail.value, "probe_ms": probe.tolist()}


def ising_batch_info(b: IsingBatch) -> dict:
    g = ctypes.c_int32(); v = ctypes.c_int64(); blk = ctypes.c_int32(); la = ctypes.c_uint64()
    _check(lib().ising_batch_info(b.ptr, ctypes.byref(g), ctypes.byref(v), ctypes.byref(blk),
                                  ctypes.byref(la)), "ising_batch_info")
    return {"num_graphs": g.value, "vertices": v.value, "block": blk.value, "launches": la.value}


def ising_batch_destroy(b: IsingBatch) -> None:
    b.close()


# ---------------------------------------------------------------------------
# flip bias and the learned warm start
# ---------------------------------------------------------------------------
def ising_set_flip_bias(g: IsingGraph, q) -> None:
    """Per-vertex flip bias q (uint8, caller order), or None to remove it."""
    if q is None:
        _check(lib().ising_set_flip_bias(g.ptr, None, 0), "ising_set_flip_bias")
        return
    p, on_dev, _keep = _buffer(q, np.uint8, g.n, False)
    _check(lib().ising_set_flip_bias(g.ptr, p, on_dev), "ising_set_flip_bias")


def ising_get_flip_bias(g: IsingGraph) -> np.ndarray:
    out = np.zeros(g.n, dtype=np.uint8)
    _check(lib().ising_get_flip_bias(g.ptr, out.ctypes.data), "ising_get_flip_bias")
    return out


class IsingGnn:
    """Owning wrapper of an ``ising_gnn*`` handle."""

    def __init__(self, ptr: int):
        self.ptr = ctypes.c_void_p(ptr)

    def close(self):
        if self.ptr and self.ptr.value:
            lib().ising_gnn_destroy(self.ptr)
            self.ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _params(params) -> np.ndarray:
    a = np.ascontiguousarray(params, dtype=np.float32)
    if a.shape != (ISING_GNN_NUM_PARAMS,):
        raise ValueError(f"expected {ISING_GNN_NUM_PARAMS} parameters")
    return a


def ising_gnn_create(params) -> IsingGnn:
    a = _params(params)
    out = ctypes.c_void_p()
    _check(lib().ising_gnn_create(a.ctypes.data, ctypes.byref(out)), "ising_gnn_create")
    return IsingGnn(out.value)


def ising_gnn_set_params(net: IsingGnn, params) -> None:
    a = _params(params)
    _check(lib().ising_gnn_set_params(net.ptr, a.ctypes.data), "ising_gnn_set_params")


def ising_gnn_get_params(net: IsingGnn) -> np.ndarray:
    out = np.zeros(ISING_GNN_NUM_PARAMS, dtype=np.float32)
    _check(lib().ising_gnn_get_params(net.ptr, out.ctypes.data), "ising_gnn_get_params")
    return out


def ising_gnn_forward(net: IsingGnn, g: IsingGraph, out=None):
    """Logits in the caller's vertex order (numpy float32, or into ``out``,
    a float32 numpy array or CUDA tensor of n elements)."""
    if out is None:
        out = np.zeros(g.n, dtype=np.float32)
    p, on_dev, _keep = _buffer(out, np.float32, g.n, True)
    _check(lib().ising_gnn_forward(net.ptr, g.ptr, p, on_dev), "ising_gnn_forward")
    return out


def ising_gnn_gradients(net: IsingGnn, g: IsingGraph, labels):
    """(loss, gradient) for int8 +-1 labels in the caller's order."""
    p, on_dev, _keep = _buffer(labels, np.int8, g.n, False)
    loss = ctypes.c_float()
    grad = np.zeros(ISING_GNN_NUM_PARAMS, dtype=np.float32)
    _check(lib().ising_gnn_gradients(net.ptr, g.ptr, p, on_dev, ctypes.byref(loss), grad.ctypes.data),
           "ising_gnn_gradients")
    return float(loss.value), grad


def ising_gnn_train_step(net: IsingGnn, g: IsingGraph, labels, lr: float, want_loss: bool = False):
    """One Adam step on the loss against ``labels``; returns the loss (before
    the step) if ``want_loss``, else None without synchronising."""
    p, on_dev, _keep = _buffer(labels, np.int8, g.n, False)
    loss = ctypes.c_float()
    _check(lib().ising_gnn_train_step(net.ptr, g.ptr, p, on_dev, float(lr),
                                      ctypes.byref(loss) if want_loss else None),
           "ising_gnn_train_step")
    return float(loss.value) if want_loss else None


def ising_gnn_warm_start(net: IsingGnn, g: IsingGraph, set_bias: bool = True) -> None:
    _check(lib().ising_gnn_warm_start(net.ptr, g.ptr, int(bool(set_bias))), "ising_gnn_warm_start")


def ising_gnn_batch_forward(net: IsingGnn, b: IsingBatch, replica: int = 0, out=None):
    """Logits of every instance of the batch from one replica's spins,
    instance by instance in batch order, each by vertex id (numpy float32, or
    into ``out``, a float32 numpy array or CUDA tensor)."""
    total = ising_batch_info(b)["vertices"]
    if out is None:
        out = np.zeros(total, dtype=np.float32)
    p, on_dev, _keep = _buffer(out, np.float32, total, True)
    _check(lib().ising_gnn_batch_forward(net.ptr, b.ptr, replica, p, on_dev), "ising_gnn_batch_forward")
    return out


def ising_gnn_batch_warm_start(net: IsingGnn, b: IsingBatch, replica: int = ISING_ALL_REPLICAS) -> None:
    _check(lib().ising_gnn_batch_warm_start(net.ptr, b.ptr, replica), "ising_gnn_batch_warm_start")


def ising_gnn_batch_gradients(net: IsingGnn, b: IsingBatch, labels, replica: int = 0):
    """(loss, gradient) over every instance of the batch; int8 +-1 labels laid
    out as the logits of ising_gnn_batch_forward."""
    total = ising_batch_info(b)["vertices"]
    p, on_dev, _keep = _buffer(labels, np.int8, total, False)
    loss = ctypes.c_float()
    grad = np.zeros(ISING_GNN_NUM_PARAMS, dtype=np.float32)
    _check(lib().ising_gnn_batch_gradients(net.ptr, b.ptr, replica, p, on_dev, ctypes.byref(loss),
                                           grad.ctypes.data), "ising_gnn_batch_gradients")
    return float(loss.value), grad


def ising_gnn_batch_train_step(net: IsingGnn, b: IsingBatch, labels, lr: float, replica: int = 0,
                               want_loss: bool = False):
    """One Adam step on the batch's instances as one minibatch; returns the
    loss (before the step) if ``want_loss``."""
    total = ising_batch_info(b)["vertices"]
    p, on_dev, _keep = _buffer(labels, np.int8, total, False)
    loss = ctypes.c_float()
    _check(lib().ising_gnn_batch_train_step(net.ptr, b.ptr, replica, p, on_dev, float(lr),
                                            ctypes.byref(loss) if want_loss else None),
           "ising_gnn_batch_train_step")
    return float(loss.value) if want_loss else None


def ising_gnn_set_dense_path(net: IsingGnn, path: int) -> None:
    """ISING_GNN_DENSE_MMA_SYNC (default) or ISING_GNN_DENSE_TCGEN05 for the
    forward layers' products."""
    _check(lib().ising_gnn_set_dense_path(net.ptr, int(path)), "ising_gnn_set_dense_path")


def ising_gnn_launch_count(net: IsingGnn) -> int:
    v = ctypes.c_uint64()
    _check(lib().ising_gnn_launch_count(net.ptr, ctypes.byref(v)), "ising_gnn_launch_count")
    return v.value


def ising_gnn_destroy(net: IsingGnn) -> None:
    net.close()
