"""Python binding of libbitssa, the sm_103a bit-sliced Gillespie library.

A thin ctypes layer over the C ABI in ``include/bitssa.h``: the functions here
have the same names as the C entry points and only marshal arguments; every
step of the simulation runs in the library's CUDA kernels.  PyTorch supplies
device memory (its caching allocator, through ``ssa_set_allocator``) and
streams.  There is no CPU fallback: importing works without a GPU, but any
call that needs the library raises if ``libbitssa.so`` is missing or if no
CUDA device is present.

Method: Castellana & Lacoste, "Parallelization of Gillespie algorithm based on
binary words" (arXiv 2412.16613).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbitssa.so")

SSA_OK, SSA_EINVAL, SSA_EUNSUPPORTED, SSA_ENOMEM = 0, -1, -2, -3
SSA_ECUDA, SSA_ETIMEOUT, SSA_EOVERFLOW, SSA_ESTATE = -4, -5, -6, -7
SSA_P64, SSA_P32_KAHAN, SSA_P32_D64ACC, SSA_P64_LOGSUM, SSA_P32_PLAIN = 0, 1, 2, 3, 4
SSA_ENGINE_BITSLICED, SSA_ENGINE_THREAD_PER_RUN, SSA_ENGINE_GENERAL = 0, 1, 2
SSA_LAYOUT_AUTO, SSA_LAYOUT_THREAD, SSA_LAYOUT_WARPS = 0, 1, 2
SSA_CLOCK_GROUP, SSA_CLOCK_LANE = 0, 1
SSA_FIELD_FINAL_COUNTS, SSA_FIELD_ABSORB_TIME, SSA_FIELD_ABSORB_OUTCOME = 0, 1, 2
SSA_FIELD_EE_HIST, SSA_FIELD_SNAP_COUNTS, SSA_FIELD_COUNTERS, SSA_FIELD_ENS_ABSORBED = 3, 4, 5, 6
SSA_N_COUNTERS = 10
COUNTER_NAMES = ["group_steps", "lane_steps", "reactions", "null_lane_steps", "redraw_rounds",
                 "absorbed", "groups_done", "error_flags", "max_group_steps", "layout"]

SSA_LAT_FINAL_COUNTS, SSA_LAT_HOMOCHIRAL_TIME, SSA_LAT_OUTCOME, SSA_LAT_EVENTS = 0, 1, 2, 3
SSA_LAT_SNAP_TOTALS, SSA_LAT_SNAP_DOMAINS, SSA_LAT_GROUPS, SSA_LAT_COUNTERS = 4, 5, 6, 7
SSA_LAT_N_COUNTERS = 8
LAT_COUNTER_NAMES = ["group_steps", "rounds", "clock_rounds", "reactions", "hops", "cap_raises", "group_errors",
                     "flagged"]
_LAT_FIELD_DTYPE = {
    SSA_LAT_FINAL_COUNTS: np.int32, SSA_LAT_HOMOCHIRAL_TIME: np.float64, SSA_LAT_OUTCOME: np.int8,
    SSA_LAT_EVENTS: np.int64, SSA_LAT_SNAP_TOTALS: np.int64, SSA_LAT_SNAP_DOMAINS: np.int32,
    SSA_LAT_GROUPS: np.int64, SSA_LAT_COUNTERS: np.uint64,
}

_FIELD_DTYPE = {
    SSA_FIELD_FINAL_COUNTS: np.int32, SSA_FIELD_ABSORB_TIME: np.float64,
    SSA_FIELD_ABSORB_OUTCOME: np.int8, SSA_FIELD_EE_HIST: np.uint64,
    SSA_FIELD_SNAP_COUNTS: np.int32, SSA_FIELD_COUNTERS: np.uint64,
    SSA_FIELD_ENS_ABSORBED: np.uint64,
}


class SSAError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"libbitssa status {status}: {message}")
        self.status = status


class ssa_options(C.Structure):
    _fields_ = [
        ("precision", C.c_int32), ("engine", C.c_int32), ("block_size", C.c_int32),
        ("blocks_per_sm", C.c_int32), ("thin_bits", C.c_int32), ("keep_snap_counts", C.c_int32),
        ("step_budget", C.c_int64), ("first_run", C.c_int64), ("cuda_stream", C.c_void_p),
        ("device", C.c_int32), ("layout", C.c_int32), ("shared_n", C.c_int32), ("pad_pow2", C.c_int32),
        ("recompute", C.c_int32), ("clock", C.c_int32), ("word_width", C.c_int32), ("tail_groups", C.c_int32),
        ("reserved", C.c_int32 * 3),
    ]


_lock = threading.Lock()
_lib = None
_alloc_refs = None

_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_int, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_int, C.c_void_p, C.c_void_p)


def build(force: bool = False) -> str:
    """Compile libbitssa.so (nvcc, sm_103a) in the package directory."""
    from . import _build
    return _build.build(force=force)


def lib():
    """The loaded libbitssa; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libbitssa.so is not built ({LIB_PATH}); run "
                                  "paper_2412_16613_gb300.build() first")
            L = C.CDLL(LIB_PATH)
            P = C.POINTER
            L.ssa_default_options.argtypes = [P(ssa_options)]
            L.ssa_default_options.restype = None
            L.ssa_create.argtypes = [P(C.c_int32), P(C.c_int32), C.c_int32, C.c_int32, P(C.c_double),
                                     P(C.c_int64), C.c_int32, C.c_int64, C.c_uint64, P(ssa_options),
                                     P(C.c_void_p)]
            L.ssa_create_batch.argtypes = [P(C.c_int32), P(C.c_int32), C.c_int32, C.c_int32, C.c_int32,
                                           P(C.c_int64), P(C.c_double), P(C.c_int64), P(C.c_uint64),
                                           P(ssa_options), P(C.c_void_p)]
            L.ssa_run.argtypes = [C.c_void_p, C.c_double, P(C.c_double), C.c_int32]
            L.ssa_tune.argtypes = [C.c_void_p, C.c_double, P(C.c_double), C.c_int32, C.c_int64, P(C.c_int32)]
            L.ssa_field_bytes.argtypes = [C.c_void_p, C.c_int32, P(C.c_size_t)]
            L.ssa_fetch.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t, C.c_int32]
            L.ssa_destroy.argtypes = [C.c_void_p]
            L.ssa_last_error.argtypes = [C.c_void_p]
            L.ssa_last_error.restype = C.c_char_p
            L.ssa_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, C.c_void_p]
            L.ssa_version.restype = C.c_int
            L.ssa_run_frank_noalloc.argtypes = [P(C.c_int64), P(C.c_double), C.c_int64, C.c_uint64,
                                                C.c_int32, C.c_double, P(C.c_double), C.c_int32,
                                                C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                                C.c_void_p, P(C.c_uint64), C.c_void_p]
            L.ssa_lattice_create.argtypes = [C.c_int32, C.c_int32, P(C.c_double), C.c_double, P(C.c_int64),
                                             C.c_int32, C.c_int64, C.c_uint64, P(ssa_options), C.c_int32,
                                             P(C.c_void_p)]
            L.ssa_lattice_run.argtypes = [C.c_void_p, C.c_double, P(C.c_double), C.c_int32]
            L.ssa_lattice_field_bytes.argtypes = [C.c_void_p, C.c_int32, P(C.c_size_t)]
            L.ssa_lattice_fetch.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t, C.c_int32]
            L.ssa_lattice_destroy.argtypes = [C.c_void_p]
            L.ssa_lattice_last_error.argtypes = [C.c_void_p]
            L.ssa_lattice_last_error.restype = C.c_char_p
            L.bitssa_test_philox.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32), C.c_int64, C.c_int32]
            L.bitssa_test_bitslice.argtypes = [C.c_int32, P(C.c_int64), P(C.c_int64), P(C.c_int64), C.c_int64]
            L.bitssa_bench_alu.argtypes = [C.c_int32, C.c_int32, P(C.c_double), P(C.c_double)]
            _lib = L
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _check(status, ctx=None):
    if status != SSA_OK:
        msg = lib().ssa_last_error(ctx)
        raise SSAError(status, msg.decode() if msg else "")
    return status


def ssa_default_options(**kw) -> ssa_options:
    """ssa_options with the library defaults, then the given fields."""
    o = ssa_options()
    lib().ssa_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "cuda_stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream  # a torch.cuda.Stream
        setattr(o, k, v)
    return o


def ssa_set_allocator(alloc=None, release=None, user=None):
    """Route device allocations through Python callables (None, None: cudaMalloc)."""
    global _alloc_refs
    if alloc is None:
        _alloc_refs = None
        return _check(lib().ssa_set_allocator(_ALLOC_FN(), _FREE_FN(), None))
    fa, ff = _ALLOC_FN(alloc), _FREE_FN(release)
    _alloc_refs = (fa, ff)
    return _check(lib().ssa_set_allocator(fa, ff, user))


def use_torch_allocator():
    """Let libbitssa take device memory from PyTorch's caching allocator."""
    import torch

    def alloc(nbytes, device, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=int(device),
                                                      stream=stream or 0)
        except Exception:
            return None

    def release(ptr, nbytes, device, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    return ssa_set_allocator(alloc, release)


def ssa_create(reactants, products, rates, N0, n_runs, seed, options=None):
    """C ssa_create.  N0: [S] shared or [n_runs][S] per run.  Returns the context handle."""
    reac = np.ascontiguousarray(reactants, dtype=np.int32)
    prod = np.ascontiguousarray(products, dtype=np.int32)
    k = np.ascontiguousarray(rates, dtype=np.float64)
    n0 = np.ascontiguousarray(N0, dtype=np.int64)
    R, S = reac.shape
    ctx = C.c_void_p()
    opt = options if options is not None else ssa_default_options()
    st = lib().ssa_create(_p(reac, C.c_int32), _p(prod, C.c_int32), S, R, _p(k, C.c_double),
                          _p(n0, C.c_int64), 1 if n0.ndim == 2 else 0, int(n_runs),
                          int(seed) & (2**64 - 1), C.byref(opt), C.byref(ctx))
    _check(st)
    return ctx


def ssa_create_batch(reactants, products, N0_ens, rates_ens, runs_ens, seed_ens, options=None):
    reac = np.ascontiguousarray(reactants, dtype=np.int32)
    prod = np.ascontiguousarray(products, dtype=np.int32)
    n0 = np.ascontiguousarray(N0_ens, dtype=np.int64)
    k = np.ascontiguousarray(rates_ens, dtype=np.float64)
    runs = np.ascontiguousarray(runs_ens, dtype=np.int64)
    seeds = np.ascontiguousarray(np.asarray(seed_ens, dtype=np.uint64))
    R, S = reac.shape
    ctx = C.c_void_p()
    opt = options if options is not None else ssa_default_options()
    st = lib().ssa_create_batch(_p(reac, C.c_int32), _p(prod, C.c_int32), S, R, len(runs),
                                _p(n0, C.c_int64), _p(k, C.c_double), _p(runs, C.c_int64),
                                _p(seeds, C.c_uint64), C.byref(opt), C.byref(ctx))
    _check(st)
    return ctx


def ssa_run(ctx, t_end, snapshot_times=()):
    snaps = np.ascontiguousarray(snapshot_times, dtype=np.float64)
    ptr = _p(snaps, C.c_double) if len(snaps) else None
    return _check(lib().ssa_run(ctx, float(t_end), ptr, len(snaps)), ctx)


def ssa_tune(ctx, t_end, snapshot_times=(), probe_steps=0):
    """C ssa_tune: time every launch configuration on this workload and keep the fastest for
    later runs; returns (layout, block size of the one-thread layout)."""
    snaps = np.ascontiguousarray(snapshot_times, dtype=np.float64)
    ptr = _p(snaps, C.c_double) if len(snaps) else None
    choice = np.zeros(2, dtype=np.int32)
    _check(lib().ssa_tune(ctx, float(t_end), ptr, len(snaps), int(probe_steps), _p(choice, C.c_int32)), ctx)
    return int(choice[0]), int(choice[1])


def ssa_field_bytes(ctx, field):
    n = C.c_size_t()
    _check(lib().ssa_field_bytes(ctx, field, C.byref(n)), ctx)
    return n.value


def ssa_fetch(ctx, field, out=None):
    """Copy a field into `out` (numpy array, or a CUDA torch tensor) or a new numpy array."""
    nbytes = ssa_field_bytes(ctx, field)
    if out is None:
        out = np.empty(nbytes // np.dtype(_FIELD_DTYPE[field]).itemsize, dtype=_FIELD_DTYPE[field])
    if isinstance(out, np.ndarray):
        assert out.flags.c_contiguous and out.nbytes >= nbytes
        _check(lib().ssa_fetch(ctx, field, out.ctypes.data, out.nbytes, 0), ctx)
    else:  # torch tensor on the context's device
        assert out.is_contiguous() and out.is_cuda
        _check(lib().ssa_fetch(ctx, field, out.data_ptr(), out.numel() * out.element_size(), 1), ctx)
    return out


def ssa_run_frank_noalloc(N0, rates, n_runs, seed, t_end, snapshot_times, final_counts, t_abs, outcome,
                          ee_hist=None, precision=SSA_P64, thin_bits=32, stream=None):
    """C ssa_run_frank_noalloc: outputs are CUDA torch tensors (or raw device pointers)
    that the caller owns; the library allocates nothing.  Returns the counters."""
    n0 = np.ascontiguousarray(N0, dtype=np.int64)
    k = np.ascontiguousarray(rates, dtype=np.float64)
    snaps = np.ascontiguousarray(snapshot_times, dtype=np.float64)
    counters = np.zeros(SSA_N_COUNTERS, dtype=np.uint64)

    def ptr(x):
        return None if x is None else (x if isinstance(x, int) else x.data_ptr())

    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    st = lib().ssa_run_frank_noalloc(_p(n0, C.c_int64), _p(k, C.c_double), int(n_runs),
                                     int(seed) & (2**64 - 1), int(thin_bits), float(t_end),
                                     _p(snaps, C.c_double) if len(snaps) else None, len(snaps),
                                     int(precision), ptr(final_counts), ptr(t_abs), ptr(outcome),
                                     ptr(ee_hist), _p(counters, C.c_uint64), stream)
    _check(st)
    return dict(zip(COUNTER_NAMES, counters.tolist()))


def ssa_destroy(ctx):
    return _check(lib().ssa_destroy(ctx))


def ssa_last_error(ctx=None):
    m = lib().ssa_last_error(ctx)
    return m.decode() if m else ""


def ssa_version():
    return lib().ssa_version()


# --------------------------------------------------------------------------
# Frank's model on a periodic lattice (ssa_lattice_* in include/bitssa.h)
# --------------------------------------------------------------------------
def _lat_check(status, ctx=None):
    if status != SSA_OK:
        msg = lib().ssa_lattice_last_error(ctx)
        raise SSAError(status, msg.decode() if msg else "")
    return status


def ssa_lattice_create(lx, ly, rates, hop, N0, n_runs, seed, options=None, cap_bits_max=0):
    """C ssa_lattice_create.  N0: [M][3] counts per site shared by every run, or [n_runs][M][3]."""
    k = np.ascontiguousarray(rates, dtype=np.float64)
    n0 = np.ascontiguousarray(N0, dtype=np.int64)
    ctx = C.c_void_p()
    opt = options if options is not None else ssa_default_options()
    st = lib().ssa_lattice_create(int(lx), int(ly), _p(k, C.c_double), float(hop), _p(n0, C.c_int64),
                                  1 if n0.ndim == 3 else 0, int(n_runs), int(seed) & (2**64 - 1), C.byref(opt),
                                  int(cap_bits_max), C.byref(ctx))
    _lat_check(st)
    return ctx


def ssa_lattice_run(ctx, t_end, snapshot_times=()):
    snaps = np.ascontiguousarray(snapshot_times, dtype=np.float64)
    ptr = _p(snaps, C.c_double) if len(snaps) else None
    return _lat_check(lib().ssa_lattice_run(ctx, float(t_end), ptr, len(snaps)), ctx)


def ssa_lattice_field_bytes(ctx, field):
    n = C.c_size_t()
    _lat_check(lib().ssa_lattice_field_bytes(ctx, field, C.byref(n)), ctx)
    return n.value


def ssa_lattice_fetch(ctx, field, out=None):
    """Copy a lattice field into `out` (numpy array, or a CUDA torch tensor) or a new numpy array."""
    nbytes = ssa_lattice_field_bytes(ctx, field)
    if out is None:
        out = np.empty(nbytes // np.dtype(_LAT_FIELD_DTYPE[field]).itemsize, dtype=_LAT_FIELD_DTYPE[field])
    if isinstance(out, np.ndarray):
        assert out.flags.c_contiguous and out.nbytes >= nbytes
        _lat_check(lib().ssa_lattice_fetch(ctx, field, out.ctypes.data, out.nbytes, 0), ctx)
    else:
        assert out.is_contiguous() and out.is_cuda
        _lat_check(lib().ssa_lattice_fetch(ctx, field, out.data_ptr(), out.numel() * out.element_size(), 1), ctx)
    return out


def ssa_lattice_destroy(ctx):
    return _lat_check(lib().ssa_lattice_destroy(ctx))


def ssa_lattice_last_error(ctx=None):
    m = lib().ssa_lattice_last_error(ctx)
    return m.decode() if m else ""


def lattice_fetch_all(ctx, M, n_snap=0):
    """Every lattice field as numpy arrays (per-run arrays in run order)."""
    out = {
        "final_counts": ssa_lattice_fetch(ctx, SSA_LAT_FINAL_COUNTS).reshape(-1, M, 3),
        "t_homochiral": ssa_lattice_fetch(ctx, SSA_LAT_HOMOCHIRAL_TIME),
        "outcome": ssa_lattice_fetch(ctx, SSA_LAT_OUTCOME),
        "events": ssa_lattice_fetch(ctx, SSA_LAT_EVENTS).reshape(-1, 2),
        "groups": ssa_lattice_fetch(ctx, SSA_LAT_GROUPS).reshape(-1, 3),
        "counters": dict(zip(LAT_COUNTER_NAMES, ssa_lattice_fetch(ctx, SSA_LAT_COUNTERS).tolist())),
    }
    if n_snap:
        out["snap_totals"] = ssa_lattice_fetch(ctx, SSA_LAT_SNAP_TOTALS).reshape(n_snap, -1, 3)
        out["snap_domains"] = ssa_lattice_fetch(ctx, SSA_LAT_SNAP_DOMAINS).reshape(n_snap, -1, 2)
    return out


# --------------------------------------------------------------------------
# Test and measurement entry points (include/bitssa_test.h)
# --------------------------------------------------------------------------
def bitssa_test_philox(ctr, key, which=0):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.zeros_like(ctr)
    _check(lib().bitssa_test_philox(_p(ctr, C.c_uint32), _p(key, C.c_uint32), _p(out, C.c_uint32),
                                    len(ctr), which))
    return out


def bitssa_test_bitslice(op, x, y):
    x = np.ascontiguousarray(x, dtype=np.int64)
    y = np.ascontiguousarray(y, dtype=np.int64)
    out = np.zeros_like(x)
    _check(lib().bitssa_test_bitslice(op, _p(x, C.c_int64), _p(y, C.c_int64), _p(out, C.c_int64), len(x)))
    return out


def bitssa_bench_alu(device=-1, iters=2000):
    ops, ms = C.c_double(), C.c_double()
    _check(lib().bitssa_bench_alu(device, iters, C.byref(ops), C.byref(ms)))
    return ops.value, ms.value


# --------------------------------------------------------------------------
# Frank's model (Eqs. 1-3), species order (L, D, A)
# --------------------------------------------------------------------------
FRANK_REACTANTS = np.array([[1, 0, 1], [0, 1, 1], [1, 1, 0]], dtype=np.int32)
FRANK_PRODUCTS = np.array([[2, 0, 0], [0, 2, 0], [0, 0, 2]], dtype=np.int32)


def fetch_all(ctx, n_species=3, snapshots=False):
    """Every per-run field and the counters as numpy arrays."""
    out = {
        "final_counts": ssa_fetch(ctx, SSA_FIELD_FINAL_COUNTS).reshape(-1, n_species),
        "t_abs": ssa_fetch(ctx, SSA_FIELD_ABSORB_TIME),
        "outcome": ssa_fetch(ctx, SSA_FIELD_ABSORB_OUTCOME),
        "ee_hist": ssa_fetch(ctx, SSA_FIELD_EE_HIST).reshape(-1, 65),
        "counters": dict(zip(COUNTER_NAMES, ssa_fetch(ctx, SSA_FIELD_COUNTERS).tolist())),
        "ens_absorbed": ssa_fetch(ctx, SSA_FIELD_ENS_ABSORBED).reshape(-1, 4),
    }
    if snapshots:
        out["snap_counts"] = ssa_fetch(ctx, SSA_FIELD_SNAP_COUNTS)
    return out
