"""CPU oracle for the bit-sliced Gillespie method (arXiv 2412.16613).

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; the product package never imports
it.  The C source (``oracle.c``) is the oracle; this module compiles it with
gcc and marshals numpy arrays through ctypes.

The oracle is a plain serial Gillespie simulation with integer counts
(Sec. 3 of the paper, steps 1-7), driven by the counter-based stream described
in ``oracle.h`` so that one run can be recomputed on its own (with its whole group
under the state-following bound, ``pad_pow2=2``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRC_LATTICE = os.path.join(_HERE, "lattice.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

P64, P32_KAHAN, P32_D64ACC, P32_PLAIN = 0, 1, 2, 3
OK, EINVAL, ETIMEOUT, ERANGE = 0, -1, -5, -6
MAX_SPECIES = 8
MAX_REACTIONS = 8


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no fp contraction, so hosts agree)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(f) > os.path.getmtime(_LIB) for f in (_SRC, _SRC_LATTICE, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-Wall", "-Wextra", "-o", tmp, _SRC, _SRC_LATTICE, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Problem(C.Structure):
    _fields_ = [
        ("n_species", C.c_int32), ("n_reactions", C.c_int32),
        ("reactants", C.POINTER(C.c_int32)), ("products", C.POINTER(C.c_int32)),
        ("rates", C.POINTER(C.c_double)), ("n_tot", C.c_int64), ("seed", C.c_uint64),
        ("precision", C.c_int32), ("thin_bits", C.c_int32), ("t_end", C.c_double),
        ("snap_times", C.POINTER(C.c_double)), ("n_snap", C.c_int32),
        ("step_budget", C.c_int64), ("shared_n", C.c_int32), ("pad_pow2", C.c_int32),
        ("ensemble_runs", C.c_int64), ("lane_clock", C.c_int32),
    ]


class Lattice(C.Structure):
    _fields_ = [
        ("lx", C.c_int32), ("ly", C.c_int32), ("rates", C.POINTER(C.c_double)), ("hop", C.c_double),
        ("seed", C.c_uint64), ("precision", C.c_int32), ("thin_bits", C.c_int32), ("t_end", C.c_double),
        ("snap_times", C.POINTER(C.c_double)), ("n_snap", C.c_int32), ("step_budget", C.c_int64),
    ]


class LatticeResult(C.Structure):
    _fields_ = [
        ("t_homochiral", C.c_double), ("outcome", C.c_int32), ("status", C.c_int32), ("steps", C.c_int64),
        ("reactions", C.c_int64), ("hops", C.c_int64), ("cap", C.c_int32), ("pad", C.c_int32),
        ("margin", C.c_double),
    ]


class Derived(C.Structure):
    _fields_ = [
        ("lambda_int", C.c_uint64), ("K", C.c_int32), ("k_max", C.c_double),
        ("lambda_", C.c_double), ("thin_always", C.c_int32 * MAX_REACTIONS),
        ("thin_T", C.c_uint64 * MAX_REACTIONS), ("any_thinning", C.c_int32),
    ]


class Result(C.Structure):
    _fields_ = [
        ("final_counts", C.c_int64 * MAX_SPECIES), ("t_abs", C.c_double), ("t_last", C.c_double),
        ("outcome", C.c_int32), ("status", C.c_int32), ("steps", C.c_int64),
        ("reactions", C.c_int64), ("redraws", C.c_int64), ("margin", C.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                            C.POINTER(C.c_uint32)]
            L.orc_philox4x32_10.restype = None
            L.orc_stream_word.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32,
                                          C.c_uint32, C.c_uint32]
            L.orc_stream_word.restype = C.c_uint32
            L.orc_derive.argtypes = [C.POINTER(Problem), C.POINTER(Derived)]
            L.orc_derive.restype = C.c_int
            L.orc_propensities.argtypes = [C.POINTER(Problem), C.POINTER(C.c_int64),
                                           C.POINTER(C.c_int64)]
            L.orc_select.argtypes = [C.POINTER(Problem), C.POINTER(C.c_int64), C.c_uint64]
            L.orc_select.restype = C.c_int32
            L.orc_run_many.argtypes = [C.POINTER(Problem), C.c_int64, C.POINTER(C.c_int64),
                                       C.c_int64, C.POINTER(C.c_int64), C.c_int32,
                                       C.POINTER(Result), C.POINTER(C.c_int64), C.c_int32]
            L.orc_run_many.restype = C.c_int
            L.orc_lattice_group.argtypes = [C.POINTER(Lattice), C.c_uint64, C.c_int32, C.POINTER(C.c_int64),
                                            C.POINTER(LatticeResult), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                            C.POINTER(C.c_int64)]
            L.orc_lattice_group.restype = C.c_int
            L.orc_ee_bin.argtypes = [C.c_int64, C.c_int64]
            L.orc_ee_bin.restype = C.c_int32
            _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


class Network:
    """A conserved mass-action network: stoichiometry [R][S] and rates [R]."""

    def __init__(self, reactants, products, rates, species=None):
        self.reactants = np.ascontiguousarray(reactants, dtype=np.int32)
        self.products = np.ascontiguousarray(products, dtype=np.int32)
        self.rates = np.ascontiguousarray(rates, dtype=np.float64)
        self.n_reactions, self.n_species = self.reactants.shape
        self.species = species or [f"X{i}" for i in range(self.n_species)]


def frank(k1=1.0, k2=1.0, k3=1.0) -> Network:
    """Frank's model in species order (L, D, A) (Eqs. 1-3): A+L->2L, A+D->2D, L+D->2A."""
    reac = [[1, 0, 1], [0, 1, 1], [1, 1, 0]]
    prod = [[2, 0, 0], [0, 2, 0], [0, 0, 2]]
    return Network(reac, prod, [k1, k2, k3], species=["L", "D", "A"])


def _problem(net: Network, n_tot, seed, precision=P64, thin_bits=32, t_end=np.inf,
             snap_times=(), step_budget=0, shared_n=False, pad_pow2=False, ensemble_runs=0, lane_clock=False):
    snaps = np.ascontiguousarray(snap_times, dtype=np.float64)
    p = Problem(net.n_species, net.n_reactions, _ptr(net.reactants, C.c_int32),
                _ptr(net.products, C.c_int32), _ptr(net.rates, C.c_double), int(n_tot),
                int(seed) & (2**64 - 1), int(precision), int(thin_bits), float(t_end),
                _ptr(snaps, C.c_double) if len(snaps) else None, len(snaps), int(step_budget),
                1 if shared_n else 0, int(pad_pow2), int(ensemble_runs), 1 if lane_clock else 0)
    p._keep = (net, snaps)  # keep the arrays alive as long as the struct
    return p


def derive(net: Network, n_tot, **kw):
    p = _problem(net, n_tot, 0, **kw)
    d = Derived()
    st = lib().orc_derive(C.byref(p), C.byref(d))
    if st != OK:
        raise ValueError(f"orc_derive failed with status {st}")
    return d


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [o[i] for i in range(4)]


def stream_word(seed, group, step, attempt, tag, k):
    return lib().orc_stream_word(seed, group, step, attempt, tag, k)


def propensities(net: Network, state):
    p = _problem(net, int(np.sum(state)), 0)
    s = np.ascontiguousarray(state, dtype=np.int64)
    h = np.zeros(net.n_reactions, dtype=np.int64)
    lib().orc_propensities(C.byref(p), _ptr(s, C.c_int64), _ptr(h, C.c_int64))
    return h


def select(net: Network, state, n):
    p = _problem(net, int(np.sum(state)), 0)
    s = np.ascontiguousarray(state, dtype=np.int64)
    return lib().orc_select(C.byref(p), _ptr(s, C.c_int64), int(n))


def ee_bin(L, D):
    return lib().orc_ee_bin(int(L), int(D))


def run(net: Network, init, n_runs=None, *, seed=0, precision=P64, thin_bits=32, t_end=np.inf,
        snap_times=(), step_budget=0, first_run=0, run_ids=None, threads=None,
        want_snapshots=True, check=True, shared_n=False, pad_pow2=False, ensemble_runs=None, lane_clock=False):
    """Run the oracle on runs first_run .. first_run+n_runs-1 (or on run_ids).

    init: [S] shared initial counts or [n_runs][S] per-run counts.
    shared_n: every run of a group of 32 uses the n of the group's lane 0 (Sec. 4, step a).
    pad_pow2: 1 (or True): the uniformisation bound is 2^K (null events fill the gap above
        lambda_int); 2: the bound follows the group's state, 2^p with p the bit length of the
        largest S_R over the group's live runs, and each run comes out of its whole group.
    lane_clock: every run has its own clock (its waiting times from its own stream) instead of
        one clock per group of 32 runs.
    ensemble_runs (pad_pow2 = 2): runs in the ensemble, which fixes the lanes of its last group;
        default first_run + n_runs without run_ids, else every group full.  A per-run init then
        holds one row per run of the ensemble, indexed by run.
    Returns a dict of numpy arrays indexed by run position.
    """
    init = np.ascontiguousarray(init, dtype=np.int64)
    per_run = 1 if init.ndim == 2 else 0
    ids = None
    if run_ids is not None:
        ids = np.ascontiguousarray(run_ids, dtype=np.int64)
        n_runs = len(ids)
    if n_runs is None:
        n_runs = init.shape[0] if per_run else 1
    pad_pow2 = int(pad_pow2)
    if ensemble_runs is None:
        ensemble_runs = first_run + n_runs if (pad_pow2 == 2 and ids is None) else 0
    if pad_pow2 == 2 and per_run:
        last = int(ids.max()) if ids is not None and len(ids) else first_run + n_runs - 1
        need = max(ensemble_runs, 32 * (last // 32 + 1)) if ensemble_runs == 0 else ensemble_runs
        if init.shape[0] < need:
            raise ValueError("pad_pow2 = 2 with per-run counts needs a row for every run of each group")
    n_tot = int(init.reshape(-1, net.n_species)[0].sum())
    p = _problem(net, n_tot, seed, precision, thin_bits, t_end, snap_times, step_budget, shared_n,
                 pad_pow2, ensemble_runs, lane_clock)
    out = (Result * max(n_runs, 1))()
    n_snap = len(snap_times)
    snaps = (np.zeros((n_snap, n_runs, net.n_species), dtype=np.int64)
             if (want_snapshots and n_snap) else None)
    threads = threads or os.cpu_count() or 1
    st = lib().orc_run_many(C.byref(p), int(first_run), _ptr(ids, C.c_int64), int(n_runs),
                            _ptr(init, C.c_int64), per_run, out, _ptr(snaps, C.c_int64),
                            int(threads))
    if check and st != OK:
        raise RuntimeError(f"oracle failed with status {st}")
    res = np.ctypeslib.as_array(out)[:n_runs]
    S = net.n_species
    return {
        "status": st,
        "final_counts": np.array(res["final_counts"][:, :S]),
        "t_abs": np.array(res["t_abs"]),
        "t_last": np.array(res["t_last"]),
        "outcome": np.array(res["outcome"]),
        "run_status": np.array(res["status"]),
        "steps": np.array(res["steps"]),
        "reactions": np.array(res["reactions"]),
        "redraws": np.array(res["redraws"]),
        "margin": np.array(res["margin"]),
        "snap_counts": snaps,
    }


def ee_histogram(snap_counts, iL=0, iD=1):
    """[n_snap][n_runs][S] counts -> [n_snap][65] histogram, bins by orc_ee_bin."""
    n_snap = snap_counts.shape[0]
    hist = np.zeros((n_snap, 65), dtype=np.uint64)
    f = lib().orc_ee_bin
    for s in range(n_snap):
        for L, D in zip(snap_counts[s, :, iL].tolist(), snap_counts[s, :, iD].tolist()):
            hist[s, f(L, D)] += 1
    return hist


def lattice_run(lx, ly, init, n_runs=None, *, rates=(1.0, 1.0, 1.0), hop=0.1, seed=0, precision=P64,
                thin_bits=32, t_end=1.0, snap_times=(), step_budget=0, groups=None, threads=None, check=True,
                lanes=32):
    """Frank's model on a periodic lx x ly lattice (orc_lattice_group), group by group.

    init: [M][3] counts shared by every run, or [n_runs][M][3] per run (site index x + lx y).
    lanes: runs per group (32 as on the GPU; 1 gives every run its own group and stream).
    groups: the group indices to run (runs lanes g .. lanes g + lanes - 1, the last group of n_runs
    ragged); default every group of n_runs.  Returns per-run arrays for the runs of those groups.
    """
    import concurrent.futures as cf
    M = lx * ly
    init = np.ascontiguousarray(init, dtype=np.int64)
    per_run = init.ndim == 3
    if n_runs is None:
        n_runs = init.shape[0] if per_run else 32
    if groups is None:
        groups = range((n_runs + lanes - 1) // lanes)
    groups = list(groups)
    per_group = lanes
    k = np.ascontiguousarray(rates, dtype=np.float64)
    snaps = np.ascontiguousarray(snap_times, dtype=np.float64)
    S = len(snaps)

    def one(g):
        lanes = min(per_group, n_runs - per_group * g)
        if per_run:
            ini = np.ascontiguousarray(init[per_group * g:per_group * g + lanes])
        else:
            ini = np.ascontiguousarray(np.broadcast_to(init, (lanes, M, 3)))
        p = Lattice(lx, ly, _ptr(k, C.c_double), float(hop), int(seed) & (2**64 - 1), int(precision),
                    int(thin_bits), float(t_end), _ptr(snaps, C.c_double) if S else None, S, int(step_budget))
        out = (LatticeResult * lanes)()
        fin = np.zeros((lanes, M, 3), dtype=np.int64)
        st_tot = np.zeros((lanes, max(S, 1), 3), dtype=np.int64)
        st_dom = np.zeros((lanes, max(S, 1), 2), dtype=np.int64)
        status = lib().orc_lattice_group(C.byref(p), int(g), lanes, _ptr(ini, C.c_int64), out,
                                         _ptr(fin, C.c_int64), _ptr(st_tot, C.c_int64), _ptr(st_dom, C.c_int64))
        res = np.ctypeslib.as_array(out)[:lanes].copy()
        return status, res, fin, st_tot[:, :S], st_dom[:, :S]

    threads = threads or os.cpu_count() or 1
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(one, groups))
    status = min((p[0] for p in parts), default=OK)
    if check and status not in (OK,):
        raise RuntimeError(f"lattice oracle failed with status {status}")
    res = np.concatenate([p[1] for p in parts]) if parts else np.zeros(0, dtype=LatticeResult)
    return {
        "status": status,
        "final_counts": np.concatenate([p[2] for p in parts]),
        "snap_totals": np.concatenate([p[3] for p in parts]),
        "snap_domains": np.concatenate([p[4] for p in parts]),
        "t_homochiral": np.array(res["t_homochiral"]), "outcome": np.array(res["outcome"]),
        "run_status": np.array(res["status"]), "steps": np.array(res["steps"]),
        "reactions": np.array(res["reactions"]), "hops": np.array(res["hops"]),
        "cap": np.array(res["cap"]), "margin": np.array(res["margin"]),
    }
