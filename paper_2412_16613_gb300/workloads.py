"""Seeded synthetic inputs shared by the tests, the benchmark and the CPU oracle runs.

Nothing here computes any part of the method: only the workload definitions
(initial counts, rates, run counts, seeds, snapshot times) drawn from numpy
generators with fixed seeds.  Frank's model species order is (L, D, A).
"""
from __future__ import annotations

import numpy as np


def log_snapshots(t_end: float = 50.0, n: int = 10) -> np.ndarray:
    """n log-spaced times t_end 10^(4 (s - (n-1)) / (n-1)), s = 0..n-1 (4 decades up to t_end)."""
    s = np.arange(n)
    return t_end * 10.0 ** (4.0 * (s - (n - 1)) / (n - 1))


def racemic_init(n_tot: int) -> np.ndarray:
    """L = D = floor(N/4), A = N - 2 floor(N/4)."""
    q = n_tot // 4
    return np.array([q, q, n_tot - 2 * q], dtype=np.int64)


def batch_ensembles(n_ens: int = 4096, runs: int = 1024, n_min: int = 16, n_max: int = 65536,
                    rate_lo: float = 0.5, rate_hi: float = 2.0, seed: int = 0x5EED):
    """Ensembles with N_tot log-uniform in [n_min, n_max] (rounded), each rate uniform in
    [rate_lo, rate_hi], racemic initial counts, `runs` runs and seed e each."""
    rng = np.random.default_rng(seed)
    n_tot = np.rint(np.exp(rng.uniform(np.log(n_min), np.log(n_max), n_ens))).astype(np.int64)
    n_tot = np.clip(n_tot, n_min, n_max)
    rates = rng.uniform(rate_lo, rate_hi, size=(n_ens, 3))
    init = np.stack([racemic_init(int(n)) for n in n_tot])
    runs_e = np.full(n_ens, runs, dtype=np.int64)
    seeds = np.arange(n_ens, dtype=np.uint64)
    return {"n_tot": n_tot, "init": init, "rates": rates, "runs": runs_e, "seeds": seeds}


def multinomial_init(n_runs: int, n_tot: int, p=(0.25, 0.25, 0.5), seed: int = 77) -> np.ndarray:
    """Independent multinomial initial states around the racemic point."""
    rng = np.random.default_rng(seed)
    return rng.multinomial(n_tot, p, size=n_runs).astype(np.int64)


def lattice_init(lx: int, ly: int, n_runs: int, mean=(8.0, 8.0, 16.0), seed: int = 0x1A77) -> np.ndarray:
    """Per-run, per-site counts of (L, D, A) on an lx x ly lattice, independent Poisson draws with
    the given means: Poisson(sum(mean)) molecules per site split multinomially in the ratio of the
    means (L:D:A = 1:1:2 by default).  Shape [n_runs][lx ly][3], site index x + lx y."""
    rng = np.random.default_rng(seed)
    return rng.poisson(mean, size=(n_runs, lx * ly, 3)).astype(np.int64)
