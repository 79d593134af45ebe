"""GPU parity at the benchmark's full sizes, in the launch configuration `bench.py` times
(bound padded to 2^K, automatic layout): sampled runs recomputed one by one by the oracle,
and invariants that hold for every run.

* N_tot = 1024, (256, 256, 512), 2^20 runs, t_end = 50, 10 log-spaced snapshots.
* N_tot = 10 000, (2500, 2500, 5000), 2^22 runs, same schedule.
* 4096 ensembles, N_tot log-uniform in [16, 65536], rates in [0.5, 2], 1024 runs each.
"""
import math
import os

import numpy as np
import pytest

import oracle
import paper_2412_16613_gb300 as pkg
from paper_2412_16613_gb300 import workloads
from tests._gpu import assert_parity, gpu_run

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4
T_END = 50.0
SNAPS = list(workloads.log_snapshots(T_END, 10))


@pytest.fixture(scope="module", autouse=True)
def device():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    oracle.build()
    torch.cuda.set_device(0)
    pkg.use_torch_allocator()
    yield
    torch.cuda.synchronize()


def _invariants(g, n_tot, n):
    fc = g["final_counts"]
    assert np.all(fc.sum(1) == n_tot)
    absorbed = g["outcome"] >= 0
    assert np.all((fc[absorbed] > 0).sum(1) == 1)
    assert np.all(np.isfinite(g["t_abs"][absorbed])) and np.all(np.isinf(g["t_abs"][~absorbed]))
    assert g["counters"]["absorbed"] == absorbed.sum()
    assert g["counters"]["redraw_rounds"] == 0  # the padded bound accepts every draw


@pytest.mark.parametrize("init,n,samples", [((256, 256, 512), 1 << 20, 64), ((2500, 2500, 5000), 1 << 22, 40)])
def test_full_size_padded_sampled(init, n, samples):
    g = gpu_run(init, n, seed=0, t_end=T_END, snaps=SNAPS, keep_snaps=False, pad_pow2=1)
    rng = np.random.default_rng(n)
    ids = np.unique(np.concatenate([[0, 31, 32, n - 1], rng.integers(0, n, samples)]))
    r = oracle.run(oracle.frank(), init, run_ids=ids, seed=0, t_end=T_END, snap_times=SNAPS, threads=THREADS,
                   pad_pow2=True)
    sub = {k: g[k][ids] for k in ("final_counts", "outcome", "t_abs")}
    assert_parity(sub, r, snaps=False, min_ok=0.95)
    _invariants(g, sum(init), n)
    assert np.all(g["ee_hist"].sum(1) == n)
    pL, pD = np.mean(g["outcome"] == 0), np.mean(g["outcome"] == 1)
    assert abs(pL - pD) < 5 * math.sqrt((pL + pD) / n)


def test_batch_full_size_padded_sampled():
    """The 4096-ensemble batch with its per-bucket layouts; sampled runs from the widest ensembles
    (K = 31, the longest runs) and from random ones."""
    import torch
    B = workloads.batch_ensembles()
    o = pkg.ssa_default_options(cuda_stream=torch.cuda.current_stream(), pad_pow2=1)
    ctx = pkg.ssa_create_batch(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, B["init"], B["rates"], B["runs"],
                               B["seeds"], o)
    try:
        pkg.ssa_run(ctx, T_END, SNAPS)
        g = pkg.fetch_all(ctx)
    finally:
        pkg.ssa_destroy(ctx)
    n_ens = len(B["runs"])
    offsets = np.concatenate([[0], np.cumsum(B["runs"])])
    rng = np.random.default_rng(99)
    widest = np.argsort(B["n_tot"])[-3:]
    picks = [(int(e), int(j)) for e in widest for j in (0, 1023)]
    picks += [(int(e), int(rng.integers(0, 1024))) for e in rng.integers(0, n_ens, 30)]
    for e, j in picks:
        r = oracle.run(oracle.frank(*B["rates"][e]), B["init"][e], run_ids=[j], seed=int(B["seeds"][e]),
                       t_end=T_END, snap_times=SNAPS, pad_pow2=True)
        row = offsets[e] + j
        sub = {k: g[k][row:row + 1] for k in ("final_counts", "outcome", "t_abs")}
        if r["margin"][0] > 1e-12:
            assert_parity(sub, r, snaps=False, min_ok=1.0)
    totals = np.repeat(B["n_tot"], B["runs"])
    assert np.all(g["final_counts"].sum(1) == totals)
    assert g["counters"]["redraw_rounds"] == 0
    assert np.all(g["ee_hist"].reshape(n_ens, len(SNAPS), 65).sum(2) == B["runs"][:, None])
