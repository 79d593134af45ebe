"""GPU parity of the bound that follows the group's state (pad_pow2 = 2: at each step the bound
is 2^p, p the bit length of the largest S_R over the group's live runs), against the oracle
stepping the same groups: runs, snapshots, counters, ragged groups, per-run initial states,
every clock, batches, and sampled runs at the benchmark's sizes."""
import math
import os

import numpy as np
import pytest

import oracle
import paper_2412_16613_gb300 as pkg
from paper_2412_16613_gb300 import workloads
from tests._gpu import assert_parity, gpu_run, log_snapshots

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


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


@pytest.mark.parametrize("N,rates", [(12, (1.0, 0.5, 2.0)), (64, (1.0, 1.0, 1.0)), (1024, (1.0, 1.0, 1.0)),
                                     (10000, (0.7, 1.3, 1.9)), (46400, (1.0, 1.0, 1.0))])
def test_parity_state_following_bound(N, rates):
    """Runs, snapshots and counters on a ragged last group, over ~10^4 steps a run (or to
    absorption for small N)."""
    init = (N // 4, N // 4, N - 2 * (N // 4))
    lam = 2 ** (N * (N - 1) // 2).bit_length() * max(rates)
    t_end = 1.2e4 / lam if N > 64 else 50.0
    snaps = [t_end / 3, 2 * t_end / 3]
    n = 96 + 5
    g = gpu_run(init, n, seed=31, t_end=t_end, snaps=snaps, rates=rates, pad_pow2=2)
    r = oracle.run(oracle.frank(*rates), init, n, seed=31, t_end=t_end, snap_times=snaps, threads=THREADS,
                   pad_pow2=2)
    ok = assert_parity(g, r)
    assert g["counters"]["redraw_rounds"] == 0
    if ok.all():
        assert g["counters"]["lane_steps"] == r["steps"].sum()
        assert g["counters"]["reactions"] == r["reactions"].sum()


def test_parity_state_following_bound_to_absorption():
    """N = 64 to absorption on 4113 runs (ragged): every run, 10 snapshots, the step counts."""
    n = 4096 + 17
    snaps = log_snapshots(10.0, 10)
    g = gpu_run((16, 16, 32), n, seed=3, t_end=10.0, snaps=snaps, pad_pow2=2)
    r = oracle.run(oracle.frank(), (16, 16, 32), n, seed=3, t_end=10.0, snap_times=snaps, threads=THREADS,
                   pad_pow2=2)
    ok = assert_parity(g, r)
    assert np.all(r["outcome"][ok] >= 0)
    if ok.all():
        assert g["counters"]["lane_steps"] == r["steps"].sum()


def test_parity_state_following_bound_per_run_init():
    """Per-run initial states, so that the group's largest S_R, not a lane's own, sets the bound."""
    rng = np.random.default_rng(12)
    n = 320 + 9
    init = rng.multinomial(500, [0.2, 0.2, 0.6], size=n)
    init[::7] = (1, 0, 499)  # near-absorbed lanes among busy ones
    g = gpu_run(init, n, seed=8, t_end=2.0, snaps=[0.001, 0.01], pad_pow2=2)
    r = oracle.run(oracle.frank(), init, seed=8, t_end=2.0, snap_times=[0.001, 0.01], threads=THREADS,
                   pad_pow2=2)
    assert_parity(g, r)


@pytest.mark.parametrize("mode,omode,rtol,tie", [
    (pkg.SSA_P64_LOGSUM, oracle.P64, 1e-12, 1e-12),
    (pkg.SSA_P32_KAHAN, oracle.P32_KAHAN, 2e-5, 1e-6),
    (pkg.SSA_P32_D64ACC, oracle.P32_D64ACC, 2e-5, 1e-6),
    (pkg.SSA_P32_PLAIN, oracle.P32_PLAIN, 2e-5, 1e-6),
])
def test_parity_state_following_bound_clocks(mode, omode, rtol, tie):
    """Every clock at the rate k_max 2^p of each step.  The 32 runs of a group share their event
    times, so a near tie leaves out a whole group: 129 groups, at least 90% of them compared."""
    snaps = log_snapshots(50.0, 10)
    n = 4096 + 5
    g = gpu_run((256, 256, 512), n, seed=4, t_end=50.0, snaps=snaps, precision=mode, pad_pow2=2)
    r = oracle.run(oracle.frank(), (256, 256, 512), n, seed=4, t_end=50.0, snap_times=snaps, precision=omode,
                   threads=THREADS, pad_pow2=2)
    assert_parity(g, r, rtol=rtol, tie=tie, min_ok=0.9)


def test_state_following_bound_runs_on_one_thread_and_tunes():
    """The automatic layout and the tuner pick one thread per group; the results do not depend
    on the block size."""
    import torch
    snaps = [0.005, 0.02]
    a = gpu_run((256, 256, 512), 64 * 152 * 32, seed=2, t_end=0.05, snaps=snaps, pad_pow2=2)
    assert a["counters"]["layout"] & pkg.SSA_LAYOUT_THREAD and not a["counters"]["layout"] & pkg.SSA_LAYOUT_WARPS
    b = gpu_run((256, 256, 512), 64 * 152 * 32, seed=2, t_end=0.05, snaps=snaps, pad_pow2=2, block_size=128)
    for k in ("final_counts", "outcome", "t_abs", "snap_counts"):
        assert np.array_equal(a[k], b[k]), k
    o = pkg.ssa_default_options(cuda_stream=torch.cuda.current_stream(), pad_pow2=2)
    ctx = pkg.ssa_create(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, [1.0, 1.0, 1.0], np.array([256, 256, 512]),
                         8192, 2, o)
    try:
        choice = pkg.ssa_tune(ctx, 0.05, snaps, 200)
        assert choice[0] == pkg.SSA_LAYOUT_THREAD
        pkg.ssa_run(ctx, 0.05, snaps)
        g = pkg.fetch_all(ctx)
    finally:
        pkg.ssa_destroy(ctx)
    assert np.array_equal(g["final_counts"], a["final_counts"][:8192])


def test_batch_state_following_bound():
    """A batch of ensembles (N_tot, rates, runs and seeds differ; ragged groups) under the
    state-following bound, every run against the oracle of its ensemble."""
    import torch
    rng = np.random.default_rng(6)
    n_ens = 12
    n_tot = np.array([16, 64, 100, 300, 1024, 1500, 4000, 16, 64, 777, 2048, 50])
    init = np.stack([n_tot // 4, n_tot // 4, n_tot - 2 * (n_tot // 4)], 1)
    rates = rng.uniform(0.5, 2.0, size=(n_ens, 3))
    runs = rng.integers(1, 90, size=n_ens)
    seeds = np.arange(n_ens, dtype=np.uint64) + 100
    o = pkg.ssa_default_options(cuda_stream=torch.cuda.current_stream(), pad_pow2=2)
    ctx = pkg.ssa_create_batch(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, init, rates, runs, seeds, o)
    t_end = 0.2
    try:
        pkg.ssa_run(ctx, t_end, [0.01])
        g = pkg.fetch_all(ctx)
    finally:
        pkg.ssa_destroy(ctx)
    off = np.concatenate([[0], np.cumsum(runs)])
    for e in range(n_ens):
        r = oracle.run(oracle.frank(*rates[e]), init[e], int(runs[e]), seed=int(seeds[e]), t_end=t_end,
                       snap_times=[0.01], threads=THREADS, pad_pow2=2)
        sub = {k: g[k][off[e]:off[e + 1]] for k in ("final_counts", "outcome", "t_abs")}
        assert_parity(sub, r, snaps=False, min_ok=0.95)


@pytest.mark.parametrize("init,n,samples", [((256, 256, 512), 1 << 20, 48), ((2500, 2500, 5000), 1 << 22, 24)])
def test_full_size_state_following_bound_sampled(init, n, samples):
    """The benchmark's sizes: sampled runs (each from its whole group in the oracle) and
    invariants over every run."""
    T_END = 50.0
    SNAPS = list(workloads.log_snapshots(T_END, 10))
    g = gpu_run(init, n, seed=0, t_end=T_END, snaps=SNAPS, keep_snaps=False, pad_pow2=2)
    rng = np.random.default_rng(n + 1)
    ids = np.unique(np.concatenate([[0, 31, 32, n - 1], rng.integers(0, n, samples)]))
    r = oracle.run(oracle.frank(), init, run_ids=ids, seed=0, t_end=T_END, snap_times=SNAPS, threads=THREADS,
                   pad_pow2=2, ensemble_runs=n)
    sub = {k: g[k][ids] for k in ("final_counts", "outcome", "t_abs")}
    assert_parity(sub, r, snaps=False, min_ok=0.95)
    fc = g["final_counts"]
    assert np.all(fc.sum(1) == sum(init))
    absorbed = g["outcome"] >= 0
    assert np.all((fc[absorbed] > 0).sum(1) == 1)
    assert g["counters"]["absorbed"] == absorbed.sum() and g["counters"]["redraw_rounds"] == 0
    assert np.all(g["ee_hist"].sum(1) == n)
    pL, pD = np.mean(g["outcome"] == 0), np.mean(g["outcome"] == 1)
    assert abs(pL - pD) < 5 * math.sqrt((pL + pD) / n)
