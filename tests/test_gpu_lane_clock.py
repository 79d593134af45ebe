"""The per-run clock (SSA_CLOCK_LANE) through the C ABI against the oracle in the same mode.

Under the group clock the 32 runs of a group share their event times (the paper's one tau for all
copies, end of Sec. 4): each run is an exact sample path, but the runs of a group are dependent.
With SSA_CLOCK_LANE every run draws its waiting times (Eq. equation-tau) from its own stream,
keeps its own snapshots and stops alone at t_end.  Counts, outcomes and histograms bit-exact;
fp64 times within 1e-12 relative, fp32 within 2e-5."""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
import paper_2412_16613_gb300 as pkg
from tests._gpu import assert_hist_parity, assert_parity, gpu_run, log_snapshots

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4
LANE = pkg.SSA_CLOCK_LANE


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


def test_lane_clock_n64_all_runs():
    """N_tot = 64, (16, 16, 32), 64 runs, t_end = 10: every run, snapshot, histogram, counter."""
    snaps = [0.01, 0.05, 0.1, 0.5, 10.0]
    g = gpu_run((16, 16, 32), 64, seed=0, t_end=10.0, snaps=snaps, clock=LANE)
    r = oracle.run(oracle.frank(), (16, 16, 32), 64, seed=0, t_end=10.0, snap_times=snaps, lane_clock=True)
    ok = assert_parity(g, r)
    assert ok.all()
    assert_hist_parity(g, r, ok)
    assert g["counters"]["reactions"] == r["reactions"].sum()
    assert g["counters"]["lane_steps"] == r["steps"].sum()
    t = g["t_abs"].reshape(2, 32)
    assert np.all(np.ptp(t, axis=1) > 0)  # the runs of a group no longer share their times


@pytest.mark.parametrize("pad", [0, 1], ids=["paper_bound", "padded"])
@pytest.mark.parametrize("mode,omode,rtol,tie", [
    (pkg.SSA_P64, oracle.P64, 1e-12, 1e-12),
    (pkg.SSA_P64_LOGSUM, oracle.P64, 1e-12, 1e-12),
    (pkg.SSA_P32_KAHAN, oracle.P32_KAHAN, 2e-5, 1e-6),
    (pkg.SSA_P32_D64ACC, oracle.P32_D64ACC, 2e-5, 1e-6),
    (pkg.SSA_P32_PLAIN, oracle.P32_PLAIN, 2e-5, 1e-6),
])
def test_lane_clock_n1024_every_clock(mode, omode, rtol, tie, pad):
    """N_tot = 1024, 2048 + 5 runs (ragged last group), the 10 log-spaced snapshots to t_end = 50."""
    n = 2048 + 5
    snaps = log_snapshots(50.0, 10)
    g = gpu_run((256, 256, 512), n, seed=3, t_end=50.0, snaps=snaps, precision=mode, pad_pow2=pad, clock=LANE)
    r = oracle.run(oracle.frank(), (256, 256, 512), n, seed=3, t_end=50.0, snap_times=snaps, precision=omode,
                   pad_pow2=bool(pad), lane_clock=True, threads=THREADS)
    ok = assert_parity(g, r, rtol=rtol, tie=tie, min_ok=0.95)
    assert_hist_parity(g, r, ok)


@pytest.mark.parametrize("t_end", [0.004, 0.02])
def test_lane_clock_runs_stop_alone_at_t_end(t_end):
    """t_end before most runs absorb: each run stops at its own last event before t_end."""
    n = 1024 + 3
    snaps = [t_end / 4, t_end / 2]
    g = gpu_run((256, 256, 512), n, seed=7, t_end=t_end, snaps=snaps, clock=LANE, pad_pow2=1)
    r = oracle.run(oracle.frank(), (256, 256, 512), n, seed=7, t_end=t_end, snap_times=snaps, pad_pow2=True,
                   lane_clock=True, threads=THREADS)
    ok = assert_parity(g, r)
    assert ok.all()
    assert_hist_parity(g, r, ok)
    assert (r["outcome"] == -1).sum() > n // 10
    assert g["counters"]["lane_steps"] == r["steps"].sum()
    assert g["counters"]["reactions"] == r["reactions"].sum()


@pytest.mark.parametrize("rates,q", [((1.0, 0.5, 0.25), 32), ((0.7, 2.0, 1.3), 64), ((0.0, 0.0, 1.0), 32)])
def test_lane_clock_thinning(rates, q):
    snaps = [0.01, 0.1]
    n = 512 + 3
    g = gpu_run((64, 64, 128), n, seed=12, t_end=2.0, snaps=snaps, rates=rates, thin_bits=q, clock=LANE)
    r = oracle.run(oracle.frank(*rates), (64, 64, 128), n, seed=12, t_end=2.0, snap_times=snaps, thin_bits=q,
                   lane_clock=True, threads=THREADS)
    assert_parity(g, r)


def test_lane_clock_per_run_initial_states_and_small_systems():
    rng = np.random.default_rng(77)
    n = 1000
    init = rng.multinomial(256, [0.25, 0.25, 0.5], size=n)
    init[:40] = (256, 0, 0)  # runs absorbed at the start
    snaps = [0.0, 0.01, 0.05]
    g = gpu_run(init, n, seed=4, t_end=1.0, snaps=snaps, clock=LANE)
    r = oracle.run(oracle.frank(), init, seed=4, t_end=1.0, snap_times=snaps, lane_clock=True, threads=THREADS)
    ok = assert_parity(g, r)
    assert_hist_parity(g, r, ok)
    for init in [(1, 0, 0), (1, 1, 0), (2, 1, 0), (0, 0, 50)]:
        g = gpu_run(init, 70, seed=2, t_end=3.0, snaps=[0.0, 0.5, 3.0], clock=LANE)
        r = oracle.run(oracle.frank(), init, 70, seed=2, t_end=3.0, snap_times=[0.0, 0.5, 3.0], lane_clock=True)
        assert_parity(g, r)


def test_lane_clock_sharded_and_launch_shape():
    """Blocks of 32 and 128 threads and two contexts split by first_run give the same runs."""
    snaps = [0.005, 0.02]
    base = gpu_run((256, 256, 512), 4096, seed=5, t_end=0.05, snaps=snaps, clock=LANE)
    for b in (32, 128):
        g = gpu_run((256, 256, 512), 4096, seed=5, t_end=0.05, snaps=snaps, clock=LANE, block_size=b)
        for k in ("final_counts", "outcome", "t_abs", "ee_hist", "snap_counts"):
            assert np.array_equal(g[k], base[k]), (b, k)
    a = gpu_run((256, 256, 512), 2048, seed=5, t_end=0.05, snaps=snaps, clock=LANE, first_run=0)
    b = gpu_run((256, 256, 512), 2048, seed=5, t_end=0.05, snaps=snaps, clock=LANE, first_run=2048)
    for k in ("final_counts", "outcome", "t_abs"):
        assert np.array_equal(np.concatenate([a[k], b[k]]), base[k]), k


@pytest.mark.parametrize("kw", [dict(layout=pkg.SSA_LAYOUT_WARPS), dict(pad_pow2=2),
                                dict(engine=pkg.SSA_ENGINE_GENERAL), dict(shared_n=1), dict(block_size=256)])
def test_lane_clock_unsupported_combinations(kw):
    with pytest.raises(pkg.SSAError) as ei:
        gpu_run((16, 16, 32), 64, t_end=1.0, clock=LANE, **kw)
    assert ei.value.status == pkg.SSA_EUNSUPPORTED


def test_correlation_within_a_group_both_clocks():
    """The dependence the group clock puts between the runs of a group, measured: the correlation
    of the absorption times of lanes 0 and 1 (and 5 and 31) over 2^20 runs.  It is largest where a
    run takes few steps: at N_tot = 16 from (4, 4, 8) the group clock gives about 0.08 (the oracle's
    figure over 20 000 groups), many standard errors above zero, and the per-run clock gives zero
    within 4.5 standard errors.  At N_tot = 1024 (about 16 000 steps a run) the shared clock's
    part of an absorption time averages out and both are near zero (printed).  At N_tot = 2 from
    (1, 1, 0), where every step fires, the group clock gives every run of a group the same time."""
    n = 1 << 20
    groups = n // 32
    se = 1 / math.sqrt(groups)
    res = {}
    for init in ((4, 4, 8), (256, 256, 512)):
        for name, clock in (("group", pkg.SSA_CLOCK_GROUP), ("lane", LANE)):
            g = gpu_run(init, n, seed=11, t_end=np.inf, keep_snaps=False, clock=clock, pad_pow2=1)
            t = g["t_abs"].reshape(groups, 32)
            res[(sum(init), name)] = [float(np.corrcoef(t[:, a], t[:, b])[0, 1]) for a, b in ((0, 1), (5, 31))]
    print("correlation of absorption times within a group (SE %.4f):" % se, res)
    assert min(res[(16, "group")]) > 8 * se, res
    assert max(abs(c) for c in res[(16, "lane")]) < 4.5 * se, res
    assert max(abs(c) for c in res[(1024, "lane")]) < 4.5 * se, res
    g = gpu_run((1, 1, 0), 3200, seed=2, t_end=np.inf, keep_snaps=False)
    assert np.all(g["t_abs"].reshape(-1, 32) == g["t_abs"].reshape(-1, 32)[:, :1])
    g = gpu_run((1, 1, 0), 3200, seed=2, t_end=np.inf, keep_snaps=False, clock=LANE)
    assert stats.kstest(g["t_abs"], "expon").pvalue > 1e-4


def test_two_seeds_ks_over_every_run_at_n10000():
    """The precision workload's size, 2^22 runs at N_tot = 10 000 (padded bound, fp64): the
    absorption times of two seeds compared by a two-sample KS test over every run.  The KS test
    assumes independent samples; under the per-run clock they are, and it passes; under the group
    clock the 32 runs of a group share their times and the test treats 2^17 groups as 2^22
    independent runs (both p-values printed)."""
    n = 1 << 22
    init = (2500, 2500, 5000)
    p = {}
    for name, clock in (("group", pkg.SSA_CLOCK_GROUP), ("lane", LANE)):
        a = gpu_run(init, n, seed=100, t_end=50.0, keep_snaps=False, clock=clock, pad_pow2=1)["t_abs"]
        b = gpu_run(init, n, seed=200, t_end=50.0, keep_snaps=False, clock=clock, pad_pow2=1)["t_abs"]
        assert np.isfinite(a).all() and np.isfinite(b).all()
        p[name] = stats.ks_2samp(a, b).pvalue
        se = math.sqrt(a.var() / n + b.var() / n)
        p[name + "_mean_diff_se"] = abs(a.mean() - b.mean()) / se
    print("two fp64 seeds over 2^22 runs:", p)
    assert p["lane"] > 1e-3 and p["lane_mean_diff_se"] < 4.5, p
