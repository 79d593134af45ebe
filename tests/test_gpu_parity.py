"""GPU parity: libbitssa through its C ABI against the CPU oracle on the same
seeded inputs.  Counts, outcomes and histograms bit-exact; fp64 event times
within 1e-12 relative; fp32 clocks within their own tolerance."""
import math
import os

import numpy as np
import pytest

import oracle
import paper_2412_16613_gb300 as pkg
from tests._gpu import FRANK_P, FRANK_R, assert_hist_parity, assert_parity, group_steps, gpu_run, log_snapshots

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4
# the two layouts of the bit-sliced engine must produce the same runs
LAYOUTS = pytest.mark.parametrize("layout", [pkg.SSA_LAYOUT_THREAD, pkg.SSA_LAYOUT_WARPS],
                                  ids=["thread", "warps"])


def same_counters(a, b):
    """Every run counter equal; the layout counter names the layout that ran."""
    return {k: v for k, v in a["counters"].items() if k != "layout"} == \
        {k: v for k, v in b["counters"].items() if k != "layout"}


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


# --------------------------------------------------------------------------
# Pieces of the hot path
# --------------------------------------------------------------------------
def test_philox_device_matches_oracle_and_curand():
    rng = np.random.default_rng(1)
    n = 4096
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    ours = pkg.bitssa_test_philox(ctr, key, which=0)
    curand = pkg.bitssa_test_philox(ctr, key, which=1)
    assert np.array_equal(ours, curand)
    for i in range(0, n, 97):
        assert oracle.philox4x32_10(ctr[i], key[i]) == curand[i].tolist()


@pytest.mark.parametrize("op", [0, 1, 2, 3, 4])
def test_bitslice_primitives_exhaustive(op):
    x, y = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    x, y = x.ravel(), y.ravel()
    out = pkg.bitssa_test_bitslice(op, x, y)
    if op == 0:
        want = x + y
    elif op == 1:
        want = x - y
    elif op == 2:
        want = (x < y).astype(np.int64)
    elif op == 3:
        want = x * y
    else:
        sel = y & 3  # the kernel reads the selector from the two low planes of y
        want = x + np.select([sel == 1, sel == 2, sel == 3], [3, -2, 5], 0)
    assert np.array_equal(out, want)


def test_paper_fig1_sum():
    """Fig. 1: augend 1 plus addend 1 gives 2 (tests/golden/paper_bitwise_examples.txt)."""
    x = np.ones(32, dtype=np.int64)
    assert np.all(pkg.bitssa_test_bitslice(0, x, x) == 2)


# --------------------------------------------------------------------------
# Whole runs against the oracle
# --------------------------------------------------------------------------
@LAYOUTS
def test_parity_n64_all_runs(layout):
    """N_tot = 64, (16, 16, 32), 64 runs in two groups, seed 0, t_end 10."""
    snaps = [0.01, 0.05, 0.1, 0.5, 10.0]
    g = gpu_run((16, 16, 32), 64, seed=0, t_end=10.0, snaps=snaps, layout=layout)
    r = oracle.run(oracle.frank(), (16, 16, 32), 64, seed=0, t_end=10.0, snap_times=snaps)
    ok = assert_parity(g, r)
    assert ok.all()
    assert g["counters"]["reactions"] == r["reactions"].sum()
    assert g["counters"]["lane_steps"] == r["steps"].sum()
    assert np.array_equal(g["ee_hist"], oracle.ee_histogram(r["snap_counts"]))


@LAYOUTS
def test_parity_n1024_subset_ragged(layout):
    """N_tot = 1024, (256, 256, 512), 4113 runs (129 groups, ragged last group), 10 log-spaced
    snapshots, t_end = 50: every run, every snapshot, the histograms and the counters."""
    n = 4096 + 17
    snaps = log_snapshots(50.0, 10)
    g = gpu_run((256, 256, 512), n, seed=0, t_end=50.0, snaps=snaps, layout=layout)
    r = oracle.run(oracle.frank(), (256, 256, 512), n, seed=0, t_end=50.0, snap_times=snaps,
                   threads=THREADS)
    ok = assert_parity(g, r)
    assert_hist_parity(g, r, ok)
    assert ok.all()  # at this seed the oracle reports no event within 1e-12 of a snapshot or t_end
    assert np.array_equal(g["ee_hist"], oracle.ee_histogram(r["snap_counts"]))
    assert g["counters"]["reactions"] == r["reactions"].sum()
    assert g["counters"]["lane_steps"] == r["steps"].sum()
    assert np.all(g["ee_hist"].sum(1) == n)
    assert np.all(g["final_counts"].sum(1) == 1024)


def test_parity_bench_configuration():
    """The benchmark's launch configuration on a subset of its workload: N_tot = 1024 from
    (256, 256, 512), the bound padded to 2^19, one thread per group in blocks of 128, the 10
    log-spaced snapshots to t_end = 50, seed 0; 8192 + 21 runs (257 groups, the last ragged).
    Every run, snapshot and histogram, and the run counters, against the oracle at the same bound."""
    n = 8192 + 21
    snaps = log_snapshots(50.0, 10)
    g = gpu_run((256, 256, 512), n, seed=0, t_end=50.0, snaps=snaps, layout=pkg.SSA_LAYOUT_THREAD,
                block_size=128, pad_pow2=1)
    r = oracle.run(oracle.frank(), (256, 256, 512), n, seed=0, t_end=50.0, snap_times=snaps, pad_pow2=True,
                   threads=THREADS)
    ok = assert_parity(g, r)
    assert_hist_parity(g, r, ok)
    assert ok.all()  # at this seed the oracle reports no event within 1e-12 of a snapshot or t_end
    assert np.array_equal(g["ee_hist"], oracle.ee_histogram(r["snap_counts"]))
    c = g["counters"]
    assert c["reactions"] == r["reactions"].sum() and c["lane_steps"] == r["steps"].sum()
    gs = group_steps(r, n)
    assert c["group_steps"] == gs.sum() and c["max_group_steps"] == gs.max()
    assert c["redraw_rounds"] == 0 and c["absorbed"] == (r["outcome"] >= 0).sum()
    assert c["groups_done"] == (n + 31) // 32 and c["layout"] & 3 == pkg.SSA_LAYOUT_THREAD


def test_parity_n1024_full_size_sampled():
    """The benchmark workload itself: 2^20 runs at N_tot = 1024; the oracle recomputes a
    sample of runs one by one, and every run satisfies the invariants."""
    n = 1 << 20
    snaps = log_snapshots(50.0, 10)
    g = gpu_run((256, 256, 512), n, seed=0, t_end=50.0, snaps=snaps, keep_snaps=False)
    rng = np.random.default_rng(2024)
    ids = np.unique(np.concatenate([[0, 31, 32, n - 1], rng.integers(0, n, 60)]))
    r = oracle.run(oracle.frank(), (256, 256, 512), run_ids=ids, seed=0, t_end=50.0, snap_times=snaps,
                   threads=THREADS)
    sub = {k: g[k][ids] for k in ("final_counts", "outcome", "t_abs")}
    assert_parity(sub, r, snaps=False, min_ok=0.95)
    fc = g["final_counts"]
    assert np.all(fc.sum(1) == 1024)
    absorbed = g["outcome"] >= 0
    assert np.all((fc[absorbed] > 0).sum(1) == 1)
    assert np.all(g["ee_hist"].sum(1) == n)
    assert g["counters"]["absorbed"] == absorbed.sum()
    pL, pD = np.mean(g["outcome"] == 0), np.mean(g["outcome"] == 1)
    assert abs(pL - pD) < 5 * math.sqrt((pL + pD) / n)


@pytest.mark.parametrize("mode,omode,rtol,tie", [
    (pkg.SSA_P64_LOGSUM, oracle.P64, 1e-12, 1e-12),
    (pkg.SSA_P32_KAHAN, oracle.P32_KAHAN, 2e-5, 1e-6),
    (pkg.SSA_P32_D64ACC, oracle.P32_D64ACC, 2e-5, 1e-6),
    (pkg.SSA_P32_PLAIN, oracle.P32_PLAIN, 2e-5, 1e-6),
])
@pytest.mark.parametrize("pad", [0, 1], ids=["paper_bound", "padded"])
@LAYOUTS
def test_parity_precision_modes(mode, omode, rtol, tie, pad, layout):
    """fp32 clocks: CUDA's logf and the host's may differ by an ulp, so event times agree to
    ~1e-7 relative; runs with an event within `tie` of a snapshot are left out of the
    count comparison (several percent of runs at 10 snapshots)."""
    snaps = log_snapshots(50.0, 10)
    n = 1024 + 5
    g = gpu_run((256, 256, 512), n, seed=3, t_end=50.0, snaps=snaps, precision=mode, layout=layout, pad_pow2=pad)
    r = oracle.run(oracle.frank(), (256, 256, 512), n, seed=3, t_end=50.0, snap_times=snaps,
                   precision=omode, threads=THREADS, pad_pow2=bool(pad))
    assert_parity(g, r, rtol=rtol, tie=tie, min_ok=0.95)


def test_results_do_not_depend_on_launch_shape():
    """Block size and resident blocks of the one-thread layout, resident blocks of the
    three-warp layout, and the layout itself: every output identical."""
    snaps = [0.005, 0.02]
    base = gpu_run((256, 256, 512), 3000, seed=5, t_end=0.05, snaps=snaps, layout=pkg.SSA_LAYOUT_THREAD)
    shapes = [dict(layout=pkg.SSA_LAYOUT_THREAD, block_size=b, blocks_per_sm=m) for b, m in
              [(32, 1), (128, 0), (256, 1)]]
    shapes += [dict(layout=pkg.SSA_LAYOUT_WARPS, blocks_per_sm=m) for m in (0, 1, 2)]
    for shape in shapes:
        g = gpu_run((256, 256, 512), 3000, seed=5, t_end=0.05, snaps=snaps, **shape)
        for k in ("final_counts", "outcome", "t_abs", "ee_hist", "snap_counts"):
            assert np.array_equal(g[k], base[k]), (shape, k)
        assert same_counters(g, base), shape


@pytest.mark.parametrize("init,n,t_end,seed", [((256, 256, 512), 1 << 16, 50.0, 21),
                                               ((3, 3, 6), 5000, 5.0, 22),
                                               ((1000, 0, 3000), 3000, 1.0, 23)])
def test_layouts_agree_bit_for_bit(init, n, t_end, seed):
    """The same context on both layouts: counts, times, histograms and every counter equal."""
    snaps = log_snapshots(t_end, 6)
    a = gpu_run(init, n, seed=seed, t_end=t_end, snaps=snaps, layout=pkg.SSA_LAYOUT_THREAD)
    b = gpu_run(init, n, seed=seed, t_end=t_end, snaps=snaps, layout=pkg.SSA_LAYOUT_WARPS)
    for k in ("final_counts", "outcome", "t_abs", "ee_hist", "snap_counts"):
        assert np.array_equal(a[k], b[k]), k
    assert same_counters(a, b)
    assert (a["counters"]["layout"] & 3, b["counters"]["layout"]) == (pkg.SSA_LAYOUT_THREAD, pkg.SSA_LAYOUT_WARPS)


@LAYOUTS
def test_sharded_contexts_equal_one_context(layout):
    """Two contexts holding runs [0, 2048) and [2048, 4096) (first_run) give the runs of one
    context of 4096: the stream is keyed by the global group index."""
    snaps = [0.01, 0.03]
    whole = gpu_run((256, 256, 512), 4096, seed=9, t_end=0.1, snaps=snaps, layout=layout)
    a = gpu_run((256, 256, 512), 2048, seed=9, t_end=0.1, snaps=snaps, first_run=0, layout=layout)
    b = gpu_run((256, 256, 512), 2048, seed=9, t_end=0.1, snaps=snaps, first_run=2048, layout=layout)
    for k in ("final_counts", "outcome", "t_abs"):
        assert np.array_equal(np.concatenate([a[k], b[k]]), whole[k]), k
    assert np.array_equal(a["ee_hist"] + b["ee_hist"], whole["ee_hist"])


@LAYOUTS
def test_parity_per_run_initial_states(layout):
    """Independent multinomial initial states around the racemic point (Sec. 5, Fig. 4)."""
    rng = np.random.default_rng(77)
    n = 2000
    init = rng.multinomial(256, [0.25, 0.25, 0.5], size=n)
    snaps = [0.01, 0.05]
    g = gpu_run(init, n, seed=4, t_end=1.0, snaps=snaps, layout=layout)
    r = oracle.run(oracle.frank(), init, seed=4, t_end=1.0, snap_times=snaps, threads=THREADS)
    assert_parity(g, r)


@LAYOUTS
def test_relabelled_species_give_the_same_runs(layout):
    """Species order (A, L, D) with the reactions in Frank's order: the same trajectories,
    reported in the caller's species order."""
    reac = [[1, 1, 0], [1, 0, 1], [0, 1, 1]]
    prod = [[0, 2, 0], [0, 0, 2], [2, 0, 0]]
    snaps = [0.02]
    base = gpu_run((16, 16, 32), 256, seed=6, t_end=1.0, snaps=snaps, layout=layout)
    g = gpu_run((32, 16, 16), 256, seed=6, t_end=1.0, snaps=snaps, reac=reac, prod=prod, layout=layout)
    assert np.array_equal(g["final_counts"][:, [1, 2, 0]], base["final_counts"])
    assert np.array_equal(g["snap_counts"][:, :, [1, 2, 0]], base["snap_counts"])
    remap = np.array([-2, -1, 2, 0, 1])  # caller's outcome -2..2 (A=0, L=1, D=2) -> (L=0, D=1, A=2)
    assert np.array_equal(remap[g["outcome"] + 2], base["outcome"])


@pytest.mark.parametrize("rates,q", [((1.0, 0.5, 0.25), 32), ((0.7, 2.0, 1.3), 64), ((0.0, 0.0, 1.0), 32),
                                     ((1.0, 1.0, 0.5), 5)])
@LAYOUTS
def test_parity_thinning(rates, q, layout):
    snaps = [0.01, 0.1]
    n = 1024 + 3
    g = gpu_run((64, 64, 128), n, seed=12, t_end=2.0, snaps=snaps, rates=rates, thin_bits=q, layout=layout)
    r = oracle.run(oracle.frank(*rates), (64, 64, 128), n, seed=12, t_end=2.0, snap_times=snaps,
                   thin_bits=q, threads=THREADS)
    assert_parity(g, r)


# --------------------------------------------------------------------------
# Edge cases
# --------------------------------------------------------------------------
def test_empty_context():
    g = gpu_run((16, 16, 32), 0, t_end=1.0, snaps=[0.5])
    assert g["final_counts"].size == 0 and g["ee_hist"].sum() == 0


@pytest.mark.parametrize("init", [(1, 0, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 0, 50), (25, 0, 0),
                                  (2, 1, 0)])
@LAYOUTS
def test_small_and_absorbed_systems(init, layout):
    n = 70
    snaps = [0.0, 0.5, 3.0]
    g = gpu_run(init, n, seed=2, t_end=3.0, snaps=snaps, layout=layout)
    r = oracle.run(oracle.frank(), init, n, seed=2, t_end=3.0, snap_times=snaps)
    assert_parity(g, r)


@LAYOUTS
def test_t_end_zero_and_snapshot_at_t_end(layout):
    g = gpu_run((10, 10, 10), 40, seed=1, t_end=0.0, snaps=[0.0], layout=layout)
    assert np.all(g["final_counts"] == [10, 10, 10]) and np.all(g["outcome"] == -1)
    assert np.all(np.isinf(g["t_abs"])) and np.all(g["snap_counts"] == [10, 10, 10])
    snaps = [0.02, 0.04]
    g = gpu_run((16, 16, 32), 96, seed=1, t_end=0.04, snaps=snaps, layout=layout)
    r = oracle.run(oracle.frank(), (16, 16, 32), 96, seed=1, t_end=0.04, snap_times=snaps)
    assert_parity(g, r)
    assert np.array_equal(g["snap_counts"][1], g["final_counts"])


@LAYOUTS
def test_step_budget_reports_timeout(layout):
    g = gpu_run((256, 256, 512), 64, seed=1, t_end=50.0, step_budget=100, expect_status=pkg.SSA_ETIMEOUT, layout=layout)
    assert g["counters"]["group_steps"] == 2 * 100
    r = oracle.run(oracle.frank(), (256, 256, 512), 64, seed=1, t_end=50.0, step_budget=100, check=False)
    assert np.array_equal(g["final_counts"], r["final_counts"])


def test_fetch_before_run_is_a_state_error():
    ctx = pkg.ssa_create(FRANK_R, FRANK_P, [1, 1, 1], (16, 16, 32), 32, 0)
    try:
        with pytest.raises(pkg.SSAError) as ei:
            pkg.ssa_fetch(ctx, pkg.SSA_FIELD_FINAL_COUNTS)
        assert ei.value.status == pkg.SSA_ESTATE
    finally:
        pkg.ssa_destroy(ctx)


def test_repeated_runs_are_identical():
    import torch
    o = pkg.ssa_default_options(cuda_stream=torch.cuda.current_stream())
    ctx = pkg.ssa_create(FRANK_R, FRANK_P, [1, 1, 1], (64, 64, 128), 5000, 3, o)
    try:
        pkg.ssa_run(ctx, 1.0, [0.01])
        a = pkg.fetch_all(ctx)
        pkg.ssa_run(ctx, 1.0, [0.01])
        b = pkg.fetch_all(ctx)
        dev = torch.empty(5000 * 3, dtype=torch.int32, device="cuda")
        pkg.ssa_fetch(ctx, pkg.SSA_FIELD_FINAL_COUNTS, dev)
    finally:
        pkg.ssa_destroy(ctx)
    for k in ("final_counts", "t_abs", "outcome", "ee_hist"):
        assert np.array_equal(a[k], b[k])
    assert a["counters"] == b["counters"]
    assert np.array_equal(dev.cpu().numpy().reshape(-1, 3), a["final_counts"])


# --------------------------------------------------------------------------
# The one-thread-per-run baseline samples the same process
# --------------------------------------------------------------------------
def test_thread_per_run_baseline_distribution():
    n = 200_000
    g = gpu_run((16, 16, 32), n, seed=8, t_end=np.inf, engine=pkg.SSA_ENGINE_THREAD_PER_RUN)
    r = oracle.run(oracle.frank(), (16, 16, 32), run_ids=np.arange(20_000) * 32, seed=8, t_end=np.inf,
                   threads=THREADS)
    assert np.all(g["outcome"] >= 0)
    assert np.all(g["final_counts"].sum(1) == 64)
    pL = np.mean(g["outcome"] == 0)
    pL_ref = np.mean(r["outcome"] == 0)
    assert abs(pL - pL_ref) < 5 * math.sqrt(0.25 / n + 0.25 / len(r["outcome"]))
    se = math.sqrt(g["t_abs"].var() / n + r["t_abs"].var() / len(r["t_abs"]))
    assert abs(g["t_abs"].mean() - r["t_abs"].mean()) < 5 * se
    assert g["counters"]["reactions"] > 0


def test_tuner_keeps_the_runs():
    """ssa_tune times each configuration and keeps the fastest; the runs after it equal an
    untuned context's, and the choice is one of the offered configurations."""
    import torch
    snaps = [0.01, 0.1]
    base = gpu_run((64, 64, 128), 3000, seed=8, t_end=1.0, snaps=snaps)
    o = pkg.ssa_default_options(cuda_stream=torch.cuda.current_stream(), keep_snap_counts=1)
    ctx = pkg.ssa_create(FRANK_R, FRANK_P, [1, 1, 1], (64, 64, 128), 3000, 8, o)
    try:
        for probe in (200, 0):
            layout, block = pkg.ssa_tune(ctx, 1.0, snaps, probe_steps=probe)
            assert (layout, block) in [(pkg.SSA_LAYOUT_AUTO, 64), (pkg.SSA_LAYOUT_THREAD, 32),
                                       (pkg.SSA_LAYOUT_THREAD, 64), (pkg.SSA_LAYOUT_THREAD, 128),
                                       (pkg.SSA_LAYOUT_WARPS, 64)]
            with pytest.raises(pkg.SSAError) as ei:
                pkg.ssa_fetch(ctx, pkg.SSA_FIELD_FINAL_COUNTS)
            assert ei.value.status == pkg.SSA_ESTATE
            pkg.ssa_run(ctx, 1.0, snaps)
            g = pkg.fetch_all(ctx, snapshots=True)
            g["snap_counts"] = g["snap_counts"].reshape(len(snaps), 3000, 3)
            for k in ("final_counts", "outcome", "t_abs", "ee_hist", "snap_counts"):
                assert np.array_equal(g[k], base[k]), (probe, k)
            assert same_counters(g, base)
    finally:
        pkg.ssa_destroy(ctx)


@pytest.mark.parametrize("layout", [pkg.SSA_LAYOUT_AUTO, pkg.SSA_LAYOUT_WARPS], ids=["auto", "warps"])
def test_parity_shared_n(layout):
    """The paper's shared draw (one n per group, Sec. 4 step a) against the oracle, with
    multinomial initial states per run (Sec. 5, Fig. 4) and a thinned rate; it runs on the
    three-warp layout, which the automatic choice takes for it."""
    rng = np.random.default_rng(31)
    n = 1024 + 7
    init = rng.multinomial(512, [0.25, 0.25, 0.5], size=n)
    snaps = [0.005, 0.05, 0.5]
    for rates in ((1.0, 1.0, 1.0), (1.0, 0.6, 1.0)):
        g = gpu_run(init, n, seed=13, t_end=2.0, snaps=snaps, rates=rates, shared_n=1, layout=layout)
        r = oracle.run(oracle.frank(*rates), init, seed=13, t_end=2.0, snap_times=snaps, shared_n=True,
                       threads=THREADS)
        assert_parity(g, r)


def test_shared_n_identical_start_gives_identical_lanes():
    g = gpu_run((64, 64, 128), 128, seed=2, t_end=3.0, snaps=[0.1], shared_n=1)
    assert g["counters"]["layout"] == pkg.SSA_LAYOUT_WARPS
    for grp in range(4):
        sl = slice(32 * grp, 32 * grp + 32)
        assert np.all(g["final_counts"][sl] == g["final_counts"][32 * grp])
        assert np.all(g["t_abs"][sl] == g["t_abs"][32 * grp])


@LAYOUTS
@pytest.mark.parametrize("N,rates", [(46400, (1.0, 1.0, 1.0)), (10000, (0.7, 1.3, 1.9)), (65536, (1.0, 1.0, 1.0))])
def test_parity_wide_n(N, rates, layout):
    """K = 26..31: the wide-n redraw (calls from the top, two at a time), including N_tot = 46 400,
    where half of all draws are rejected, against the oracle over ~10^4 steps per run."""
    init = (N // 4, N // 4, N - 2 * (N // 4))
    lam = N * (N - 1) / 2 * max(rates)
    t_end = 1.2e4 / lam
    snaps = [t_end / 3, 2 * t_end / 3]
    n = 96 + 5
    g = gpu_run(init, n, seed=17, t_end=t_end, snaps=snaps, rates=rates, layout=layout)
    r = oracle.run(oracle.frank(*rates), init, n, seed=17, t_end=t_end, snap_times=snaps, threads=THREADS)
    assert_parity(g, r)
    assert g["counters"]["redraw_rounds"] > 0


@LAYOUTS
@pytest.mark.parametrize("N,rates", [(1024, (1.0, 1.0, 1.0)), (46400, (1.0, 1.0, 1.0)), (10000, (0.7, 1.3, 1.9)),
                                     (12, (1.0, 0.5, 2.0))])
def test_parity_padded_bound(N, rates, layout):
    """pad_pow2: the bound raised to 2^K (null events above N (N - 1) / 2), so no draw is
    rejected; runs, snapshots and counters against the oracle in the same mode."""
    init = (N // 4, N // 4, N - 2 * (N // 4))
    lam = 2 ** (N * (N - 1) // 2).bit_length() * max(rates)
    t_end = 1.2e4 / lam if N > 64 else 50.0
    snaps = [t_end / 3, 2 * t_end / 3]
    n = 96 + 5
    g = gpu_run(init, n, seed=29, t_end=t_end, snaps=snaps, rates=rates, layout=layout, pad_pow2=1)
    r = oracle.run(oracle.frank(*rates), init, n, seed=29, t_end=t_end, snap_times=snaps, threads=THREADS,
                   pad_pow2=True)
    ok = assert_parity(g, r)
    assert_hist_parity(g, r, ok)
    assert g["counters"]["redraw_rounds"] == 0 and r["redraws"].sum() == 0
    assert ok.all()  # at this seed the oracle reports no event within 1e-12 of a snapshot or t_end
    assert np.array_equal(g["ee_hist"], oracle.ee_histogram(r["snap_counts"]))
    assert g["counters"]["lane_steps"] == r["steps"].sum()
    assert g["counters"]["reactions"] == r["reactions"].sum()


def test_parity_padded_bound_shared_n():
    """The paper's shared draw with the padded bound (three-warp layout)."""
    rng = np.random.default_rng(37)
    n = 256 + 3
    init = rng.multinomial(300, [0.25, 0.25, 0.5], size=n)
    g = gpu_run(init, n, seed=5, t_end=2.0, snaps=[0.01, 0.1], shared_n=1, pad_pow2=1)
    r = oracle.run(oracle.frank(), init, seed=5, t_end=2.0, snap_times=[0.01, 0.1], shared_n=True,
                   pad_pow2=True, threads=THREADS)
    assert_parity(g, r)


@LAYOUTS
def test_a_later_t_end_extends_the_same_runs(layout):
    """A run is a fixed function of its stream: the final counts of a run stopped at t1 are the
    snapshot at t1 of the same run continued to t2 > t1 (absorbed runs: the same t_abs)."""
    t1, t2 = 0.01, 0.05
    a = gpu_run((256, 256, 512), 2048, seed=9, t_end=t1, layout=layout, pad_pow2=1)
    b = gpu_run((256, 256, 512), 2048, seed=9, t_end=t2, snaps=[t1], layout=layout, pad_pow2=1)
    assert np.array_equal(a["final_counts"], b["snap_counts"][0])
    done = np.isfinite(a["t_abs"])
    assert np.array_equal(a["t_abs"][done], b["t_abs"][done])


TAIL_CASES = [
    dict(init=(256, 256, 512), n=4096 + 17, t_end=50.0, seed=41, snaps=log_snapshots(50.0, 10)),
    dict(init=(256, 256, 512), n=4096 + 17, t_end=50.0, seed=41, snaps=log_snapshots(50.0, 10), pad_pow2=1),
    dict(init=(256, 256, 512), n=2048 + 3, t_end=50.0, seed=42, snaps=log_snapshots(50.0, 6), pad_pow2=2),
    dict(init=(256, 256, 512), n=2048 + 3, t_end=50.0, seed=43, snaps=log_snapshots(50.0, 6),
         precision=pkg.SSA_P32_KAHAN),
    dict(init=(256, 256, 512), n=2048, t_end=50.0, seed=44, snaps=[0.01, 0.1], precision=pkg.SSA_P64_LOGSUM),
    dict(init=(2500, 2500, 5000), n=1024 + 1, t_end=0.002, seed=45, snaps=[0.0005, 0.001]),
    dict(init=(11600, 11600, 23200), n=512 + 9, t_end=5e-6, seed=46, snaps=[1e-6, 3e-6]),
    dict(init=(3, 3, 6), n=3000, t_end=5.0, seed=47, snaps=[0.1, 1.0]),
    dict(init=(256, 256, 512), n=4096, t_end=0.03, seed=48, snaps=[0.01, 0.02]),
]


@pytest.mark.parametrize("case", range(len(TAIL_CASES)))
@pytest.mark.parametrize("block", [32, 128])
def test_tail_hand_off_keeps_the_runs(case, block):
    """The one-thread kernel's tail hand-off (the last groups of a warp finished one run per
    thread) gives every run, snapshot, histogram, absorption time and counter of the kernel
    without it, bit for bit: paper's, padded and state-following bounds, every clock, wide n with
    heavy rejection (N = 46 400), t_end before absorption, and a hand-off threshold of 1 and 4."""
    kw = dict(TAIL_CASES[case])
    init, n, t_end, seed, snaps = kw.pop("init"), kw.pop("n"), kw.pop("t_end"), kw.pop("seed"), kw.pop("snaps")
    base = gpu_run(init, n, seed=seed, t_end=t_end, snaps=snaps, layout=pkg.SSA_LAYOUT_THREAD, block_size=block,
                   tail_groups=-1, **kw)
    assert not base["counters"]["layout"] & 16
    for tail in (4, 1):
        g = gpu_run(init, n, seed=seed, t_end=t_end, snaps=snaps, layout=pkg.SSA_LAYOUT_THREAD, block_size=block,
                    tail_groups=tail, **kw)
        assert g["counters"]["layout"] & 16, tail
        for k in ("final_counts", "outcome", "t_abs", "ee_hist", "snap_counts", "ens_absorbed"):
            assert np.array_equal(g[k], base[k]), (tail, k)
        assert same_counters(g, base), (tail, g["counters"], base["counters"])


def test_tail_hand_off_on_a_batch():
    """A batch of ensembles with different N_tot and seeds: the tail hand-off keeps every run."""
    import torch
    init = np.array([[16, 16, 32], [256, 256, 512], [100, 60, 340], [2500, 2500, 5000]])
    runs = np.array([100, 2048, 777, 513])
    seeds = np.array([3, 4, 5, 6], dtype=np.uint64)
    out = []
    for tail in (-1, 4):
        o = pkg.ssa_default_options(cuda_stream=torch.cuda.current_stream(), layout=pkg.SSA_LAYOUT_THREAD,
                                    tail_groups=tail, keep_snap_counts=1)
        ctx = pkg.ssa_create_batch(FRANK_R, FRANK_P, init, np.ones((4, 3)), runs, seeds, o)
        try:
            pkg.ssa_run(ctx, 1.0, [0.001, 0.01])
            out.append(pkg.fetch_all(ctx, snapshots=True))
        finally:
            pkg.ssa_destroy(ctx)
    for k in ("final_counts", "outcome", "t_abs", "ee_hist", "snap_counts", "ens_absorbed"):
        assert np.array_equal(out[0][k], out[1][k]), k
    assert same_counters(out[0], out[1])
    assert out[1]["counters"]["layout"] & 16


def test_tail_hand_off_with_groups_absorbed_at_start():
    """Per-run initial states where whole groups start absorbed (a single species) next to groups
    that run, to absorption (t_end = inf): the hand-off finishes the absorbed groups first and the
    runs equal those without it and the oracle's."""
    rng = np.random.default_rng(91)
    n = 32 * 9 + 5
    init = rng.multinomial(128, [0.25, 0.25, 0.5], size=n)
    init[0:32] = (128, 0, 0)
    init[64:96] = (0, 0, 128)
    init[200:232] = (0, 128, 0)
    snaps = [0.001, 0.01, 0.1]
    base = gpu_run(init, n, seed=5, t_end=np.inf, snaps=snaps, layout=pkg.SSA_LAYOUT_THREAD, tail_groups=-1)
    g = gpu_run(init, n, seed=5, t_end=np.inf, snaps=snaps, layout=pkg.SSA_LAYOUT_THREAD, tail_groups=4)
    assert g["counters"]["layout"] & 16
    for k in ("final_counts", "outcome", "t_abs", "ee_hist", "snap_counts", "ens_absorbed"):
        assert np.array_equal(g[k], base[k]), k
    assert same_counters(g, base)
    r = oracle.run(oracle.frank(), init, seed=5, t_end=np.inf, snap_times=snaps, threads=THREADS)
    assert_parity(g, r)
