"""GPU parity of the general-network kernel: any conserved network of order <= 2 with up to
8 species and 8 reactions, propensities recomputed every step by bit-sliced products
(Sec. 4.1), against the CPU oracle on the same seeded inputs; and Frank's model on the
general kernel against Frank's own kernels, bit for bit."""
import os

import numpy as np
import pytest

import oracle
import paper_2412_16613_gb300 as pkg
from tests._gpu import FRANK_P, FRANK_R, assert_parity, gpu_run, log_snapshots

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4
GENERAL = pkg.SSA_ENGINE_GENERAL


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


# name: (reactants, products, rates, initial counts, t_end)
NETWORKS = {
    # two reactions on one pair (m_pair = 2): the Moran / voter model
    "moran": ([[1, 1], [1, 1]], [[2, 0], [0, 2]], [1.0, 1.0], (40, 60), 5.0),
    # S + I -> 2I, I -> R: a first-order reaction (u_max = 1) next to a pair
    "sir": ([[1, 1, 0], [0, 1, 0]], [[0, 2, 0], [0, 0, 1]], [1.0, 3.0], (190, 10, 0), 2.0),
    # 2A -> A + B, A + B -> 2A, B -> A: a homodimer, a pair, a first-order reaction, thinning
    "dimer": ([[2, 0], [1, 1], [0, 1]], [[1, 1], [2, 0], [1, 0]], [1.0, 0.5, 3.0], (70, 30), 0.5),
    # four species, four reactions, a zero rate
    "four": ([[1, 1, 0, 0], [0, 0, 1, 1], [0, 1, 0, 0], [0, 0, 2, 0]],
             [[0, 0, 2, 0], [2, 0, 0, 0], [0, 0, 0, 1], [1, 1, 0, 0]],
             [1.0, 0.8, 5.0, 0.0], (30, 30, 20, 20), 1.0),
    # first order only: N_tot = 50 000 needs more count planes than K = 16 products would read
    "isomer": ([[1, 0], [0, 1]], [[0, 1], [1, 0]], [1.0, 0.25], (50000, 0), 0.05),
    # one species, a reaction that changes nothing: never absorbs
    "null": ([[2]], [[2]], [1.0], (9,), 3.0),
}


def _oracle_net(reac, prod, rates):
    return oracle.Network(reac, prod, rates)


def _layout(reac, recompute):
    """The layout word the general kernel reports: incremented (4) or recomputed (8) propensities,
    and the planes in registers (32) for incremental mode on a network of at most 4 species and 4
    reactions with a reaction of order 2 (its counts then fit the planes the products read)."""
    if recompute == 1:
        return pkg.SSA_LAYOUT_THREAD | 8
    small = len(reac) <= 4 and len(reac[0]) <= 4 and max(sum(r) for r in reac) == 2
    return pkg.SSA_LAYOUT_THREAD | 4 | (32 if small and recompute != 3 else 0)


def _check(g, r, S, snaps):
    ok = assert_parity(g, r)
    assert np.all(g["final_counts"].sum(1) == r["final_counts"].sum(1))
    if ok.all():
        assert g["counters"]["reactions"] == r["reactions"].sum()
        assert g["counters"]["lane_steps"] == r["steps"].sum()
        if S >= 2 and len(snaps):
            assert np.array_equal(g["ee_hist"], oracle.ee_histogram(r["snap_counts"], 0, 1))
    return ok


@pytest.mark.parametrize("name", sorted(NETWORKS))
@pytest.mark.parametrize("pad,recompute", [(0, 0), (1, 0), (0, 1), (1, 1), (1, 2), (0, 3), (1, 3)])
def test_general_network_parity(name, pad, recompute):
    """Every run, snapshot and histogram, 3 groups and a ragged tail, against the oracle, with the
    propensities kept and incremented (default; planes in registers where the network fits, in
    shared memory with recompute = 3) or recomputed by products every step."""
    reac, prod, rates, init, t_end = NETWORKS[name]
    S = len(init)
    snaps = [t_end / 10, t_end / 3, t_end / 2]
    n = 96 + 7
    g = gpu_run(init, n, seed=41, t_end=t_end, snaps=snaps, rates=rates, reac=reac, prod=prod, pad_pow2=pad,
                recompute=recompute)
    r = oracle.run(_oracle_net(reac, prod, rates), init, n, seed=41, t_end=t_end, snap_times=snaps,
                   threads=THREADS, pad_pow2=bool(pad))
    _check(g, r, S, snaps)
    assert g["counters"]["layout"] == _layout(reac, recompute)
    if pad:
        assert g["counters"]["redraw_rounds"] == 0


@pytest.mark.parametrize("N,regs", [(1700, True), (2500, False)])
def test_general_register_plane_limit(N, regs):
    """Moran at N_tot = 1700 (lambda_int = N (N - 1) has K = 22 planes, the most a thread keeps in
    registers) and 2500 (K = 23, shared memory): every run and snapshot against the oracle, and
    the layout bit of the mode that ran."""
    reac, prod, rates, _, _ = NETWORKS["moran"]
    init = (N // 2, N - N // 2)
    t_end = 2e-3
    snaps = [t_end / 2]
    n = 64 + 5
    g = gpu_run(init, n, seed=23, t_end=t_end, snaps=snaps, rates=rates, reac=reac, prod=prod, pad_pow2=1)
    r = oracle.run(_oracle_net(reac, prod, rates), init, n, seed=23, t_end=t_end, snap_times=snaps,
                   threads=THREADS, pad_pow2=True)
    _check(g, r, 2, snaps)
    assert g["counters"]["layout"] == pkg.SSA_LAYOUT_THREAD | 4 | (32 if regs else 0)
    assert g["counters"]["reactions"] > 0


@pytest.mark.parametrize("name", ["moran", "sir", "four"])
def test_general_per_run_initial_states(name):
    reac, prod, rates, init, t_end = NETWORKS[name]
    rng = np.random.default_rng(3)
    n = 64 + 9
    tot = sum(init)
    init_runs = rng.multinomial(tot, np.full(len(init), 1.0 / len(init)), size=n)
    snaps = [t_end / 4]
    g = gpu_run(init_runs, n, seed=5, t_end=t_end, snaps=snaps, rates=rates, reac=reac, prod=prod)
    r = oracle.run(_oracle_net(reac, prod, rates), init_runs, seed=5, t_end=t_end, snap_times=snaps,
                   threads=THREADS)
    _check(g, r, len(init), snaps)


def test_general_shared_draw():
    """The paper's shared draw on the general kernel (one thread per group)."""
    reac, prod, rates, init, t_end = NETWORKS["dimer"]
    rng = np.random.default_rng(8)
    n = 96
    init_runs = rng.multinomial(100, [0.5, 0.5], size=n)
    g = gpu_run(init_runs, n, seed=12, t_end=t_end, snaps=[0.1], rates=rates, reac=reac, prod=prod, shared_n=1)
    r = oracle.run(_oracle_net(reac, prod, rates), init_runs, seed=12, t_end=t_end, snap_times=[0.1],
                   shared_n=True, threads=THREADS)
    _check(g, r, 2, [0.1])


def test_general_absorption_to_completion():
    """Moran runs to fixation (t_end = inf): every run absorbed, outcome and time as the oracle."""
    reac, prod, rates, _, _ = NETWORKS["moran"]
    n = 256
    g = gpu_run((20, 30), n, seed=2, rates=rates, reac=reac, prod=prod)
    r = oracle.run(_oracle_net(reac, prod, rates), (20, 30), n, seed=2, threads=THREADS)
    _check(g, r, 2, [])
    assert np.all(g["outcome"] >= 0)
    assert g["counters"]["absorbed"] == n
    tally = g["ens_absorbed"][0]
    assert tally[0] == np.sum(g["outcome"] == 0) and tally[1] == np.sum(g["outcome"] == 1)


def test_general_batch_against_oracle():
    """A batch of one network with per-ensemble totals, rates and seeds."""
    reac, prod, _, _, _ = NETWORKS["dimer"]
    N0 = np.array([[70, 30], [5, 1], [600, 400], [2000, 0]])
    rates = np.array([[1.0, 0.5, 3.0], [1.0, 1.0, 1.0], [0.3, 2.0, 0.1], [1.0, 0.7, 0.0]])
    runs = np.array([40, 33, 64, 32])
    seeds = np.array([9, 10, 11, 12], dtype=np.uint64)
    t_end = 0.05
    snaps = [0.01, 0.03]
    import torch
    o = pkg.ssa_default_options(cuda_stream=torch.cuda.current_stream(), keep_snap_counts=1)
    ctx = pkg.ssa_create_batch(reac, prod, N0, rates, runs, seeds, o)
    try:
        pkg.ssa_run(ctx, t_end, snaps)
        g = pkg.fetch_all(ctx, n_species=2, snapshots=True)
    finally:
        pkg.ssa_destroy(ctx)
    snap_all = g["snap_counts"].reshape(len(snaps), -1, 2)
    hist = g["ee_hist"].reshape(len(N0), len(snaps), 65)
    off = 0
    for e in range(len(N0)):
        r = oracle.run(_oracle_net(reac, prod, rates[e]), N0[e], int(runs[e]), seed=int(seeds[e]), t_end=t_end,
                       snap_times=snaps, threads=THREADS)
        sl = slice(off, off + runs[e])
        sub = {"final_counts": g["final_counts"][sl], "outcome": g["outcome"][sl], "t_abs": g["t_abs"][sl],
               "snap_counts": snap_all[:, sl]}
        ok = assert_parity(sub, r)
        if ok.all():
            assert np.array_equal(hist[e], oracle.ee_histogram(r["snap_counts"], 0, 1))
        off += runs[e]


@pytest.mark.parametrize("recompute", [0, 1, 3])
@pytest.mark.parametrize("init,n,rates,pad", [((16, 16, 32), 64, (1.0, 1.0, 1.0), 0),
                                              ((256, 256, 512), 4096 + 17, (1.0, 1.0, 1.0), 1),
                                              ((256, 256, 512), 2048, (0.7, 1.0, 1.6), 0),
                                              ((2500, 2500, 5000), 256, (1.0, 1.0, 1.0), 0)])
def test_frank_on_general_kernel_equals_frank_kernel(init, n, rates, pad, recompute):
    """Frank's model through the general kernel gives Frank's kernel's runs bit for bit: the
    same stream and rule, with the propensities incremented by the general rule (planes in
    registers up to K = 22, or in shared memory) or recomputed by products instead of Frank's
    hand-derived increments."""
    N = sum(init)
    t_end = 50.0 if N <= 1024 else 3e-4
    snaps = log_snapshots(t_end, 6)
    a = gpu_run(init, n, seed=7, t_end=t_end, snaps=snaps, rates=rates, pad_pow2=pad,
                layout=pkg.SSA_LAYOUT_THREAD)
    b = gpu_run(init, n, seed=7, t_end=t_end, snaps=snaps, rates=rates, pad_pow2=pad, engine=GENERAL,
                recompute=recompute)
    for k in ("final_counts", "outcome", "ee_hist", "snap_counts", "ens_absorbed"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["t_abs"], b["t_abs"])
    assert {k: v for k, v in a["counters"].items() if k != "layout"} == \
        {k: v for k, v in b["counters"].items() if k != "layout"}


def test_frank_relabelled_on_general_kernel():
    """Species order (A, L, D) on the general engine: the same runs as Frank's kernel, and the
    histogram bins Frank's L and D."""
    reac = [[1, 1, 0], [1, 0, 1], [0, 1, 1]]
    prod = [[0, 2, 0], [0, 0, 2], [2, 0, 0]]
    snaps = [0.01, 0.1]
    a = gpu_run((32, 16, 16), 96, seed=4, t_end=5.0, snaps=snaps, reac=reac, prod=prod)
    b = gpu_run((32, 16, 16), 96, seed=4, t_end=5.0, snaps=snaps, reac=reac, prod=prod, engine=GENERAL)
    for k in ("final_counts", "outcome", "t_abs", "ee_hist", "snap_counts"):
        assert np.array_equal(a[k], b[k]), k


def test_general_step_budget_and_t_end_zero():
    reac, prod, rates, init, _ = NETWORKS["sir"]
    g = gpu_run(init, 64, seed=1, t_end=10.0, rates=rates, reac=reac, prod=prod, step_budget=5,
                expect_status=pkg.SSA_ETIMEOUT)
    assert g["counters"]["max_group_steps"] == 5
    g = gpu_run(init, 64, seed=1, t_end=0.0, snaps=[0.0], rates=rates, reac=reac, prod=prod)
    assert np.all(g["final_counts"] == init) and g["counters"]["group_steps"] == 0


def test_tuner_picks_a_general_mode_and_keeps_the_runs():
    """ssa_tune on a general network times blocks of 32/64/128 with the propensities incremented
    and recomputed; the runs after tuning are the runs before it."""
    import torch
    reac, prod, rates, init, t_end = NETWORKS["dimer"]
    o = pkg.ssa_default_options(cuda_stream=torch.cuda.current_stream(), keep_snap_counts=1, pad_pow2=1)
    ctx = pkg.ssa_create(reac, prod, rates, init, 2048, 3, o)
    try:
        pkg.ssa_run(ctx, t_end, [0.1])
        before = pkg.fetch_all(ctx, n_species=2, snapshots=True)
        layout, block = pkg.ssa_tune(ctx, t_end, [0.1])
        assert layout == pkg.SSA_LAYOUT_THREAD and block in (32, 64, 128)
        pkg.ssa_run(ctx, t_end, [0.1])
        after = pkg.fetch_all(ctx, n_species=2, snapshots=True)
    finally:
        pkg.ssa_destroy(ctx)
    for k in ("final_counts", "outcome", "t_abs", "ee_hist", "snap_counts"):
        assert np.array_equal(before[k], after[k]), k
    assert after["counters"]["layout"] in (pkg.SSA_LAYOUT_THREAD | 4 | 32, pkg.SSA_LAYOUT_THREAD | 8)


@pytest.mark.parametrize("pad,recompute", [(0, 2), (1, 2), (1, 1)])
def test_general_maximum_sizes(pad, recompute):
    """8 species and 8 reactions (a ring X_i + X_{i+1} -> 2 X_{i+1}) at N_tot = 65536: K = 31,
    17 count planes, the largest shared-memory layout (more than the default 48 KB a block)."""
    S = 8
    reac = [[1 if j in (i, (i + 1) % S) else 0 for j in range(S)] for i in range(S)]
    prod = [[2 if j == (i + 1) % S else 0 for j in range(S)] for i in range(S)]
    rates = [1.0, 0.9, 0.8, 0.7, 1.0, 0.6, 0.5, 0.4]
    init = (8192,) * S
    N = sum(init)
    lam = (2 ** 31 if pad else N * (N - 1) // 2) * max(rates)
    t_end = 3000 / lam
    snaps = [t_end / 2]
    n = 64 + 5
    g = gpu_run(init, n, seed=19, t_end=t_end, snaps=snaps, rates=rates, reac=reac, prod=prod, pad_pow2=pad,
                recompute=recompute)
    r = oracle.run(_oracle_net(reac, prod, rates), init, n, seed=19, t_end=t_end, snap_times=snaps,
                   threads=THREADS, pad_pow2=bool(pad))
    _check(g, r, S, snaps)
    assert g["counters"]["reactions"] > 0


def test_general_batch_graph_replay_and_legacy_stream():
    """A general-network batch runs its K buckets as one captured graph; a replay and a run on the
    legacy default stream (no capture) give the same runs."""
    import torch
    reac, prod, _, _, _ = NETWORKS["moran"]
    N0 = np.array([[40, 60], [3, 2], [500, 524], [9000, 1000]])
    rates = np.array([[1.0, 1.0], [1.0, 0.5], [0.7, 1.3], [1.0, 1.0]])
    runs = np.array([64, 40, 64, 33])
    seeds = np.array([1, 2, 3, 4], dtype=np.uint64)
    outs = []
    for stream in (torch.cuda.current_stream(), None):
        o = pkg.ssa_default_options(cuda_stream=stream, pad_pow2=1)
        ctx = pkg.ssa_create_batch(reac, prod, N0, rates, runs, seeds, o)
        try:
            for _ in range(2):
                pkg.ssa_run(ctx, 0.02, [0.005])
                outs.append(pkg.fetch_all(ctx, n_species=2))
        finally:
            pkg.ssa_destroy(ctx)
    for g in outs[1:]:
        for k in ("final_counts", "outcome", "t_abs", "ee_hist"):
            assert np.array_equal(outs[0][k], g[k]), k
    off = 0
    for e in range(len(N0)):
        r = oracle.run(_oracle_net(reac, prod, rates[e]), N0[e], int(runs[e]), seed=int(seeds[e]), t_end=0.02,
                       snap_times=[0.005], threads=THREADS, pad_pow2=True)
        sl = slice(off, off + runs[e])
        assert_parity({k: outs[0][k][sl] for k in ("final_counts", "outcome", "t_abs")}, r, snaps=False)
        off += runs[e]


@pytest.mark.parametrize("init,n", [((0, 5), 40), ((1, 0), 33), ((3, 3), 0)])
def test_general_degenerate_and_empty(init, n):
    """Runs that start absorbed (one species left, or N_tot = 1) keep their state with t_abs = 0;
    a context with no runs runs and fetches nothing."""
    reac, prod, rates, _, _ = NETWORKS["moran"]
    g = gpu_run(init, n, seed=6, t_end=1.0, snaps=[0.5] if n else [], rates=rates, reac=reac, prod=prod)
    if n == 0:
        assert g["final_counts"].size == 0 and g["counters"]["group_steps"] == 0
        return
    r = oracle.run(_oracle_net(reac, prod, rates), init, n, seed=6, t_end=1.0, snap_times=[0.5], threads=THREADS)
    _check(g, r, 2, [0.5])
    assert np.all(g["t_abs"] == 0.0) and np.all(g["final_counts"] == init)
    assert g["counters"]["group_steps"] == 0
