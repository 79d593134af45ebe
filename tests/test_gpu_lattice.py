"""GPU parity of Frank's model on a periodic lattice (ssa_lattice_* through the C ABI) against the
lattice oracle on the same seeded inputs: every site count of every run, the lattice totals and
domain counts at every snapshot, the reactions and hops of every run, every group's steps and cap
bit-exact; fp64 times within 1e-12 relative, fp32 times within 2e-5.  Groups whose oracle clock
comes within the tie tolerance of a snapshot or t_end are left out as a whole (they share one
clock)."""
import math

import numpy as np
import pytest

import oracle
import paper_2412_16613_gb300 as pkg
from paper_2412_16613_gb300 import workloads

pytestmark = pytest.mark.gpu

ORC_PRECISION = {pkg.SSA_P64: oracle.P64, pkg.SSA_P64_LOGSUM: oracle.P64, pkg.SSA_P32_KAHAN: oracle.P32_KAHAN,
                 pkg.SSA_P32_D64ACC: oracle.P32_D64ACC, pkg.SSA_P32_PLAIN: oracle.P32_PLAIN}


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


def gpu_lattice(lx, ly, init, n_runs, *, rates=(1.0, 1.0, 1.0), hop=0.1, seed=0, t_end=0.1, snaps=(),
                cap_bits_max=0, expect_status=0, **opt):
    import torch
    o = pkg.ssa_default_options(cuda_stream=torch.cuda.current_stream(), **opt)
    ctx = pkg.ssa_lattice_create(lx, ly, rates, hop, init, n_runs, seed, o, cap_bits_max=cap_bits_max)
    try:
        try:
            pkg.ssa_lattice_run(ctx, t_end, snaps)
        except pkg.SSAError as e:
            if e.status != expect_status:
                raise
        else:
            assert expect_status == 0
        return pkg.lattice_fetch_all(ctx, lx * ly, len(snaps))
    finally:
        pkg.ssa_lattice_destroy(ctx)


def orc_lattice(lx, ly, init, n_runs, *, rates=(1.0, 1.0, 1.0), hop=0.1, seed=0, t_end=0.1, snaps=(),
                precision=pkg.SSA_P64, step_budget=0, groups=None, check=True, thin_bits=32):
    return oracle.lattice_run(lx, ly, init, n_runs, rates=rates, hop=hop, seed=seed, t_end=t_end,
                              snap_times=snaps, precision=ORC_PRECISION[precision], step_budget=step_budget,
                              groups=groups, check=check, thin_bits=thin_bits)


def assert_lattice_parity(g, r, n_snap, runs=None, tie=1e-12, rtol=1e-12, min_ok=0.9):
    """runs: the run indices the oracle computed (default all).  Returns the runs compared."""
    n = len(r["outcome"])
    runs = np.arange(n) if runs is None else np.asarray(runs)
    ok = r["margin"] > tie
    assert ok.mean() >= min_ok, ok.mean()
    gr = runs[ok]
    assert np.array_equal(g["final_counts"][gr], r["final_counts"][ok])
    assert np.array_equal(g["outcome"][gr], r["outcome"][ok])
    fin = np.isfinite(r["t_homochiral"][ok])
    assert np.array_equal(np.isfinite(g["t_homochiral"][gr]), fin)
    np.testing.assert_allclose(g["t_homochiral"][gr][fin], r["t_homochiral"][ok][fin], rtol=rtol, atol=0)
    assert np.array_equal(g["events"][gr, 0], r["reactions"][ok])
    assert np.array_equal(g["events"][gr, 1], r["hops"][ok])
    assert np.array_equal(g["groups"][gr // 32, 0], r["steps"][ok])
    assert np.array_equal(g["groups"][gr // 32, 1], r["cap"][ok])
    if n_snap:
        assert np.array_equal(g["snap_totals"][:, gr].transpose(1, 0, 2), r["snap_totals"][ok])
        assert np.array_equal(g["snap_domains"][:, gr].transpose(1, 0, 2), r["snap_domains"][ok])
    return gr


SNAPS_8 = [0.01, 0.03, 0.05, 0.05, 0.08]


@pytest.mark.parametrize("block", [32, 128, 224])
def test_lattice_8x8_per_run_init(block):
    """8 x 8 lattice, 80 runs (a ragged last group) from per-run Poisson counts (means 2, 2, 4), unit
    rates, d = 0.1 (rho_r = 10), t_end = 0.1 with five snapshots (one repeated): bit-exact, whatever
    the number of pending steps (block size)."""
    init = workloads.lattice_init(8, 8, 80, mean=(2.0, 2.0, 4.0), seed=11)
    g = gpu_lattice(8, 8, init, 80, seed=3, t_end=0.1, snaps=SNAPS_8, block_size=block)
    r = orc_lattice(8, 8, init, 80, seed=3, t_end=0.1, snaps=SNAPS_8)
    assert_lattice_parity(g, r, len(SNAPS_8))
    assert g["counters"]["reactions"] > 0 and g["counters"]["hops"] > 0
    assert g["counters"]["group_errors"] == 0
    assert g["counters"]["group_steps"] == int(g["groups"][:, 0].sum())


def test_lattice_shared_init_and_block_invariance():
    """Counts shared by every run (16 x 4 lattice, 64 runs): all block sizes give the same runs, every
    field, and the oracle agrees."""
    rng = np.random.default_rng(5)
    init = rng.poisson((3, 3, 6), size=(64, 3)).astype(np.int64)
    outs = [gpu_lattice(16, 4, init, 64, seed=9, t_end=0.05, snaps=[0.02], block_size=b, hop=0.25)
            for b in (32, 64, 96, 224)]
    for o in outs[1:]:
        for k in ("final_counts", "t_homochiral", "outcome", "events", "groups", "snap_totals", "snap_domains"):
            assert np.array_equal(o[k], outs[0][k]), k
    r = orc_lattice(16, 4, init, 64, seed=9, t_end=0.05, snaps=[0.02], hop=0.25)
    assert_lattice_parity(outs[0], r, 1)


@pytest.mark.parametrize("lx,ly", [(1, 1), (2, 1), (1, 4), (2, 2), (4, 2), (2, 8)])
def test_lattice_small_sides(lx, ly):
    """Sides of length 1 (a hop comes back to its own site) and 2 (two directions lead to the same
    neighbour), with fast hops (d = 2, rho_h = 2): every window is a chain of dependent steps."""
    M = lx * ly
    init = workloads.lattice_init(lx, ly, 40, mean=(1.5, 1.5, 3.0), seed=12 + M)
    g = gpu_lattice(lx, ly, init, 40, rates=(1.0, 1.0, 1.0), hop=2.0, seed=4, t_end=0.3, snaps=[0.1, 0.2])
    r = orc_lattice(lx, ly, init, 40, rates=(1.0, 1.0, 1.0), hop=2.0, seed=4, t_end=0.3, snaps=[0.1, 0.2])
    assert_lattice_parity(g, r, 2)
    assert np.array_equal(g["final_counts"].sum(axis=(1, 2)), init.sum(axis=(1, 2)))
    if M <= 2:
        assert np.isfinite(r["t_homochiral"]).any()  # runs whose whole lattice came to one species


def test_lattice_thinning():
    """Rates (1, 0.5, 2) with d = 0.5: rho_r = 4, reactions 1 and 2 thinned with q = 32 bits."""
    init = workloads.lattice_init(4, 4, 64, mean=(3.0, 3.0, 6.0), seed=13)
    kw = dict(rates=(1.0, 0.5, 2.0), hop=0.5, seed=6, t_end=0.05, snaps=[0.02])
    g = gpu_lattice(4, 4, init, 64, **kw)
    r = orc_lattice(4, 4, init, 64, **kw)
    assert_lattice_parity(g, r, 1)
    g2 = gpu_lattice(4, 4, init, 64, thin_bits=7, **kw)
    r2 = orc_lattice(4, 4, init, 64, thin_bits=7, **kw)
    assert_lattice_parity(g2, r2, 1)


def test_lattice_cap_doubles():
    """Sites start at exactly the cap m = 8 and hops are fast (d = 4): a hop soon pushes a site above
    m, the cap moves to 10, 12, ... (K and the rate change from the next step), and the runs still
    agree."""
    M, runs = 16, 64
    init = np.zeros((runs, M, 3), dtype=np.int64)
    init[:, :, 0] = 2
    init[:, :, 1] = 2
    init[:, :, 2] = 4   # 8 molecules on every site: m = 8
    kw = dict(rates=(1.0, 1.0, 1.0), hop=4.0, seed=7, t_end=0.2, snaps=[0.1])
    g = gpu_lattice(4, 4, init, runs, cap_bits_max=6, **kw)
    r = orc_lattice(4, 4, init, runs, **kw)
    assert_lattice_parity(g, r, 1)
    assert np.all(g["groups"][:, 1] > 8)
    assert g["counters"]["cap_raises"] >= 2 and g["counters"]["flagged"] > 0


def test_lattice_capacity_error_then_larger_planes():
    """Site 0 starts with 8 molecules (cap 8), the others with one: the kernel takes 4 count planes
    (caps up to 8), fast hops (d = 8) soon bring a ninth molecule to a full site and the run stops
    with SSA_EOVERFLOW; cap_bits_max = 6 takes 8 planes (caps up to 64) and the run agrees with the
    oracle, whose counts have no width."""
    init = np.zeros((32, 16, 3), dtype=np.int64)
    init[:, :, 0] = 1
    init[:, 0] = (4, 4, 0)
    kw = dict(rates=(1.0, 1.0, 1.0), hop=8.0, seed=8, t_end=1.0)
    g = gpu_lattice(4, 4, init, 32, expect_status=pkg.SSA_EOVERFLOW, **kw)
    assert g["groups"][0, 2] == 3 and g["groups"][0, 1] == 10  # stopped, needing the cap 10
    r = orc_lattice(4, 4, init, 32, **kw)
    assert r["cap"].max() <= 64
    g = gpu_lattice(4, 4, init, 32, cap_bits_max=6, **kw)
    assert_lattice_parity(g, r, 0)


@pytest.mark.parametrize("precision", [pkg.SSA_P32_KAHAN, pkg.SSA_P32_D64ACC, pkg.SSA_P32_PLAIN])
def test_lattice_fp32_clocks(precision):
    """The fp32 clocks: the same integer steps, times within 2e-5 (an ulp of logf per step), groups
    with an event within 1e-5 of a snapshot or t_end left out."""
    init = workloads.lattice_init(8, 8, 64, mean=(2.0, 2.0, 4.0), seed=14)
    kw = dict(seed=10, t_end=0.05, snaps=[0.01, 0.03])
    g = gpu_lattice(8, 8, init, 64, precision=precision, **kw)
    r = orc_lattice(8, 8, init, 64, precision=precision, **kw)
    assert_lattice_parity(g, r, 2, tie=1e-5, rtol=2e-5, min_ok=0.5)


def test_lattice_step_budget():
    """A step budget stops every group at exactly that many steps with SSA_ETIMEOUT, as the oracle."""
    init = workloads.lattice_init(4, 4, 64, mean=(2.0, 2.0, 4.0), seed=15)
    g = gpu_lattice(4, 4, init, 64, seed=2, t_end=10.0, step_budget=777, expect_status=pkg.SSA_ETIMEOUT)
    r = orc_lattice(4, 4, init, 64, seed=2, t_end=10.0, step_budget=777, check=False)
    assert r["status"] == oracle.ETIMEOUT
    assert np.all(g["groups"][:, 0] == 777) and np.all(g["groups"][:, 2] == 1)
    assert np.array_equal(g["final_counts"], r["final_counts"])
    assert np.array_equal(g["events"][:, 0], r["reactions"]) and np.array_equal(g["events"][:, 1], r["hops"])


def test_lattice_k_beyond_32_planes():
    """rho_r = 40000 with 600 molecules on a site (cap 640) needs K = 33 > 32 planes of n: the oracle
    and the kernel both stop before the first step."""
    init = np.zeros((32, 2, 3), dtype=np.int64)
    init[:, 0] = (200, 200, 200)
    kw = dict(rates=(1.0, 1.0, 1.0), hop=1.0 / 40000, seed=1, t_end=1.0)
    g = gpu_lattice(2, 1, init, 32, expect_status=pkg.SSA_EOVERFLOW, **kw)
    r = orc_lattice(2, 1, init, 32, check=False, **kw)
    assert r["status"] == oracle.ERANGE
    assert np.all(g["groups"][:, 0] == 0) and np.all(g["groups"][:, 2] == 2)
    assert np.array_equal(g["final_counts"], r["final_counts"])


def test_lattice_empty_and_homochiral_start():
    """No runs; and runs whose lattice holds one species from the start (time 0, that species)."""
    init = np.zeros((16, 3), dtype=np.int64)
    g = gpu_lattice(4, 4, init, 0, t_end=0.1)
    assert g["final_counts"].size == 0 and g["counters"]["group_steps"] == 0
    init[:, 0] = 3
    g = gpu_lattice(4, 4, init, 35, t_end=0.05, snaps=[0.01])
    r = orc_lattice(4, 4, init, 35, t_end=0.05, snaps=[0.01])
    assert_lattice_parity(g, r, 1)
    assert np.all(g["t_homochiral"] == 0.0) and np.all(g["outcome"] == 0)
    assert np.all(g["events"][:, 0] == 0)


def test_lattice_first_run_shards():
    """Two contexts, first_run 0 and 64, reproduce one context of 128 runs."""
    init = workloads.lattice_init(8, 4, 128, mean=(2.0, 2.0, 4.0), seed=16)
    whole = gpu_lattice(8, 4, init, 128, seed=5, t_end=0.05, snaps=[0.02])
    a = gpu_lattice(8, 4, init[:64], 64, seed=5, t_end=0.05, snaps=[0.02])
    b = gpu_lattice(8, 4, init[64:], 64, seed=5, t_end=0.05, snaps=[0.02], first_run=64)
    for k in ("final_counts", "t_homochiral", "outcome", "events"):
        assert np.array_equal(np.concatenate([a[k], b[k]]), whole[k]), k
    assert np.array_equal(np.concatenate([a["snap_totals"], b["snap_totals"]], axis=1), whole["snap_totals"])


def test_lattice_64x64_full_size_sampled():
    """The 64 x 64 workload: 4096 runs from per-site Poisson(8, 8, 16) counts, unit rates, d = 0.1,
    to t_end = 0.01 with two snapshots (1.3e5 to 5.4e5 steps a group), fp64 clock: events come
    every 2e-6 of t relative, far above the fp64 tie tolerance but not above an fp32 clock's, whose
    parity the 8 x 8 tests check.  Three sampled groups (first, middle, last) bit-exact against
    the oracle; over every run the total count is conserved, the snapshot totals conserve it too,
    and the cap holds every site."""
    lx = ly = 64
    runs = 4096
    init = workloads.lattice_init(lx, ly, runs)
    snaps = [0.002, 0.005]
    kw = dict(seed=0, t_end=0.01, snaps=snaps, precision=pkg.SSA_P64)
    g = gpu_lattice(lx, ly, init, runs, **kw)
    groups = [0, 63, 127]
    r = orc_lattice(lx, ly, init, runs, groups=groups, **kw)
    sel = np.concatenate([np.arange(32 * k, 32 * k + 32) for k in groups])
    assert_lattice_parity(g, r, len(snaps), runs=sel, min_ok=0.6)
    tot = init.sum(axis=(1, 2))
    assert np.array_equal(g["final_counts"].sum(axis=(1, 2)), tot)
    assert np.all(g["snap_totals"].sum(axis=2) == tot[None, :])
    cap = g["groups"][:, 1]
    assert np.all(g["final_counts"].sum(axis=2).max(axis=1) <= np.repeat(cap, 32))
    assert g["counters"]["group_errors"] == 0


def test_lattice_largest_lattice():
    """128 x 128 sites, the most the kernel's per-site shared-memory tables hold (16 384 sites, 218 KB
    of shared memory a block), 40 runs (a ragged second group), to t_end = 0.001: bit-exact."""
    init = workloads.lattice_init(128, 128, 40, mean=(1.0, 1.0, 2.0), seed=17)
    kw = dict(seed=12, t_end=0.001, snaps=[0.0005])
    g = gpu_lattice(128, 128, init, 40, **kw)
    r = orc_lattice(128, 128, init, 40, **kw)
    assert_lattice_parity(g, r, 1, min_ok=0.5)
    assert g["counters"]["group_steps"] > 1000
