"""Batched ensembles (one context, many N_tot / rates / seeds) against the oracle and
against one context per ensemble."""
import os

import numpy as np
import pytest

import oracle
import paper_2412_16613_gb300 as pkg
from paper_2412_16613_gb300 import workloads
from tests._gpu import assert_parity

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4
LAYOUTS = pytest.mark.parametrize("layout", [pkg.SSA_LAYOUT_THREAD, pkg.SSA_LAYOUT_WARPS],
                                  ids=["thread", "warps"])


@pytest.fixture(scope="module", autouse=True)
def device():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    oracle.build()
    torch.cuda.set_device(0)
    pkg.use_torch_allocator()


def run_batch(ens, t_end, snaps, **opt):
    import torch
    o = pkg.ssa_default_options(cuda_stream=torch.cuda.current_stream(), keep_snap_counts=1 if len(snaps) else 0,
                                **opt)
    ctx = pkg.ssa_create_batch(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, ens["init"], ens["rates"], ens["runs"],
                               ens["seeds"], o)
    try:
        pkg.ssa_run(ctx, t_end, snaps)
        out = pkg.fetch_all(ctx, snapshots=bool(len(snaps)))
    finally:
        pkg.ssa_destroy(ctx)
    n_total = int(ens["runs"].sum())
    if len(snaps):
        out["snap_counts"] = out["snap_counts"].reshape(len(snaps), n_total, 3)
    out["ee_hist"] = out["ee_hist"].reshape(len(ens["runs"]), len(snaps), 65)
    return out


@LAYOUTS
def test_batch_matches_oracle_per_ensemble(layout):
    ens = workloads.batch_ensembles(n_ens=14, runs=70, n_min=6, n_max=2500, seed=11)
    ens["runs"][3] = 33     # ragged groups
    ens["runs"][5] = 1
    ens["rates"][2] = [1.0, 1.0, 1.0]  # one unit-rate ensemble (no thinning)
    snaps = [0.001, 0.01, 0.1]
    t_end = 50.0
    g = run_batch(ens, t_end, snaps, layout=layout)
    off = np.concatenate([[0], np.cumsum(ens["runs"])])
    for e in range(len(ens["runs"])):
        sl = slice(off[e], off[e + 1])
        r = oracle.run(oracle.frank(*ens["rates"][e]), ens["init"][e], int(ens["runs"][e]),
                       seed=int(ens["seeds"][e]), t_end=t_end, snap_times=snaps, threads=THREADS)
        ge = {"final_counts": g["final_counts"][sl], "outcome": g["outcome"][sl], "t_abs": g["t_abs"][sl],
              "snap_counts": g["snap_counts"][:, sl]}
        ok = assert_parity(ge, r, min_ok=0.9)
        if ok.all():
            assert np.array_equal(g["ee_hist"][e], oracle.ee_histogram(r["snap_counts"])), e
        tally = [np.sum(r["outcome"] == k) for k in range(3)] + [np.sum(r["outcome"] < 0)]
        assert list(g["ens_absorbed"][e]) == tally, e


@pytest.mark.parametrize("precision", [pkg.SSA_P64, pkg.SSA_P32_KAHAN])
@LAYOUTS
def test_batch_equals_separate_contexts(precision, layout):
    import torch
    ens = workloads.batch_ensembles(n_ens=6, runs=100, n_min=20, n_max=5000, seed=3)
    snaps = [0.001, 0.01]
    g = run_batch(ens, 1.0, snaps, precision=precision, layout=layout)
    off = np.concatenate([[0], np.cumsum(ens["runs"])])
    for e in range(6):
        o = pkg.ssa_default_options(cuda_stream=torch.cuda.current_stream(), precision=precision,
                                    layout=pkg.SSA_LAYOUT_THREAD)
        ctx = pkg.ssa_create(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, ens["rates"][e], ens["init"][e],
                             int(ens["runs"][e]), int(ens["seeds"][e]), o)
        try:
            pkg.ssa_run(ctx, 1.0, snaps)
            one = pkg.fetch_all(ctx)
        finally:
            pkg.ssa_destroy(ctx)
        sl = slice(off[e], off[e + 1])
        assert np.array_equal(g["final_counts"][sl], one["final_counts"])
        assert np.array_equal(g["outcome"][sl], one["outcome"])
        assert np.array_equal(g["t_abs"][sl], one["t_abs"])
        assert np.array_equal(g["ee_hist"][e], one["ee_hist"].reshape(len(snaps), 65))


def test_batch_graph_replay_and_recapture():
    """A batch is one captured graph per launch plan: a second run replays it, a run with other
    snapshot times records a new one; every output equals a fresh context's."""
    import torch
    ens = workloads.batch_ensembles(n_ens=9, runs=64, n_min=8, n_max=3000, seed=5)
    o = pkg.ssa_default_options(cuda_stream=torch.cuda.current_stream(), keep_snap_counts=1)
    ctx = pkg.ssa_create_batch(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, ens["init"], ens["rates"], ens["runs"],
                               ens["seeds"], o)
    try:
        outs = []
        for snaps in ([0.01, 0.1], [0.01, 0.1], [0.002, 0.02, 0.2]):
            pkg.ssa_run(ctx, 1.0, snaps)
            outs.append((snaps, pkg.fetch_all(ctx, snapshots=True)))
    finally:
        pkg.ssa_destroy(ctx)
    for k in ("final_counts", "outcome", "t_abs", "ee_hist", "snap_counts"):
        assert np.array_equal(outs[0][1][k], outs[1][1][k]), k
    fresh = run_batch(ens, 1.0, outs[2][0])
    for k in ("final_counts", "outcome", "t_abs"):
        assert np.array_equal(outs[2][1][k], fresh[k]), k
    assert np.array_equal(outs[2][1]["ee_hist"].reshape(fresh["ee_hist"].shape), fresh["ee_hist"])


def test_batch_on_the_legacy_default_stream_and_tuned():
    """A batch on the legacy default stream (which cannot be captured) launches directly; a tuned
    batch context keeps its runs."""
    ens = workloads.batch_ensembles(n_ens=5, runs=96, n_min=10, n_max=4000, seed=8)
    snaps = [0.01, 0.1]
    ref = run_batch(ens, 1.0, snaps)
    o = pkg.ssa_default_options(cuda_stream=None, keep_snap_counts=1)
    ctx = pkg.ssa_create_batch(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, ens["init"], ens["rates"], ens["runs"],
                               ens["seeds"], o)
    try:
        pkg.ssa_run(ctx, 1.0, snaps)
        a = pkg.fetch_all(ctx, snapshots=True)
        choice = pkg.ssa_tune(ctx, 1.0, snaps, probe_steps=300)
        assert choice[0] in (pkg.SSA_LAYOUT_AUTO, pkg.SSA_LAYOUT_THREAD, pkg.SSA_LAYOUT_WARPS)
        pkg.ssa_run(ctx, 1.0, snaps)
        b = pkg.fetch_all(ctx, snapshots=True)
    finally:
        pkg.ssa_destroy(ctx)
    for out in (a, b):
        for k in ("final_counts", "outcome", "t_abs"):
            assert np.array_equal(out[k], ref[k]), k
        assert np.array_equal(out["ee_hist"].reshape(ref["ee_hist"].shape), ref["ee_hist"])


def test_batch_wide_n_against_the_oracle():
    """Ensembles from K = 22 to K = 31 in one batch (N_tot up to 65536, one of them where half of
    all draws are rejected, non-unit rates), each against the oracle."""
    import torch
    Ns = np.array([3000, 20000, 46400, 65536])
    init = np.stack([Ns // 4, Ns // 4, Ns - 2 * (Ns // 4)], 1)
    rates = np.array([[1.0, 1.0, 1.0], [0.7, 1.3, 1.9], [1.0, 1.0, 1.0], [1.2, 0.8, 1.0]])
    runs = np.array([40, 33, 64, 40])
    seeds = np.array([101, 102, 103, 104], dtype=np.uint64)
    lam = np.sort(Ns * (Ns - 1) / 2 * rates.max(1))[1]
    t_end = 1.0e4 / lam  # 10^2 .. 7 10^4 steps per run across the four
    snaps = [t_end / 4, t_end / 2]
    ens = {"init": init, "rates": rates, "runs": runs, "seeds": seeds}
    g = run_batch(ens, t_end, snaps)
    off = np.concatenate([[0], np.cumsum(runs)])
    for e in range(len(Ns)):
        sl = slice(off[e], off[e + 1])
        r = oracle.run(oracle.frank(*rates[e]), init[e], int(runs[e]), seed=int(seeds[e]), t_end=t_end,
                       snap_times=snaps, threads=THREADS)
        ge = {"final_counts": g["final_counts"][sl], "outcome": g["outcome"][sl], "t_abs": g["t_abs"][sl],
              "snap_counts": g["snap_counts"][:, sl]}
        assert_parity(ge, r)
