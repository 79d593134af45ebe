"""Helpers for the GPU tests: run libbitssa through its C ABI and compare with the oracle."""
import numpy as np

import oracle
import paper_2412_16613_gb300 as pkg

FRANK_R, FRANK_P = pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS


def log_snapshots(t_end=50.0, n=10):
    """Log-spaced snapshot times t_s = t_end 10^(4 (s - (n-1)) / (n-1)), s = 0..n-1."""
    s = np.arange(n)
    return t_end * 10.0 ** (4.0 * (s - (n - 1)) / (n - 1))


def gpu_run(init, n_runs, seed=0, t_end=np.inf, snaps=(), rates=(1.0, 1.0, 1.0), reac=FRANK_R,
            prod=FRANK_P, keep_snaps=True, expect_status=0, **opt):
    import torch
    stream = torch.cuda.current_stream()
    keep = 1 if (keep_snaps and len(snaps)) else 0
    o = pkg.ssa_default_options(keep_snap_counts=keep, cuda_stream=stream, **opt)
    ctx = pkg.ssa_create(reac, prod, rates, init, n_runs, seed, o)
    try:
        try:
            pkg.ssa_run(ctx, t_end, snaps)
        except pkg.SSAError as e:
            if e.status != expect_status:
                raise
        else:
            assert expect_status == 0
        S = np.asarray(reac).shape[1]
        out = pkg.fetch_all(ctx, n_species=S, snapshots=bool(keep))
        if keep:
            out["snap_counts"] = out["snap_counts"].reshape(len(snaps), n_runs, S)
    finally:
        pkg.ssa_destroy(ctx)
    return out


def assert_parity(g, r, rtol=1e-12, tie=1e-12, snaps=True, min_ok=0.99):
    """Bit-exact counts and outcomes, times within rtol, on runs without a near tie
    (a snapshot or t_end within `tie` relative of an event time)."""
    ok = r["margin"] > tie
    assert ok.mean() >= min_ok, ok.mean()
    assert np.array_equal(g["final_counts"][ok], r["final_counts"][ok])
    assert np.array_equal(g["outcome"][ok], r["outcome"][ok])
    fin = np.isfinite(r["t_abs"])
    assert np.array_equal(np.isfinite(g["t_abs"])[ok], fin[ok])
    m = ok & fin
    np.testing.assert_allclose(g["t_abs"][m], r["t_abs"][m], rtol=rtol, atol=0)
    if snaps and r["snap_counts"] is not None and "snap_counts" in g:
        assert np.array_equal(g["snap_counts"][:, ok], r["snap_counts"][:, ok])
    return ok


def assert_hist_parity(g, r, ok):
    """ee_hist: the GPU's histogram is the histogram of its own per-run snapshot counts (all
    runs), and on the runs without a near tie those counts bin exactly as the oracle's."""
    assert np.array_equal(g["ee_hist"].reshape(-1, 65), oracle.ee_histogram(g["snap_counts"]))
    assert np.array_equal(oracle.ee_histogram(g["snap_counts"][:, ok]), oracle.ee_histogram(r["snap_counts"][:, ok]))


def group_steps(r, n_runs):
    """Per group of 32 runs: the steps of its longest run (a group steps until its last run stops)."""
    steps = np.zeros(((n_runs + 31) // 32) * 32, dtype=np.int64)
    steps[:n_runs] = r["steps"]
    return steps.reshape(-1, 32).max(1)
