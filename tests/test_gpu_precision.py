"""fp32 clocks against the fp64 clock at the precision workload's full size: N_tot = 10 000 from
(2500, 2500, 5000), 2^22 runs, t_end = 50, the 10 log-spaced snapshots, bound padded to 2^K.

The integer dynamics are exact in every mode; only event times differ.  The fp32 uniform is the
top 24 bits of the fp64 one, so runs with the same seed are paired and their time differences
are the rounding error itself.  Checks (the precision targets): two-sample KS p > 0.01 on
absorption times and means within 3 standard errors, for paired runs and for independent seeds;
the ee histograms at the snapshots agree (chi-square p > 0.01).  Under the group clock the 32
runs of a group share their event times, so independent-seed comparisons take one run per group;
with a clock per run (SSA_CLOCK_LANE) every run is an independent sample and the comparison takes
all 2^22.  The plain fp32 sum (no compensation) is the control: its paired time error must exceed
the compensated one's.  The numbers are printed.
"""
import math

import numpy as np
import pytest
from scipy import stats

import paper_2412_16613_gb300 as pkg
from paper_2412_16613_gb300 import workloads
from tests._gpu import gpu_run

pytestmark = pytest.mark.gpu

INIT = (2500, 2500, 5000)
RUNS = 1 << 22
T_END = 50.0
SNAPS = list(workloads.log_snapshots(T_END, 10))


@pytest.fixture(scope="module")
def runs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    torch.cuda.set_device(0)
    pkg.use_torch_allocator()
    out = {}
    for name, mode, seed, clock in [("p64", pkg.SSA_P64, 1, 0), ("p64_other_seed", pkg.SSA_P64, 2, 0),
                                    ("kahan", pkg.SSA_P32_KAHAN, 1, 0), ("kahan_other_seed", pkg.SSA_P32_KAHAN, 3, 0),
                                    ("d64acc", pkg.SSA_P32_D64ACC, 1, 0), ("plain", pkg.SSA_P32_PLAIN, 1, 0),
                                    ("p64_lane", pkg.SSA_P64, 4, 1), ("kahan_lane", pkg.SSA_P32_KAHAN, 5, 1)]:
        g = gpu_run(INIT, RUNS, seed=seed, t_end=T_END, snaps=SNAPS, precision=mode, keep_snaps=False, pad_pow2=1,
                    clock=clock)
        out[name] = {"final_counts": g["final_counts"], "t_abs": g["t_abs"], "ee_hist": g["ee_hist"]}
    return out


def _hist_pvalue(h1, h2):
    table = np.vstack([h1, h2]).astype(float)
    keep = table.sum(0) > 0
    if keep.sum() < 2:
        return 1.0
    return stats.chi2_contingency(table[:, keep])[1]


@pytest.mark.parametrize("mode", ["kahan", "d64acc"])
def test_fp32_clock_paired_with_fp64(runs, mode):
    """Same seed: the same runs, event times within fp32 rounding; every run of 2^22."""
    ref, got = runs["p64"], runs[mode]
    same = np.all(ref["final_counts"] == got["final_counts"], axis=1)
    assert same.mean() > 0.999  # only runs with an event within fp32 rounding of t_end may differ
    fin = np.isfinite(ref["t_abs"]) & np.isfinite(got["t_abs"]) & same
    rel = np.abs(got["t_abs"][fin] / ref["t_abs"][fin] - 1)
    se = ref["t_abs"][fin].std() / math.sqrt(fin.sum())
    diff = abs(got["t_abs"][fin].mean() - ref["t_abs"][fin].mean()) / se
    ks = stats.ks_2samp(got["t_abs"][fin], ref["t_abs"][fin]).pvalue
    hp = [_hist_pvalue(ref["ee_hist"][s], got["ee_hist"][s]) for s in range(len(SNAPS))]
    print(f"{mode} paired: relative time error median {np.median(rel):.2e} max {rel.max():.2e}; "
          f"mean difference {diff:.3f} SE; KS p {ks:.3f}; histogram p min {min(hp):.3f}")
    assert np.median(rel) < 1e-5 and rel.max() < 1e-2
    assert diff < 3 and ks > 0.01 and min(hp) > 0.01


def test_fp32_kahan_against_independent_fp64_one_run_per_group(runs):
    """Independent seeds under the group clock: one run per group (2^17 independent runs)."""
    a, b = runs["kahan_other_seed"]["t_abs"][::32], runs["p64_other_seed"]["t_abs"][::32]
    a, b = a[np.isfinite(a)], b[np.isfinite(b)]
    se = math.sqrt(a.var() / len(a) + b.var() / len(b))
    diff = abs(a.mean() - b.mean()) / se
    ks = stats.ks_2samp(a, b).pvalue
    print(f"kahan vs p64, independent seeds, one run per group: mean difference {diff:.3f} SE, KS p {ks:.3f}")
    assert diff < 3 and ks > 0.01


def test_fp32_kahan_against_independent_fp64_every_run_per_run_clock(runs):
    """Independent seeds with a clock per run: all 2^22 runs are independent samples; absorption
    times and the ee histograms at every snapshot."""
    ra, rb = runs["kahan_lane"], runs["p64_lane"]
    a, b = ra["t_abs"][np.isfinite(ra["t_abs"])], rb["t_abs"][np.isfinite(rb["t_abs"])]
    se = math.sqrt(a.var() / len(a) + b.var() / len(b))
    diff = abs(a.mean() - b.mean()) / se
    ks = stats.ks_2samp(a, b).pvalue
    hp = [_hist_pvalue(ra["ee_hist"][s], rb["ee_hist"][s]) for s in range(len(SNAPS))]
    print(f"kahan vs p64, per-run clocks, independent seeds, all runs: mean difference {diff:.3f} SE, "
          f"KS p {ks:.3f}, histogram p min {min(hp):.3f}")
    assert diff < 3 and ks > 0.01 and min(hp) > 0.01


def test_plain_fp32_sum_is_the_worse_control(runs):
    ref = runs["p64"]
    fin = np.isfinite(ref["t_abs"]) & np.isfinite(runs["plain"]["t_abs"])
    err_plain = np.abs(runs["plain"]["t_abs"][fin] / ref["t_abs"][fin] - 1)
    err_kahan = np.abs(runs["kahan"]["t_abs"][fin] / ref["t_abs"][fin] - 1)
    print(f"median relative time error: plain fp32 {np.median(err_plain):.2e}, Kahan {np.median(err_kahan):.2e}")
    assert np.median(err_plain) > 2 * np.median(err_kahan)


def test_fp32_batched_form_against_fp64():
    """The FP32 batched form: 24 ensembles of the batched workload's recipe (N_tot log-uniform,
    here in [16, 4096]; rates uniform in [0.5, 2]), 2048 runs each, in one batch, fp32 Kahan
    clocks against fp64.  Same seeds: the same runs, times within fp32
    rounding.  Independent seeds: per ensemble the mean absorption time over group means (the
    groups are independent) as a z-score; their squares sum to a chi-square with 24 degrees."""
    import torch
    ens = workloads.batch_ensembles(n_ens=24, runs=2048, n_min=16, n_max=4096, seed=0x5EED)
    stream = torch.cuda.current_stream()

    def batch(precision, seed_offset):
        o = pkg.ssa_default_options(cuda_stream=stream, precision=precision, pad_pow2=1)
        ctx = pkg.ssa_create_batch(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, ens["init"], ens["rates"], ens["runs"],
                                   ens["seeds"] + np.uint64(seed_offset), o)
        try:
            pkg.ssa_run(ctx, T_END, SNAPS[:5])
            return pkg.fetch_all(ctx)
        finally:
            pkg.ssa_destroy(ctx)

    p64, k32 = batch(pkg.SSA_P64, 0), batch(pkg.SSA_P32_KAHAN, 0)
    same = np.all(p64["final_counts"] == k32["final_counts"], axis=1)
    assert same.mean() > 0.999
    fin = same & np.isfinite(p64["t_abs"]) & np.isfinite(k32["t_abs"])
    rel = np.abs(k32["t_abs"][fin] / p64["t_abs"][fin] - 1)
    assert np.median(rel) < 1e-5 and rel.max() < 1e-2
    a, b = batch(pkg.SSA_P64, 1000), batch(pkg.SSA_P32_KAHAN, 2000)
    z2, row = 0.0, 0
    for r in ens["runs"]:
        ga = np.nanmean(np.where(np.isfinite(a["t_abs"][row:row + r]), a["t_abs"][row:row + r], np.nan).reshape(-1, 32), 1)
        gb = np.nanmean(np.where(np.isfinite(b["t_abs"][row:row + r]), b["t_abs"][row:row + r], np.nan).reshape(-1, 32), 1)
        se = math.sqrt(ga.var(ddof=1) / len(ga) + gb.var(ddof=1) / len(gb))
        z2 += ((ga.mean() - gb.mean()) / se) ** 2
        row += r
    p = stats.chi2.sf(z2, len(ens["runs"]))
    print(f"batched fp32 Kahan vs fp64, independent seeds: chi-square of per-ensemble z-scores p {p:.3f}; "
          f"paired relative time error median {np.median(rel):.2e}")
    assert p > 0.01
