"""fp32 clocks against the fp64 clock at N_tot = 10000 (2500, 2500, 5000).

The integer dynamics are exact in every mode; only event times differ.  The fp32
uniform is the top 24 bits of the fp64 one, so runs with the same seed are paired
and their time differences are the rounding error itself.  Checks (the precision
targets): two-sample KS p > 0.01 on absorption times and means within 3 standard
errors, both for paired runs and for independent seeds (one run per group); the ee histograms at the
snapshots agree (chi-square p > 0.01).  The plain fp32 sum (no compensation) is
the control: its paired time error must exceed the compensated one's.
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
RUNS = 1 << 15
SNAPS = list(workloads.log_snapshots(0.05, 6))


@pytest.fixture(scope="module")
def runs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    torch.cuda.set_device(0)
    pkg.use_torch_allocator()
    out = {}
    for name, mode, seed in [("p64", pkg.SSA_P64, 1), ("p64_other_seed", pkg.SSA_P64, 2),
                             ("kahan", pkg.SSA_P32_KAHAN, 1), ("kahan_other_seed", pkg.SSA_P32_KAHAN, 3),
                             ("d64acc", pkg.SSA_P32_D64ACC, 1), ("plain", pkg.SSA_P32_PLAIN, 1)]:
        out[name] = gpu_run(INIT, RUNS, seed=seed, t_end=1.0, snaps=SNAPS, precision=mode, keep_snaps=False)
    return out


def _hist_pvalue(h1, h2):
    table = np.vstack([h1, h2]).astype(float)
    keep = table.sum(0) > 0
    if keep.sum() < 2:
        return 1.0
    return stats.chi2_contingency(table[:, keep])[1]


@pytest.mark.parametrize("mode", ["kahan", "d64acc"])
def test_fp32_clock_paired_with_fp64(runs, mode):
    ref, got = runs["p64"], runs[mode]
    assert np.array_equal(ref["final_counts"], got["final_counts"])  # the integer dynamics are shared
    fin = np.isfinite(ref["t_abs"])
    assert np.array_equal(fin, np.isfinite(got["t_abs"]))
    rel = np.abs(got["t_abs"][fin] / ref["t_abs"][fin] - 1)
    assert np.median(rel) < 1e-5 and rel.max() < 1e-2
    se = ref["t_abs"][fin].std() / math.sqrt(fin.sum())
    assert abs(got["t_abs"][fin].mean() - ref["t_abs"][fin].mean()) < 3 * se
    assert stats.ks_2samp(got["t_abs"][fin], ref["t_abs"][fin]).pvalue > 0.01
    for s in range(len(SNAPS)):
        assert _hist_pvalue(ref["ee_hist"][s], got["ee_hist"][s]) > 0.01


def test_fp32_kahan_against_independent_fp64(runs):
    """Independent seeds, one run per group: the 32 runs of a group share the group's clock, so
    their absorption times are not independent samples and a KS test over all runs would be too
    strict (over 2^22 runs it separates two fp64 seeds at p = 0.005; one run per group, p = 0.40)."""
    a, b = runs["kahan_other_seed"], runs["p64_other_seed"]
    ta, tb = a["t_abs"][::32], b["t_abs"][::32]
    ta, tb = ta[np.isfinite(ta)], tb[np.isfinite(tb)]
    se = math.sqrt(ta.var() / len(ta) + tb.var() / len(tb))
    assert abs(ta.mean() - tb.mean()) < 3 * se
    assert stats.ks_2samp(ta, tb).pvalue > 0.01
    for s in range(len(SNAPS)):
        assert _hist_pvalue(a["ee_hist"][s], b["ee_hist"][s]) > 0.01


def test_plain_fp32_sum_is_the_worse_control(runs):
    ref = runs["p64"]
    fin = np.isfinite(ref["t_abs"])
    err_plain = np.abs(runs["plain"]["t_abs"][fin] / ref["t_abs"][fin] - 1)
    err_kahan = np.abs(runs["kahan"]["t_abs"][fin] / ref["t_abs"][fin] - 1)
    assert np.mean(err_plain) > np.mean(err_kahan)
