"""The seeded workload definitions (CPU)."""
import numpy as np

from paper_2412_16613_gb300 import workloads


def test_batch_workload_definition():
    """4096 ensembles: N_tot log-uniform over [16, 65536], rates in [0.5, 2], racemic starts."""
    ens = workloads.batch_ensembles()
    assert len(ens["n_tot"]) == 4096 and ens["n_tot"].min() >= 16 and ens["n_tot"].max() <= 65536
    assert np.all(ens["init"].sum(1) == ens["n_tot"])
    assert np.all(ens["init"][:, 0] == ens["n_tot"] // 4) and np.all(ens["init"][:, 0] == ens["init"][:, 1])
    assert np.all((ens["rates"] >= 0.5) & (ens["rates"] <= 2.0))
    assert np.all(ens["runs"] == 1024) and np.array_equal(ens["seeds"], np.arange(4096))
    logn = np.log(ens["n_tot"])
    assert abs(np.median(logn) - 0.5 * (np.log(16) + np.log(65536))) < 0.3   # log-uniform
    again = workloads.batch_ensembles()
    assert np.array_equal(again["n_tot"], ens["n_tot"]) and np.array_equal(again["rates"], ens["rates"])


def test_log_snapshots():
    s = workloads.log_snapshots(50.0, 10)
    assert np.isclose(s[0], 50e-4) and np.isclose(s[-1], 50.0) and np.all(np.diff(np.log10(s)) > 0)
