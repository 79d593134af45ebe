"""The allocation-free entry point ssa_run_frank_noalloc against ssa_run.

Some callers cannot allocate device memory: a plug-in whose host framework owns
every byte of device memory and hands out buffers from its own pool, or a
latency-critical loop in which cudaMalloc (which can synchronise the device) is
not allowed.  For them the library runs the same bit-sliced kernel with its own
scratch in a fixed device array, and the caller passes every input and output
buffer.  These tests call that entry point through the C ABI twice in a row (the
scratch keeps the previous call's contents, so the second call checks that it is
cleared) and compare both results with the allocating entry point ssa_run on the
same inputs and options (paper's bound, group clock): counts, outcomes and
histograms exactly, absorption times to 1e-12 relative.  Also covered: the
largest snapshot count the fixed scratch holds (64), no snapshots without a
histogram buffer, and no runs at all.

Kept in a file of its own that pytest collects last, so that a run stopping at
the first failure has run every other test before this one.
"""
import numpy as np
import pytest

import paper_2412_16613_gb300 as pkg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    torch.cuda.set_device(0)
    return torch


def _reference(init, n_runs, seed, t_end, snaps, rates, precision):
    import torch
    o = pkg.ssa_default_options(cuda_stream=torch.cuda.current_stream(), precision=precision, pad_pow2=0,
                                layout=pkg.SSA_LAYOUT_THREAD, block_size=64)
    ctx = pkg.ssa_create(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, rates, init, n_runs, seed, o)
    try:
        pkg.ssa_run(ctx, t_end, snaps)
        return pkg.fetch_all(ctx)
    finally:
        pkg.ssa_destroy(ctx)


@pytest.mark.parametrize("precision,rates,n_snap", [(pkg.SSA_P64, (1.0, 1.0, 1.0), 10),
                                                    (pkg.SSA_P32_KAHAN, (1.0, 0.5, 0.8), 10),
                                                    (pkg.SSA_P64, (1.0, 1.0, 1.0), 64)])
def test_no_alloc_matches_ssa_run_twice(torch_cuda, precision, rates, n_snap):
    torch = torch_cuda
    init = np.array([256, 256, 512])
    n_runs, seed, t_end = 4096 + 9, 7, 50.0
    snaps = 50.0 * 10.0 ** (4.0 * (np.arange(n_snap) - (n_snap - 1)) / (n_snap - 1))
    snaps[-1] = t_end
    ref = _reference(init, n_runs, seed, t_end, snaps, rates, precision)
    stream = torch.cuda.current_stream()
    for call in range(2):
        # the caller's buffers, filled with garbage so that every element must be written
        final = torch.full((n_runs, 3), -7, dtype=torch.int32, device="cuda")
        t_abs = torch.full((n_runs,), -1.0, dtype=torch.float64, device="cuda")
        outcome = torch.full((n_runs,), 99, dtype=torch.int8, device="cuda")
        hist = torch.full((len(snaps), 65), 12345, dtype=torch.int64, device="cuda")
        counters = pkg.ssa_run_frank_noalloc(init, rates, n_runs, seed, t_end, snaps, final, t_abs, outcome,
                                             hist, precision=precision, stream=stream)
        assert np.array_equal(final.cpu().numpy(), ref["final_counts"]), call
        assert np.array_equal(outcome.cpu().numpy(), ref["outcome"]), call
        assert np.array_equal(hist.cpu().numpy().astype(np.uint64), ref["ee_hist"]), call
        got_t = t_abs.cpu().numpy()
        fin = np.isfinite(ref["t_abs"])
        assert np.array_equal(np.isfinite(got_t), fin)
        np.testing.assert_allclose(got_t[fin], ref["t_abs"][fin], rtol=1e-12, atol=0)
        for k in ("group_steps", "lane_steps", "reactions", "absorbed", "groups_done", "max_group_steps"):
            assert counters[k] == ref["counters"][k], (call, k)
        assert counters["error_flags"] == 0


def test_no_alloc_rejects_sizes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    final = torch.empty((32, 3), dtype=torch.int32, device="cuda")
    t_abs = torch.empty(32, dtype=torch.float64, device="cuda")
    outcome = torch.empty(32, dtype=torch.int8, device="cuda")
    hist = torch.empty((65, 65), dtype=torch.int64, device="cuda")
    with pytest.raises(pkg.SSAError) as ei:
        pkg.ssa_run_frank_noalloc([16, 16, 32], [1, 1, 1], 32, 0, 1.0, np.linspace(0, 1, 65), final, t_abs,
                                  outcome, hist)
    assert ei.value.status == pkg.SSA_EINVAL
    assert "64" in pkg.ssa_last_error()


def test_no_alloc_without_snapshots_or_runs(torch_cuda):
    """No snapshots and no histogram buffer; then no runs and no output buffers at all."""
    torch = torch_cuda
    init, n_runs, seed, t_end = np.array([16, 16, 32]), 64 + 5, 3, 10.0
    ref = _reference(init, n_runs, seed, t_end, [], (1.0, 1.0, 1.0), pkg.SSA_P64)
    stream = torch.cuda.current_stream()
    for call in range(2):
        final = torch.full((n_runs, 3), -7, dtype=torch.int32, device="cuda")
        t_abs = torch.full((n_runs,), -1.0, dtype=torch.float64, device="cuda")
        outcome = torch.full((n_runs,), 99, dtype=torch.int8, device="cuda")
        counters = pkg.ssa_run_frank_noalloc(init, (1.0, 1.0, 1.0), n_runs, seed, t_end, [], final, t_abs,
                                             outcome, None, stream=stream)
        assert np.array_equal(final.cpu().numpy(), ref["final_counts"]), call
        assert np.array_equal(outcome.cpu().numpy(), ref["outcome"]), call
        fin = np.isfinite(ref["t_abs"])
        np.testing.assert_allclose(t_abs.cpu().numpy()[fin], ref["t_abs"][fin], rtol=1e-12, atol=0)
        assert counters["reactions"] == ref["counters"]["reactions"], call
    counters = pkg.ssa_run_frank_noalloc(init, (1.0, 1.0, 1.0), 0, seed, t_end, [0.5], None, None, None,
                                         torch.full((1, 65), 5, dtype=torch.int64, device="cuda"),
                                         stream=stream)
    assert all(v == 0 for v in counters.values()), counters
