"""Allocation failure through the caller's allocator hook (ssa_set_allocator).

The hook hands out device memory from PyTorch's caching allocator until a budget of
successful calls is spent, then returns NULL.  For every budget below what a create
and a run need, the failing call must return SSA_ENOMEM, and every buffer the hook
handed out must come back through its release callback (at once for a failed create,
at ssa_destroy for a failed run): nothing leaks."""
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
    yield torch
    pkg.use_torch_allocator()


class BudgetAllocator:
    def __init__(self, torch, budget):
        self.torch, self.budget, self.live, self.calls = torch, budget, {}, 0

    def alloc(self, nbytes, device, stream, user):
        self.calls += 1
        if self.budget is not None and self.budget <= 0:
            return None
        if self.budget is not None:
            self.budget -= 1
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes), device=int(device), stream=stream or 0)
        self.live[p] = int(nbytes)
        return p

    def release(self, ptr, nbytes, device, stream, user):
        assert self.live.pop(ptr) == int(nbytes)
        self.torch.cuda.caching_allocator_delete(ptr)


def _create_and_run(kind, opt):
    if kind == "single":
        ctx = pkg.ssa_create(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, [1.0, 1.0, 1.0], np.array([16, 16, 32]), 100,
                             0, opt)
    elif kind == "per_run":
        init = np.tile(np.array([16, 16, 32]), (100, 1))
        ctx = pkg.ssa_create(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, [1.0, 1.0, 1.0], init, 100, 0, opt)
    else:
        init = np.array([[16, 16, 32], [25, 25, 50]])
        ctx = pkg.ssa_create_batch(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, init, np.ones((2, 3)),
                                   np.array([64, 40]), np.array([1, 2], dtype=np.uint64), opt)
    try:
        pkg.ssa_run(ctx, 1.0, [0.1, 0.5])
    finally:
        pkg.ssa_destroy(ctx)


@pytest.mark.parametrize("kind", ["single", "per_run", "batch"])
def test_allocation_failure_returns_enomem_without_leak(torch_cuda, kind):
    torch = torch_cuda
    opt = pkg.ssa_default_options(cuda_stream=torch.cuda.current_stream(), keep_snap_counts=1)
    full = BudgetAllocator(torch, None)
    pkg.ssa_set_allocator(full.alloc, full.release)
    _create_and_run(kind, opt)
    assert not full.live and full.calls > 0
    for budget in range(full.calls):
        a = BudgetAllocator(torch, budget)
        pkg.ssa_set_allocator(a.alloc, a.release)
        with pytest.raises(pkg.SSAError) as ei:
            _create_and_run(kind, opt)
        assert ei.value.status == pkg.SSA_ENOMEM, (budget, ei.value)
        assert not a.live, (budget, a.live)
    pkg.use_torch_allocator()
