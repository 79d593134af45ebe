"""The C-ABI library: it builds, loads, exports every declared symbol, and
validates its arguments before touching the GPU (runs on CPU)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2412_16613_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return pkg.lib()


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("typedef",) and not text[m.start():m.end()].lstrip().startswith("typedef"):
                names.add(name)
    return names


def test_headers_declare_the_boundary():
    names = declared_functions()
    for n in ["ssa_create", "ssa_create_batch", "ssa_run", "ssa_fetch", "ssa_destroy", "ssa_last_error",
              "ssa_set_allocator", "ssa_default_options", "ssa_field_bytes", "ssa_version", "ssa_tune",
              "bitssa_test_philox", "bitssa_test_bitslice", "bitssa_bench_alu", "ssa_lattice_create",
              "ssa_lattice_run", "ssa_lattice_fetch", "ssa_lattice_field_bytes", "ssa_lattice_destroy",
              "ssa_lattice_last_error"]:
        assert n in names, n


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = declared_functions() - exported
    assert not missing, missing
    for n in declared_functions():
        assert getattr(lib, n) is not None


def test_default_options(lib):
    o = pkg.ssa_default_options()
    assert o.precision == pkg.SSA_P64 and o.engine == pkg.SSA_ENGINE_BITSLICED
    assert o.thin_bits == 32 and o.device == -1 and o.step_budget == 0 and o.first_run == 0
    assert C.sizeof(pkg.ssa_options) == 96
    assert o.clock == pkg.SSA_CLOCK_GROUP and o.word_width == 0 and o.tail_groups == 0


def _create(reac, prod, rates=(1.0, 1.0, 1.0), N0=(16, 16, 32), n_runs=64, **opt):
    return pkg.ssa_create(reac, prod, rates, N0, n_runs, 0, pkg.ssa_default_options(**opt))


F_R, F_P = pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS


@pytest.mark.parametrize("kw,status", [
    (dict(reac=[[1, 1, 1], [0, 1, 1], [1, 1, 0]], prod=F_P), pkg.SSA_EINVAL),      # order 3
    (dict(reac=F_R, prod=[[2, 0, 1], [0, 2, 0], [0, 0, 2]]), pkg.SSA_EINVAL),      # not conserving
    (dict(reac=F_R, prod=F_P, rates=(1.0, -1.0, 1.0)), pkg.SSA_EINVAL),            # negative rate
    (dict(reac=F_R, prod=F_P, rates=(0.0, 0.0, 0.0)), pkg.SSA_EINVAL),             # no positive rate
    (dict(reac=F_R, prod=F_P, rates=(1.0, float("nan"), 1.0)), pkg.SSA_EINVAL),    # nan rate
    (dict(reac=F_R, prod=F_P, N0=(0, 0, 0)), pkg.SSA_EINVAL),                      # empty system
    (dict(reac=F_R, prod=F_P, N0=(-1, 1, 1)), pkg.SSA_EINVAL),                     # negative count
    (dict(reac=F_R, prod=F_P, N0=(30000, 30000, 6000)), pkg.SSA_EUNSUPPORTED),     # N_tot > 65536
    (dict(reac=F_R, prod=F_P, n_runs=-1), pkg.SSA_EINVAL),
    (dict(reac=F_R, prod=F_P, thin_bits=0), pkg.SSA_EINVAL),
    (dict(reac=F_R, prod=F_P, thin_bits=65), pkg.SSA_EINVAL),
    (dict(reac=F_R, prod=F_P, precision=7), pkg.SSA_EINVAL),
    (dict(reac=F_R, prod=F_P, block_size=48), pkg.SSA_EINVAL),
    (dict(reac=F_R, prod=F_P, first_run=16), pkg.SSA_EINVAL),
    (dict(reac=F_R, prod=F_P, layout=3), pkg.SSA_EINVAL),
    (dict(reac=F_R, prod=F_P, shared_n=2), pkg.SSA_EINVAL),
    (dict(reac=F_R, prod=F_P, shared_n=1, engine=pkg.SSA_ENGINE_THREAD_PER_RUN), pkg.SSA_EUNSUPPORTED),
    (dict(reac=F_R, prod=F_P, shared_n=1, layout=pkg.SSA_LAYOUT_THREAD), pkg.SSA_EUNSUPPORTED),
    (dict(reac=F_R, prod=F_P, pad_pow2=3), pkg.SSA_EINVAL),
    (dict(reac=F_R, prod=F_P, pad_pow2=2, layout=pkg.SSA_LAYOUT_WARPS), pkg.SSA_EUNSUPPORTED),
    (dict(reac=F_R, prod=F_P, pad_pow2=2, shared_n=1), pkg.SSA_EUNSUPPORTED),
    (dict(reac=F_R, prod=F_P, pad_pow2=2, engine=pkg.SSA_ENGINE_GENERAL), pkg.SSA_EUNSUPPORTED),
    (dict(reac=F_R, prod=F_P, pad_pow2=2, engine=pkg.SSA_ENGINE_THREAD_PER_RUN), pkg.SSA_EUNSUPPORTED),
    (dict(reac=[[1, 1], [1, 1]], prod=[[2, 0], [0, 2]], N0=(3, 3), pad_pow2=2), pkg.SSA_EUNSUPPORTED),
    (dict(reac=F_R, prod=F_P, pad_pow2=-1), pkg.SSA_EINVAL),
    (dict(reac=F_R, prod=F_P, pad_pow2=1, engine=pkg.SSA_ENGINE_THREAD_PER_RUN), pkg.SSA_EUNSUPPORTED),
    (dict(reac=[[1] + [0] * 8], prod=[[0, 1] + [0] * 7]), pkg.SSA_EUNSUPPORTED),    # 9 species
    (dict(reac=[[1, 0]] * 9, prod=[[0, 1]] * 9, rates=[1.0] * 9, N0=(3, 3)), pkg.SSA_EUNSUPPORTED),  # 9 reactions
    (dict(reac=[[1, 1], [1, 1]], prod=[[2, 0], [0, 2]], N0=(32768, 32768)), pkg.SSA_EUNSUPPORTED),  # bound >= 2^31
    (dict(reac=[[1, 1], [1, 1]], prod=[[2, 0], [0, 2]], N0=(3, 3), rates=(1.0, -1.0)), pkg.SSA_EINVAL),
    (dict(reac=[[1, 1], [1, 1]], prod=[[2, 0], [0, 2]], N0=(3, 3), engine=pkg.SSA_ENGINE_THREAD_PER_RUN),
     pkg.SSA_EUNSUPPORTED),                                                           # baseline: Frank only
    (dict(reac=[[1, 1], [1, 1]], prod=[[2, 0], [0, 2]], N0=(3, 3), layout=pkg.SSA_LAYOUT_WARPS),
     pkg.SSA_EUNSUPPORTED),                                                           # general: one layout
    (dict(reac=F_R, prod=F_P, engine=pkg.SSA_ENGINE_GENERAL, layout=pkg.SSA_LAYOUT_WARPS), pkg.SSA_EUNSUPPORTED),
    (dict(reac=F_R, prod=F_P, engine=3), pkg.SSA_EINVAL),
    (dict(reac=F_R, prod=F_P, recompute=4), pkg.SSA_EINVAL),
    (dict(reac=F_R, prod=F_P, clock=2), pkg.SSA_EINVAL),
    (dict(reac=F_R, prod=F_P, word_width=16), pkg.SSA_EINVAL),
    (dict(reac=F_R, prod=F_P, word_width=64), pkg.SSA_EUNSUPPORTED),
    (dict(reac=F_R, prod=F_P, tail_groups=5), pkg.SSA_EINVAL),
    (dict(reac=F_R, prod=F_P, clock=pkg.SSA_CLOCK_LANE, layout=pkg.SSA_LAYOUT_WARPS), pkg.SSA_EUNSUPPORTED),
    (dict(reac=F_R, prod=F_P, clock=pkg.SSA_CLOCK_LANE, pad_pow2=2), pkg.SSA_EUNSUPPORTED),
    (dict(reac=F_R, prod=F_P, clock=pkg.SSA_CLOCK_LANE, shared_n=1), pkg.SSA_EUNSUPPORTED),
    (dict(reac=F_R, prod=F_P, clock=pkg.SSA_CLOCK_LANE, engine=pkg.SSA_ENGINE_GENERAL), pkg.SSA_EUNSUPPORTED),
    (dict(reac=F_R, prod=F_P, clock=pkg.SSA_CLOCK_LANE, engine=pkg.SSA_ENGINE_THREAD_PER_RUN), pkg.SSA_EUNSUPPORTED),
    (dict(reac=F_R, prod=F_P, clock=pkg.SSA_CLOCK_LANE, block_size=256), pkg.SSA_EUNSUPPORTED),
    (dict(reac=[[1, 1], [1, 1]], prod=[[2, 0], [0, 2]], N0=(3, 3), clock=pkg.SSA_CLOCK_LANE), pkg.SSA_EUNSUPPORTED),
    (dict(reac=F_R, prod=F_P, tail_groups=-2), pkg.SSA_EINVAL),
])
def test_validation_before_any_cuda_call(lib, kw, status):
    with pytest.raises(pkg.SSAError) as ei:
        _create(**kw)
    assert ei.value.status == status
    assert pkg.ssa_last_error()


def test_per_run_totals_must_agree(lib):
    N0 = np.array([[16, 16, 32], [16, 16, 31]])
    with pytest.raises(pkg.SSAError) as ei:
        pkg.ssa_create(F_R, F_P, [1, 1, 1], N0, 2, 0)
    assert ei.value.status == pkg.SSA_EINVAL


def test_null_and_order_errors(lib):
    L = lib
    assert L.ssa_run(None, 1.0, None, 0) == pkg.SSA_EINVAL
    assert L.ssa_fetch(None, 0, None, 0, 0) == pkg.SSA_EINVAL
    assert L.ssa_destroy(None) == pkg.SSA_OK
    ctx = C.c_void_p()
    assert L.ssa_create(None, None, 3, 3, None, None, 0, 1, 0, None, C.byref(ctx)) == pkg.SSA_EINVAL
    assert not ctx.value


@pytest.mark.parametrize("reac,prod,N0", [
    ([[1, 0, 1], [0, 1, 1]], [[2, 0, 0], [0, 2, 0]], (3, 3, 3)),                          # not Frank
    ([[1, 1, 0], [0, 1, 1], [1, 0, 1]], [[0, 0, 2], [0, 2, 0], [2, 0, 0]], (3, 3, 3)),     # Frank, other order
    ([[1, 1, 0], [0, 1, 0]], [[0, 2, 0], [0, 0, 1]], (9, 1, 0)),                          # S + I -> 2I, I -> R
    ([[2]], [[2]], (5,)),                                                                 # one species
])
def test_general_networks_pass_validation(lib, reac, prod, N0):
    """Networks that are not Frank's model go to the general kernel: validation accepts them
    and, without a GPU, the call stops at the device."""
    try:
        ctx = _create(reac, prod, rates=[1.0] * len(reac), N0=N0)
    except pkg.SSAError as e:
        assert e.status == pkg.SSA_ECUDA  # no device here
    else:
        pkg.ssa_destroy(ctx)


def test_frank_relabelled_passes_validation(lib):
    """Species order (A, L, D): validation accepts it; without a GPU the call stops at the device."""
    reac = [[1, 1, 0], [1, 0, 1], [0, 1, 1]]
    prod = [[0, 2, 0], [0, 0, 2], [2, 0, 0]]
    try:
        ctx = _create(reac, prod, N0=(32, 16, 16))
    except pkg.SSAError as e:
        assert e.status == pkg.SSA_ECUDA  # no device here
    else:
        pkg.ssa_destroy(ctx)


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle and has no host implementation of the step."""
    src_dir = os.path.join(ROOT, "paper_2412_16613_gb300")
    for name in os.listdir(src_dir):
        if name.endswith(".py"):
            text = open(os.path.join(src_dir, name)).read()
            assert "import oracle" not in text and "from oracle" not in text, name


@pytest.mark.parametrize("kw", [dict(pad_pow2=2, layout=pkg.SSA_LAYOUT_WARPS), dict(pad_pow2=2, shared_n=1),
                                dict(pad_pow2=2, engine=pkg.SSA_ENGINE_GENERAL), dict(pad_pow2=3),
                                dict(clock=pkg.SSA_CLOCK_LANE)])
def test_batch_validates_the_bound_option(lib, kw):
    """A batch goes through the same option checks, before any CUDA call."""
    init = np.array([[16, 16, 32], [25, 25, 50]])
    with pytest.raises(pkg.SSAError) as ei:
        pkg.ssa_create_batch(F_R, F_P, init, np.ones((2, 3)), np.array([64, 32]), np.array([1, 2], dtype=np.uint64),
                             pkg.ssa_default_options(**kw))
    assert ei.value.status == (pkg.SSA_EINVAL if kw.get("pad_pow2") == 3 else pkg.SSA_EUNSUPPORTED)


def _lattice_create(lx=4, ly=4, rates=(1.0, 1.0, 1.0), hop=0.1, N0=None, n_runs=32, cap_bits_max=0, **opt):
    if N0 is None:
        N0 = np.full((lx * ly if lx > 0 and ly > 0 else 1, 3), 2, dtype=np.int64)
    return pkg.ssa_lattice_create(lx, ly, rates, hop, N0, n_runs, 0, pkg.ssa_default_options(**opt),
                                  cap_bits_max=cap_bits_max)


@pytest.mark.parametrize("kw,status", [
    (dict(lx=3), pkg.SSA_EINVAL),                                   # sides are powers of two
    (dict(ly=0), pkg.SSA_EINVAL),
    (dict(lx=256, ly=128), pkg.SSA_EUNSUPPORTED),                   # more than 16384 sites
    (dict(rates=(0.0, 0.0, 0.0)), pkg.SSA_EINVAL),
    (dict(rates=(-1.0, 1.0, 1.0)), pkg.SSA_EINVAL),
    (dict(hop=0.0), pkg.SSA_EINVAL),
    (dict(hop=0.3), pkg.SSA_EINVAL),                                # k_max / d not an integer
    (dict(hop=1.0 / 70000), pkg.SSA_EUNSUPPORTED),                  # rho_r above 2^16
    (dict(N0=np.full((16, 3), -1)), pkg.SSA_EINVAL),
    (dict(N0=np.full((16, 3), 40000)), pkg.SSA_EINVAL),
    (dict(cap_bits_max=16), pkg.SSA_EINVAL),
    (dict(n_runs=-1), pkg.SSA_EINVAL),
    (dict(precision=7), pkg.SSA_EINVAL),
    (dict(thin_bits=0), pkg.SSA_EINVAL),
    (dict(block_size=48), pkg.SSA_EINVAL),
    (dict(block_size=512), pkg.SSA_EINVAL),
    (dict(first_run=5), pkg.SSA_EINVAL),
    (dict(clock=pkg.SSA_CLOCK_LANE), pkg.SSA_EUNSUPPORTED),
    (dict(pad_pow2=1), pkg.SSA_EUNSUPPORTED),
    (dict(engine=pkg.SSA_ENGINE_GENERAL), pkg.SSA_EUNSUPPORTED),
])
def test_lattice_validation_before_any_cuda_call(lib, kw, status):
    """ssa_lattice_create checks every argument before it touches the GPU."""
    with pytest.raises(pkg.SSAError) as ei:
        _lattice_create(**kw)
    assert ei.value.status == status
    assert pkg.ssa_lattice_last_error()
    assert pkg.ssa_last_error()  # the thread's message is shared with ssa_create's


def test_lattice_valid_arguments_reach_the_device(lib):
    """Valid arguments pass validation; without a GPU the call stops at the device."""
    try:
        ctx = _lattice_create(8, 8, N0=np.random.default_rng(0).poisson(3, size=(40, 64, 3)), n_runs=40)
    except pkg.SSAError as e:
        assert e.status == pkg.SSA_ECUDA
    else:
        pkg.ssa_lattice_destroy(ctx)
    L = lib
    assert L.ssa_lattice_run(None, 1.0, None, 0) == pkg.SSA_EINVAL
    assert L.ssa_lattice_fetch(None, 0, None, 0, 0) == pkg.SSA_EINVAL
    assert L.ssa_lattice_destroy(None) == pkg.SSA_OK
