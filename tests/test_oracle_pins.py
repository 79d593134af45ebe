"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: an
independent Philox implementation, exhaustive enumeration of the reaction
rule, the chemical master equation solved by expm / linear algebra, closed
forms of single-reaction networks, exact one-step probabilities, and the
invariants of the Frank model (Sec. 2).
"""
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
from scipy import stats

from tests import _master_equation as me

FRANK_REAC = [[1, 0, 1], [0, 1, 1], [1, 1, 0]]
FRANK_PROD = [[2, 0, 0], [0, 2, 0], [0, 0, 2]]


def frank_h(L, D, A):
    """Eq. equation-as: a1 = A L, a2 = A D, a3 = L D (k_A = k_I = 1)."""
    return [A * L, A * D, L * D]


# --------------------------------------------------------------------------
# Philox4x32-10: the oracle's implementation against Triton's, run on the CPU
# by Triton's interpreter (an implementation written by other people).
# --------------------------------------------------------------------------
def test_philox_matches_triton_interpreter(orc):
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    ctrs = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64)
    ctrs[0] = 0
    ctrs[1] = 2**32 - 1
    seed = 0x0123456789ABCDEF
    code = textwrap.dedent("""
        import os, sys, json
        os.environ["TRITON_INTERPRET"] = "1"
        import torch, triton, triton.language as tl
        @triton.jit
        def k(c_ptr, o_ptr, seed, N: tl.constexpr):
            i = tl.arange(0, N)
            c0 = tl.load(c_ptr + 4 * i + 0)
            c1 = tl.load(c_ptr + 4 * i + 1)
            c2 = tl.load(c_ptr + 4 * i + 2)
            c3 = tl.load(c_ptr + 4 * i + 3)
            a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
            tl.store(o_ptr + 4 * i + 0, a)
            tl.store(o_ptr + 4 * i + 1, b)
            tl.store(o_ptr + 4 * i + 2, c)
            tl.store(o_ptr + 4 * i + 3, d)
        ctr = torch.tensor(json.loads(sys.argv[1]), dtype=torch.int64).to(torch.uint32)
        out = torch.zeros_like(ctr)
        k[(1,)](ctr, out, int(sys.argv[2]), N=ctr.shape[0])
        print(json.dumps(out.to(torch.int64).tolist()))
    """)
    import json
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", code, json.dumps(ctrs.tolist()), str(seed)],
                       capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        pytest.skip(f"triton interpreter unavailable: {r.stderr[-300:]}")
    theirs = json.loads(r.stdout.strip().splitlines()[-1])
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for c, t in zip(ctrs.tolist(), theirs):
        assert orc.philox4x32_10(c, key) == t


def test_stream_word_layout(orc):
    """Word k of a stream is element k % 4 of Philox call k // 4 on the documented counter."""
    seed, g, s = 0xDEADBEEFCAFEF00D, 12345, (7 << 32) | 99
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for attempt, tag in [(0, 0), (3, 0), (0, 1)]:
        for k in range(10):
            ctr = [g, s & 0xFFFFFFFF, ((s >> 32) & 0xFFFF) | (attempt << 16) | (tag << 24), k // 4]
            assert orc.stream_word(seed, g, s, attempt, tag, k) == orc.philox4x32_10(ctr, key)[k % 4]


# --------------------------------------------------------------------------
# The uniformisation constant (Eq. equation-z) and its generalisation.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N,K", [(64, 11), (1024, 19), (10000, 26), (65536, 31)])
def test_lambda_frank_is_Z(orc, N, K):
    d = orc.derive(orc.frank(), N)
    assert d.lambda_int == N * (N - 1) // 2          # Eq. equation-z
    assert d.K == K and 2 ** (K - 1) <= d.lambda_int < 2 ** K
    assert d.lambda_ == float(N * (N - 1) // 2)


@pytest.mark.parametrize("N,K", [(12, 7), (64, 11), (1024, 19), (46400, 31), (65536, 31)])
def test_lambda_padded_to_a_power_of_two(orc, N, K):
    """Padding keeps K (the bit length of Z) and raises the bound to 2^K > Z."""
    d = orc.derive(orc.frank(1.0, 0.5, 2.0), N, pad_pow2=True)
    assert d.K == K and d.lambda_int == 2 ** K > N * (N - 1) // 2
    assert d.lambda_ == 2.0 * 2 ** K


def test_lambda_is_a_bound_by_brute_force(orc):
    """max over all states of sum_r h_r <= lambda_int, with equality for Frank + ghosts."""
    nets = [
        (FRANK_REAC, FRANK_PROD),
        ([[1, 0, 1], [1, 0, 1], [0, 2, 0]], [[2, 0, 0], [0, 1, 1], [1, 1, 0]]),  # pair used twice
        ([[1, 0, 0], [0, 1, 0], [1, 1, 0]], [[0, 1, 0], [1, 0, 0], [0, 0, 2]]),  # first order
    ]
    for reac, prod in nets:
        net = orc.Network(reac, prod, [1.0] * len(reac))
        for N in (5, 9, 16):
            d = orc.derive(net, N)
            best = max(sum(me.propensity(r, s) for r in reac) for s in me.states(3, N))
            assert best <= d.lambda_int
    # Frank: sum of the three real and three ghost propensities is exactly Z for every state
    for s in me.states(3, 12):
        L, D, A = s
        ghosts = L * (L - 1) // 2 + D * (D - 1) // 2 + A * (A - 1) // 2
        assert sum(frank_h(L, D, A)) + ghosts == 12 * 11 // 2


# --------------------------------------------------------------------------
# The reaction rule: the CDF walk (Sec. 3 step 5, Fig. 2) must give each
# reaction exactly h_r of the lambda_int integers, ghosts the rest.
# --------------------------------------------------------------------------
def test_select_exhaustive_small(orc):
    net = orc.frank()
    for N in (2, 3, 7, 12):
        Z = N * (N - 1) // 2
        for (L, D, A) in me.states(3, N):
            counts = [0, 0, 0, 0]
            for n in range(Z):
                counts[orc.select(net, (L, D, A), n) + 1] += 1
            h = frank_h(L, D, A)
            assert counts[1:] == h
            assert counts[0] == Z - sum(h)


def test_select_boundaries_N64(orc):
    net = orc.frank()
    N, Z = 64, 2016
    for (L, D, A) in me.states(3, N):
        h = frank_h(L, D, A)
        S = np.cumsum(h)
        lo = 0
        for r in range(3):
            if h[r]:
                assert orc.select(net, (L, D, A), lo) == r
                assert orc.select(net, (L, D, A), S[r] - 1) == r
            lo = S[r]
        if S[2] < Z:
            assert orc.select(net, (L, D, A), S[2]) == -1
            assert orc.select(net, (L, D, A), Z - 1) == -1


def test_propensities_definition(orc):
    net = orc.frank()
    for (L, D, A) in me.states(3, 9):
        assert list(orc.propensities(net, (L, D, A))) == frank_h(L, D, A)


# --------------------------------------------------------------------------
# One step: the drawn integer is uniform on [0, lambda_int), so the first
# reaction has probability k_r h_r / (k_max lambda_int) exactly.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("rates", [(1.0, 1.0, 1.0), (1.0, 0.5, 0.25), (0.7, 2.0, 1.3)])
def test_first_step_probabilities(orc, rates):
    net = orc.frank(*rates)
    init = (16, 16, 32)
    n = 200_000
    r = orc.run(net, init, n, seed=11, step_budget=1, check=False)
    assert np.all((r["run_status"] == orc.OK) | (r["run_status"] == orc.ETIMEOUT))
    delta = r["final_counts"] - np.array(init)
    fired = np.full(n, 3)
    fired[(delta == [1, 0, -1]).all(1)] = 0
    fired[(delta == [0, 1, -1]).all(1)] = 1
    fired[(delta == [-1, -1, 2]).all(1)] = 2
    assert np.all((fired == 3) == (delta == 0).all(1))
    Z = 64 * 63 // 2
    kmax = max(rates)
    h = frank_h(16, 16, 32)
    p = [rates[i] * h[i] / (kmax * Z) for i in range(3)]
    p.append(1 - sum(p))
    obs = np.bincount(fired, minlength=4)
    chi2, pval = stats.chisquare(obs, np.array(p) * n)
    assert pval > 1e-4, (obs, np.array(p) * n)


@pytest.mark.parametrize("init", [(1, 1, 10), (6, 0, 6), (2, 9, 1), (11, 1, 0), (4, 4, 4)])
def test_first_step_probabilities_under_heavy_rejection(orc, init):
    """N_tot = 12: lambda_int = 66 of 2^7 = 128 draws, so about half the draws are redrawn;
    the first reaction must still have probability h_r / 66 exactly, for states whose
    reactions cover different parts of [0, 66)."""
    n = 150_000
    r = orc.run(orc.frank(), init, n, seed=19, step_budget=1, check=False)
    delta = r["final_counts"] - np.array(init)
    fired = np.full(n, 3)
    for k, nu in enumerate(([1, 0, -1], [0, 1, -1], [-1, -1, 2])):
        fired[(delta == nu).all(1)] = k
    h = frank_h(*init)
    p = np.array(h + [66 - sum(h)], dtype=float) / 66
    obs = np.bincount(fired, minlength=4)
    keep = p > 0
    assert np.all(obs[~keep] == 0)
    assert stats.chisquare(obs[keep], p[keep] * n).pvalue > 1e-4, (obs, p * n)
    assert r["redraws"].sum() > 0.5 * n


@pytest.mark.parametrize("init", [(1, 1, 10), (6, 0, 6), (4, 4, 4)])
def test_first_step_probabilities_padded(orc, init):
    """With the bound padded to 2^7 = 128 at N_tot = 12, reaction r takes h_r of the 128
    equally likely draws and nothing is redrawn."""
    n = 150_000
    r = orc.run(orc.frank(), init, n, seed=23, step_budget=1, check=False, pad_pow2=True)
    delta = r["final_counts"] - np.array(init)
    fired = np.full(n, 3)
    for k, nu in enumerate(([1, 0, -1], [0, 1, -1], [-1, -1, 2])):
        fired[(delta == nu).all(1)] = k
    h = frank_h(*init)
    p = np.array(h + [128 - sum(h)], dtype=float) / 128
    obs = np.bincount(fired, minlength=4)
    keep = p > 0
    assert np.all(obs[~keep] == 0)
    assert stats.chisquare(obs[keep], p[keep] * n).pvalue > 1e-4, (obs, p * n)
    assert r["redraws"].sum() == 0


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_waiting_time_exponential(orc, precision):
    """Eq. equation-tau: tau ~ Exp(Lambda), one clock per 32-lane group."""
    net = orc.frank()
    N = 64
    Z = N * (N - 1) // 2
    groups = 40_000
    r = orc.run(net, (16, 16, 32), run_ids=np.arange(groups) * 32, seed=3, step_budget=1,
                precision=precision, check=False)
    tau = r["t_last"] * Z
    assert abs(tau.mean() - 1.0) < 4.5 / math.sqrt(groups)
    assert stats.kstest(tau, "expon").pvalue > 1e-4
    # lanes of one group share the clock
    r2 = orc.run(net, (16, 16, 32), run_ids=np.arange(8) * 32 + 5, seed=3, step_budget=1,
                 precision=precision, check=False)
    assert np.array_equal(r2["t_last"], r["t_last"][:8])


def test_padded_steps_scale_with_the_bound(orc):
    """Uniformisation at rate Lambda makes the expected number of steps before absorption
    Lambda E[T]: padding Z = 2016 to 2048 at N_tot = 64 keeps E[T] and scales the steps by
    2048 / 2016, with no redraws."""
    runs = 20_000
    ids = np.arange(runs) * 32 + 7
    a = orc.run(orc.frank(), (16, 16, 32), run_ids=ids, seed=8, t_end=np.inf)
    b = orc.run(orc.frank(), (16, 16, 32), run_ids=ids, seed=8, t_end=np.inf, pad_pow2=True)
    assert b["redraws"].sum() == 0 and a["redraws"].sum() > 0
    se_t = math.hypot(a["t_abs"].std(), b["t_abs"].std()) / math.sqrt(runs)
    assert abs(a["t_abs"].mean() - b["t_abs"].mean()) < 4.5 * se_t
    ratio = b["steps"].mean() / a["steps"].mean()
    se_r = ratio * math.hypot(a["steps"].std() / a["steps"].mean(),
                              b["steps"].std() / b["steps"].mean()) / math.sqrt(runs)
    assert abs(ratio - 2048 / 2016) < 4.5 * se_r
    # the real reactions do not depend on the bound: same law of the jump chain
    se_x = math.hypot(a["reactions"].std(), b["reactions"].std()) / math.sqrt(runs)
    assert abs(a["reactions"].mean() - b["reactions"].mean()) < 4.5 * se_x


def test_redraw_rate(orc):
    """n >= lambda_int is redrawn: extra attempts per step are geometric with p = 1 - Z / 2^K."""
    net = orc.frank()
    r = orc.run(net, (16, 16, 32), 4096, seed=5, t_end=np.inf)
    p = 1 - 2016 / 2048
    steps = r["steps"].sum()
    expected = steps * p / (1 - p)
    assert abs(r["redraws"].sum() - expected) < 5 * math.sqrt(expected)


# --------------------------------------------------------------------------
# The chemical master equation, N_tot = 12 (91 states).
# --------------------------------------------------------------------------
def _frank_me(N, rates=(1.0, 1.0, 1.0)):
    return me.generator(FRANK_REAC, FRANK_PROD, list(rates), N)


@pytest.mark.parametrize("lane,shared,pad", [(0, False, False), (17, False, False), (17, True, False),
                                            (5, False, True), (9, True, True), (0, False, 2), (23, False, 2)])
def test_master_equation_distribution(orc, lane, shared, pad):
    """Each lane is an exact sample path, also when it reacts to the n of its group's lane 0
    (one n for all copies, Sec. 4 step a): n never depends on the state; also with the
    bound padded from Z = 66 to 128 (uniformisation at a larger rate); and with a bound that
    follows the state of the lane's whole group (pad = 2: a rate that changes between steps)."""
    N, init = 12, (3, 3, 6)
    st, index, Q = _frank_me(N)
    snaps = [0.02, 0.05, 0.1, 0.2, 0.4]
    runs = 40_000 if pad != 2 else 20_000
    # one lane per group: groups draw from independent counters
    r = orc.run(orc.frank(), init, run_ids=np.arange(runs) * 32 + lane, seed=21, t_end=0.5,
                snap_times=snaps, shared_n=shared, pad_pow2=pad)
    p0 = np.zeros(len(st))
    p0[index[init]] = 1.0
    for s, t in enumerate(snaps):
        p = me.distribution(Q, p0, t)
        obs = np.zeros(len(st))
        for c in r["snap_counts"][s]:
            obs[index[tuple(int(x) for x in c)]] += 1
        exp = p * runs
        big = exp >= 5
        o = np.append(obs[big], obs[~big].sum())
        e = np.append(exp[big], exp[~big].sum())
        if e[-1] < 5:
            o, e = o[:-1], e[:-1]
            e *= o.sum() / e.sum()
        stat, pval = stats.power_divergence(o, e, lambda_="log-likelihood")
        assert pval > 1e-4, (t, pval)


GENERAL_NETWORKS = [
    # 2A -> A + B, A + B -> 2A, B -> A: a homodimer, a pair, a first-order reaction, thinning
    ([[2, 0], [1, 1], [0, 1]], [[1, 1], [2, 0], [1, 0]], [1.0, 0.5, 3.0], (7, 3)),
    # S + I -> 2I, I -> R (u_max = 1 next to a pair)
    ([[1, 1, 0], [0, 1, 0]], [[0, 2, 0], [0, 0, 1]], [1.0, 0.7], (8, 2, 0)),
    # two reactions on one pair (m_pair = 2) and a zero rate
    ([[1, 1, 0], [1, 1, 0], [0, 0, 1]], [[2, 0, 0], [0, 2, 0], [1, 0, 0]], [1.0, 2.0, 0.0], (4, 4, 2)),
    # four species
    ([[1, 1, 0, 0], [0, 0, 1, 1], [0, 1, 0, 0], [0, 0, 2, 0]],
     [[0, 0, 2, 0], [2, 0, 0, 0], [0, 0, 0, 1], [1, 1, 0, 0]], [1.0, 0.8, 2.0, 0.5], (3, 2, 2, 1)),
]


@pytest.mark.parametrize("net_i", range(len(GENERAL_NETWORKS)))
@pytest.mark.parametrize("pad", [False, True])
def test_master_equation_general_networks(orc, net_i, pad):
    """Networks other than Frank's (order-2 pairs and homodimers, first-order reactions,
    m_pair = 2, four species, non-unit and zero rates) against the master equation."""
    reac, prod, rates, init = GENERAL_NETWORKS[net_i]
    N = sum(init)
    st, index, Q = me.generator(reac, prod, rates, N)
    snaps = [0.05, 0.2, 0.6]
    runs = 30_000
    r = orc.run(orc.Network(reac, prod, rates), init, run_ids=np.arange(runs) * 32 + 11, seed=77 + net_i,
                t_end=0.6, snap_times=snaps, pad_pow2=pad)
    p0 = np.zeros(len(st))
    p0[index[init]] = 1.0
    for s, t in enumerate(snaps):
        p = me.distribution(Q, p0, t)
        obs = np.zeros(len(st))
        for c in r["snap_counts"][s]:
            obs[index[tuple(int(x) for x in c)]] += 1
        exp = p * runs
        big = exp >= 5
        o = np.append(obs[big], obs[~big].sum())
        e = np.append(exp[big], exp[~big].sum())
        if e[-1] < 5:
            o, e = o[:-1], e[:-1]
            e *= o.sum() / e.sum()
        assert stats.power_divergence(o, e, lambda_="log-likelihood")[1] > 1e-4, (t, net_i)


def test_shared_n_lanes_follow_one_draw(orc):
    """Shared n: from one initial state every lane of a group repeats lane 0's run (the reason
    the paper's shared draw needs distinct initial states); lane 0 itself is the run it is
    without sharing; with per-run initial states the lanes differ and each conserves N."""
    r = orc.run(orc.frank(), (40, 40, 80), 96, seed=3, t_end=5.0, shared_n=True)
    for g in range(3):
        sl = slice(32 * g, 32 * g + 32)
        assert np.all(r["final_counts"][sl] == r["final_counts"][32 * g])
        assert np.all(r["t_abs"][sl] == r["t_abs"][32 * g]) and np.all(r["steps"][sl] == r["steps"][32 * g])
    rng = np.random.default_rng(4)
    init = rng.multinomial(160, [0.25, 0.25, 0.5], size=96)
    a = orc.run(orc.frank(), init, seed=3, t_end=5.0, shared_n=True)
    b = orc.run(orc.frank(), init, seed=3, t_end=5.0, shared_n=False)
    for g in range(3):
        assert np.array_equal(a["final_counts"][32 * g], b["final_counts"][32 * g])
        assert a["t_abs"][32 * g] == b["t_abs"][32 * g] or (np.isinf(a["t_abs"][32 * g]) and np.isinf(b["t_abs"][32 * g]))
        assert a["steps"][32 * g] == b["steps"][32 * g]
    assert np.all(a["final_counts"].sum(1) == 160)
    assert len({tuple(x) for x in a["final_counts"][:32]}) > 1


@pytest.mark.parametrize("pad", [False, True, 2])
def test_master_equation_absorption(orc, pad):
    """Absorption probabilities and mean absorption time from the fundamental matrix."""
    N, init = 12, (5, 2, 5)
    st, index, Q = _frank_me(N)
    absorbing, B, T, transient = me.absorption(Q)
    i0 = transient.index(index[init])
    runs = 40_000 if pad != 2 else 20_000
    r = orc.run(orc.frank(), init, run_ids=np.arange(runs) * 32, seed=33, t_end=np.inf, pad_pow2=pad)
    assert np.all(r["outcome"] >= 0)
    for col, a in enumerate(absorbing):
        survivor = int(np.argmax(st[a]))
        p = B[i0, col]
        frac = np.mean(r["outcome"] == survivor)
        assert abs(frac - p) < 4.5 * math.sqrt(p * (1 - p) / runs) + 1e-12, (st[a], frac, p)
    se = r["t_abs"].std() / math.sqrt(runs)
    assert abs(r["t_abs"].mean() - T[i0]) < 4.5 * se


# --------------------------------------------------------------------------
# Closed forms of single-reaction networks.
# --------------------------------------------------------------------------
def test_closed_form_inhibition_only(orc):
    """L+D->2A alone from L = D = m0: T = sum_{m=1}^{m0} Exp(m^2)."""
    net = orc.Network([[1, 1, 0]], [[0, 0, 2]], [1.0])
    m0, A0 = 8, 4
    runs = 40_000
    r = orc.run(net, (m0, m0, A0), run_ids=np.arange(runs) * 32, seed=44, t_end=np.inf)
    assert np.all(r["final_counts"] == [0, 0, 2 * m0 + A0])
    mean = sum(1 / m**2 for m in range(1, m0 + 1))
    var = sum(1 / m**4 for m in range(1, m0 + 1))
    assert abs(r["t_abs"].mean() - mean) < 4.5 * math.sqrt(var / runs)
    assert abs(r["t_abs"].var() - var) < 0.05 * var
    assert np.all(r["reactions"] == m0)


def test_closed_form_autocatalysis_only(orc):
    """A+L->2L alone from (L0, 0, N-L0): T = sum_{L=L0}^{N-1} Exp(L (N-L))."""
    net = orc.Network([[1, 0, 1]], [[2, 0, 0]], [1.0])
    N, L0 = 20, 3
    runs = 40_000
    r = orc.run(net, (L0, 0, N - L0), run_ids=np.arange(runs) * 32 + 3, seed=45, t_end=np.inf)
    assert np.all(r["final_counts"] == [N, 0, 0])
    rates = [L * (N - L) for L in range(L0, N)]
    mean = sum(1 / a for a in rates)
    var = sum(1 / a**2 for a in rates)
    assert abs(r["t_abs"].mean() - mean) < 4.5 * math.sqrt(var / runs)


@pytest.mark.parametrize("init,final", [((1, 1, 0), (0, 0, 2)), ((1, 0, 1), (2, 0, 0))])
def test_two_molecules_exponential(orc, init, final):
    runs = 40_000
    r = orc.run(orc.frank(), init, run_ids=np.arange(runs) * 32, seed=46, t_end=np.inf)
    assert np.all(r["final_counts"] == final)
    assert stats.kstest(r["t_abs"], "expon").pvalue > 1e-4


# --------------------------------------------------------------------------
# Invariants of the Frank model (Sec. 2) and the L <-> D symmetry.
# --------------------------------------------------------------------------
def test_frank_invariants_and_symmetry(orc):
    runs = 20_000
    snaps = [0.01, 0.05, 0.1, 0.3]
    r = orc.run(orc.frank(), (16, 16, 32), runs, seed=8, t_end=1e9, snap_times=snaps)
    fc = r["final_counts"]
    assert np.all(fc.sum(1) == 64)
    assert np.all((fc > 0).sum(1) == 1)               # a single species survives
    assert np.all(r["outcome"] == np.argmax(fc, 1))
    assert np.all(r["snap_counts"].sum(2) == 64)
    pL = np.mean(r["outcome"] == 0)
    pD = np.mean(r["outcome"] == 1)
    se = math.sqrt((pL + pD) / runs)
    assert abs(pL - pD) < 4.5 * se
    for s in range(len(snaps)):
        L = r["snap_counts"][s, :, 0].astype(float)
        D = r["snap_counts"][s, :, 1].astype(float)
        ee = np.where(L + D > 0, (L - D) / np.maximum(L + D, 1), 0.0)
        assert abs(ee.mean()) < 4.5 * ee.std() / math.sqrt(runs) + 1e-12


def test_precision_modes_share_the_trajectory(orc):
    """The integer stream does not depend on the clock: counts and steps agree across modes."""
    base = orc.run(orc.frank(), (16, 16, 32), 512, seed=9, t_end=np.inf)
    for prec in (orc.P32_KAHAN, orc.P32_D64ACC):
        r = orc.run(orc.frank(), (16, 16, 32), 512, seed=9, t_end=np.inf, precision=prec)
        assert np.array_equal(r["final_counts"], base["final_counts"])
        assert np.array_equal(r["steps"], base["steps"])
        # the fp32 uniform is the top 24 bits of the fp64 one, so the clocks are paired
        rel = np.abs(r["t_abs"] / base["t_abs"] - 1)
        assert np.median(rel) < 1e-5 and np.quantile(rel, 0.99) < 1e-3


def test_plain_fp32_sum_shares_the_trajectory_and_loses_more(orc):
    """The plain fp32 clock (Eq. eq-update-time summed in fp32 without compensation): the same
    counts and steps as the other modes, every time an fp32 value, and a larger error against the
    fp64 sum than the Kahan-compensated fp32 sum of the same fp32 waiting times.  An fp64
    accumulator in its place would give times that are not fp32 values; a compensated sum would
    give Kahan's error."""
    init, n, th = (256, 256, 512), 256, os.cpu_count() or 4  # about 16 000 steps a run
    base = orc.run(orc.frank(), init, n, seed=11, t_end=np.inf, threads=th)
    kahan = orc.run(orc.frank(), init, n, seed=11, t_end=np.inf, precision=orc.P32_KAHAN, threads=th)
    plain = orc.run(orc.frank(), init, n, seed=11, t_end=np.inf, precision=orc.P32_PLAIN, threads=th)
    for r in (kahan, plain):
        assert np.array_equal(r["final_counts"], base["final_counts"])
        assert np.array_equal(r["steps"], base["steps"])
    assert np.array_equal(plain["t_abs"].astype(np.float32).astype(np.float64), plain["t_abs"])
    assert np.array_equal(plain["t_last"].astype(np.float32).astype(np.float64), plain["t_last"])
    rel_k = np.abs(kahan["t_abs"] / base["t_abs"] - 1)
    rel_p = np.abs(plain["t_abs"] / base["t_abs"] - 1)
    assert np.median(rel_p) > 2.0 * np.median(rel_k), (np.median(rel_p), np.median(rel_k))
    assert np.median(rel_p) < 1e-4


def test_ee_bin_definition(orc):
    assert orc.ee_bin(0, 0) == 64
    assert orc.ee_bin(0, 7) == 0          # ee = -1
    assert orc.ee_bin(7, 0) == 63         # ee = +1 folds into the top bin
    assert orc.ee_bin(5, 5) == 32         # ee = 0
    for L in range(0, 40):
        for D in range(0, 40):
            if L + D:
                ee = (L - D) / (L + D)
                assert orc.ee_bin(L, D) == min(63, math.floor((ee + 1) / 2 * 64 + 1e-12))


# --------------------------------------------------------------------------
# Degenerate cases and errors.
# --------------------------------------------------------------------------
def test_degenerate_cases(orc):
    net = orc.frank()
    r = orc.run(net, (1, 0, 0), 3, seed=1, t_end=5.0, snap_times=[0.0, 1.0])  # N = 1: no pair
    assert np.all(r["t_abs"] == 0.0) and np.all(r["outcome"] == 0) and np.all(r["steps"] == 0)
    assert np.all(r["snap_counts"] == [1, 0, 0])
    r = orc.run(net, (0, 0, 30), 3, seed=1, t_end=5.0)           # absorbed all-A start
    assert np.all(r["t_abs"] == 0.0) and np.all(r["outcome"] == 2)
    r = orc.run(net, (10, 10, 10), 64, seed=1, t_end=0.0, snap_times=[0.0])  # nothing happens by t=0
    assert np.all(r["final_counts"] == [10, 10, 10]) and np.all(r["steps"] == 0)
    assert np.all(r["outcome"] == -1) and np.all(np.isinf(r["t_abs"]))
    assert np.all(r["snap_counts"] == [10, 10, 10])
    r = orc.run(net, (10, 10, 10), 4, seed=1, t_end=np.inf, step_budget=5, check=False)
    assert r["status"] == orc.ETIMEOUT and np.all(r["steps"] == 5)


@pytest.mark.parametrize("reac,prod,rates", [
    ([[1, 1, 1]], [[3, 0, 0]], [1.0]),          # order 3
    ([[1, 0, 1]], [[2, 0, 1]], [1.0]),          # not conserving
    ([[1, 0, 1]], [[2, 0, 0]], [-1.0]),         # negative rate
    ([[1, 0, 1]], [[2, 0, 0]], [0.0]),          # no positive rate
])
def test_invalid_networks(orc, reac, prod, rates):
    with pytest.raises(ValueError):
        orc.derive(orc.Network(reac, prod, rates), 10)


def test_invalid_snapshots(orc):
    with pytest.raises(ValueError):
        orc.derive(orc.frank(), 10, t_end=1.0, snap_times=[0.5, 0.2])
    with pytest.raises(ValueError):
        orc.derive(orc.frank(), 10, t_end=1.0, snap_times=[2.0])


# --------------------------------------------------------------------------
# The paper's printed rules and examples (tests/golden).
# --------------------------------------------------------------------------
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _appendix_rules():
    rules = []
    with open(os.path.join(GOLDEN, "appendix_a_increments.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                r, a, expr = line.split()
                rules.append((int(r), a, expr))
    return rules


def test_appendix_a_increments_match_products():
    """App. A (Eqs. equation-a-nobit-1..3): each printed increment, in pre-update counts,
    equals the change of the recomputed product; unlisted propensities do not change."""
    nu = {1: (1, 0, -1), 2: (0, 1, -1), 3: (-1, -1, 2)}     # Eq. eq_nu

    def a_all(L, D, A):
        return {"a1": A * L, "a2": A * D, "a3": L * D, "a4": L * (L - 1) // 2,
                "a5": D * (D - 1) // 2, "a6": A * (A - 1) // 2}

    rules = _appendix_rules()
    for N in range(2, 31):
        for (L, D, A) in me.states(3, N):
            before = a_all(L, D, A)
            for r, (dL, dD, dA) in nu.items():
                if min(L + dL, D + dD, A + dA) < 0:
                    continue
                after = a_all(L + dL, D + dD, A + dA)
                listed = {a: eval(expr, {}, {"L": L, "D": D, "A": A})
                          for rr, a, expr in rules if rr == r}
                for name in before:
                    assert after[name] - before[name] == listed.get(name, 0), (r, name, L, D, A)
                assert sum(after.values()) == sum(before.values())  # Z is conserved


def _golden_examples():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_bitwise_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split("=")
                vals[k.strip()] = [int(x) for x in v.split()]
    return vals


def test_sum_pseudocode_reading():
    """Sec. 4.1: the printed partial sum s = b1 & b2 cannot give Fig. 1's 1 + 1 = 2;
    the full-adder sum s = b1 ^ b2 ^ c with the printed carry can."""
    g = _golden_examples()

    def ripple(x, y, width, printed):
        c, out = 0, 0
        for i in range(width):
            b1, b2 = (x >> i) & 1, (y >> i) & 1
            s = (b1 & b2) if printed else (b1 ^ b2 ^ c)
            c = (b2 & (b1 | c)) | (b1 & c)          # the carry as printed
            out |= s << i
        return out | (c << width)

    a, b, want = g["fig1_augend"][0], g["fig1_addend"][0], g["fig1_sum"][0]
    assert ripple(a, b, 1, printed=False) == want
    assert ripple(a, b, 1, printed=True) != want
    for x in range(16):
        for y in range(16):
            assert ripple(x, y, 4, printed=False) == x + y
    assert [p & q for p, q in zip(g["and_b1"], g["and_b2"])] == g["and_out"]


# --------------------------------------------------------------------------
# Closed forms of networks other than Frank's.
# --------------------------------------------------------------------------
def test_closed_form_isomerisation(orc):
    """A -> B at rate a, B -> A at rate b (first order, thinned when a != b): each molecule flips
    on its own, so n_A(t) is Bin(n_A0, p_AA(t)) + Bin(n_B0, p_BA(t)) with
    p_AA = (b + a e^{-(a+b)t}) / (a+b) and p_BA = b (1 - e^{-(a+b)t}) / (a+b)."""
    a, b = 1.0, 0.4
    nA0, nB0 = 14, 6
    net = orc.Network([[1, 0], [0, 1]], [[0, 1], [1, 0]], [a, b])
    snaps = [0.3, 1.2]
    runs = 40_000
    r = orc.run(net, (nA0, nB0), run_ids=np.arange(runs) * 32 + 2, seed=61, t_end=1.2, snap_times=snaps)
    for s, t in enumerate(snaps):
        e = math.exp(-(a + b) * t)
        p_aa, p_ba = (b + a * e) / (a + b), b * (1 - e) / (a + b)
        pmf = np.convolve(stats.binom.pmf(np.arange(nA0 + 1), nA0, p_aa), stats.binom.pmf(np.arange(nB0 + 1), nB0, p_ba))
        obs = np.bincount(r["snap_counts"][s][:, 0], minlength=nA0 + nB0 + 1).astype(float)
        exp = pmf * runs
        big = exp >= 5
        o, ex = np.append(obs[big], obs[~big].sum()), np.append(exp[big], exp[~big].sum())
        assert stats.power_divergence(o, ex, lambda_="log-likelihood")[1] > 1e-4, t


@pytest.mark.parametrize("k", [(1.0, 1.0), (1.0, 0.6)])
def test_closed_form_moran_fixation(orc, k):
    """A + B -> 2A (k1), A + B -> 2B (k2): the jump chain of n_A is a gambler's ruin with up-step
    probability p = k1 / (k1 + k2), so A fixes from i with probability (1 - (q/p)^i) / (1 - (q/p)^N)
    (i / N when p = 1/2)."""
    net = orc.Network([[1, 1], [1, 1]], [[2, 0], [0, 2]], list(k))
    i, N = 7, 20
    runs = 40_000
    r = orc.run(net, (i, N - i), run_ids=np.arange(runs) * 32 + 9, seed=71, t_end=np.inf)
    assert np.all(r["outcome"] >= 0)
    p = k[0] / (k[0] + k[1])
    rho = (1 - p) / p
    want = i / N if p == 0.5 else (1 - rho ** i) / (1 - rho ** N)
    got = np.mean(r["outcome"] == 0)
    assert abs(got - want) < 4.5 * math.sqrt(want * (1 - want) / runs), (got, want)


# --------------------------------------------------------------------------
# The bound that follows the group's state (pad_pow2 = 2).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("others", [None, (16, 16, 32)])
def test_state_following_bound_first_step(orc, others):
    """The first step of a run in state (1, 1, 62): reaction r with probability h_r / 2^p and a
    waiting time of mean 1 / 2^p, p the bit length of the largest S_R in the group. Alone with
    its copies S_R = 62 + 62 + 1 = 125 and 2^p = 128; next to runs in (16, 16, 32)
    (S_R = 1280) 2^p = 2048, the padded bound of N = 64."""
    groups = 6000
    init = np.tile(np.array([16, 16, 32] if others else [1, 1, 62]), (32 * groups, 1))
    init[::32] = (1, 1, 62)
    r = orc.run(orc.frank(), init, seed=41, step_budget=1, check=False, pad_pow2=2)
    bound = 2048 if others else 128
    lanes = np.arange(32 * groups) % 32 == 0 if others else np.ones(32 * groups, bool)
    fc = r["final_counts"][lanes]
    m = lanes.sum()
    h = np.array([62, 62, 1])
    got = [np.sum(fc[:, 0] == 2), np.sum(fc[:, 1] == 2), np.sum(fc[:, 2] == 64)]
    for k in range(3):
        p = h[k] / bound
        assert abs(got[k] - m * p) < 4.5 * math.sqrt(m * p * (1 - p)) + 1, (k, got[k], m * p)
    t1 = r["t_last"][::32]  # one clock per group
    assert abs(t1.mean() * bound - 1.0) < 4.5 / math.sqrt(groups)


@pytest.mark.parametrize("net_i", [0, 3])
def test_state_following_bound_general_networks(orc, net_i):
    """Networks other than Frank's under the state-following bound, against the master equation."""
    reac, prod, rates, init = GENERAL_NETWORKS[net_i]
    N = sum(init)
    st, index, Q = me.generator(reac, prod, rates, N)
    snaps = [0.05, 0.2, 0.6]
    runs = 15_000
    r = orc.run(orc.Network(reac, prod, rates), init, run_ids=np.arange(runs) * 32 + 11, seed=97 + net_i,
                t_end=0.6, snap_times=snaps, pad_pow2=2)
    p0 = np.zeros(len(st))
    p0[index[init]] = 1.0
    for s, t in enumerate(snaps):
        p = me.distribution(Q, p0, t)
        obs = np.zeros(len(st))
        for c in r["snap_counts"][s]:
            obs[index[tuple(int(x) for x in c)]] += 1
        exp = p * runs
        big = exp >= 5
        o = np.append(obs[big], obs[~big].sum())
        e = np.append(exp[big], exp[~big].sum())
        if e[-1] < 5:
            o, e = o[:-1], e[:-1]
            e *= o.sum() / e.sum()
        assert stats.power_divergence(o, e, lambda_="log-likelihood")[1] > 1e-4, (t, net_i)


def test_state_following_bound_isomerisation(orc):
    """A <-> B (rates 1 and 0.4) under the state-following bound: the binomial closed form."""
    a, b = 1.0, 0.4
    nA0, nB0 = 14, 6
    net = orc.Network([[1, 0], [0, 1]], [[0, 1], [1, 0]], [a, b])
    snaps = [0.3, 1.2]
    runs = 20_000
    r = orc.run(net, (nA0, nB0), run_ids=np.arange(runs) * 32 + 30, seed=62, t_end=1.2, snap_times=snaps,
                pad_pow2=2)
    for s, t in enumerate(snaps):
        e = math.exp(-(a + b) * t)
        p_aa, p_ba = (b + a * e) / (a + b), b * (1 - e) / (a + b)
        pmf = np.convolve(stats.binom.pmf(np.arange(nA0 + 1), nA0, p_aa), stats.binom.pmf(np.arange(nB0 + 1), nB0, p_ba))
        obs = np.bincount(r["snap_counts"][s][:, 0], minlength=nA0 + nB0 + 1).astype(float)
        exp = pmf * runs
        big = exp >= 5
        o, ex = np.append(obs[big], obs[~big].sum()), np.append(exp[big], exp[~big].sum())
        assert stats.power_divergence(o, ex, lambda_="log-likelihood")[1] > 1e-4, t


def test_state_following_bound_group_consistency(orc):
    """A run's result does not depend on which runs of its group are asked for, and a partial
    last group holds only its own lanes."""
    a = orc.run(orc.frank(), (40, 40, 80), 70, seed=5, t_end=3.0, pad_pow2=2)
    ids = np.array([69, 3, 64, 31, 0])
    b = orc.run(orc.frank(), (40, 40, 80), run_ids=ids, seed=5, t_end=3.0, pad_pow2=2, ensemble_runs=70)
    for k in ("final_counts", "t_abs", "steps", "reactions"):
        assert np.array_equal(a[k][ids], b[k]), k
    full = orc.run(orc.frank(), (40, 40, 80), 96, seed=5, t_end=3.0, pad_pow2=2)
    assert np.array_equal(full["final_counts"][:64], a["final_counts"][:64])
    assert np.all(a["final_counts"].sum(1) == 160) and np.all(a["redraws"] == 0)
    with pytest.raises(RuntimeError):
        orc.run(orc.frank(), (40, 40, 80), run_ids=[70], seed=5, pad_pow2=2, ensemble_runs=70)


# --------------------------------------------------------------------------
# The per-run clock: every run draws its waiting times from its own stream
# --------------------------------------------------------------------------
def test_lane_clock_waiting_times_are_independent_exponentials(orc):
    """Eq. equation-tau per run: the first waiting time of every run is Exp(Lambda), and the 32
    runs of a group no longer share it (the group clock gives them one value)."""
    N, groups = 64, 4000
    Z = N * (N - 1) // 2
    r = orc.run(orc.frank(), (16, 16, 32), groups * 32, seed=3, step_budget=1, check=False, lane_clock=True)
    tau = r["t_last"] * Z
    assert abs(tau.mean() - 1.0) < 4.5 / math.sqrt(len(tau))
    assert stats.kstest(tau, "expon").pvalue > 1e-4
    by_group = tau.reshape(groups, 32)
    assert np.all(np.ptp(by_group, axis=1) > 0)
    c = np.corrcoef(by_group[:, 0], by_group[:, 1])[0, 1]
    assert abs(c) < 4.5 / math.sqrt(groups), c
    g = orc.run(orc.frank(), (16, 16, 32), 64, seed=3, step_budget=1, check=False)
    assert np.all(g["t_last"].reshape(2, 32) == g["t_last"].reshape(2, 32)[:, :1])


@pytest.mark.parametrize("pad", [False, True])
def test_master_equation_lane_clock(orc, pad):
    """Every run of every group (40 000 runs in 1250 groups, all lanes) against the master
    equation at N = 12: with its own clock each run is an exact sample path and the runs of a
    group are independent samples."""
    N, init = 12, (3, 3, 6)
    st, index, Q = _frank_me(N)
    snaps = [0.02, 0.05, 0.1, 0.2, 0.4]
    runs = 40_000
    r = orc.run(orc.frank(), init, runs, seed=27, t_end=0.5, snap_times=snaps, pad_pow2=pad, lane_clock=True)
    p0 = np.zeros(len(st))
    p0[index[init]] = 1.0
    for s, t in enumerate(snaps):
        p = me.distribution(Q, p0, t)
        obs = np.zeros(len(st))
        for c in r["snap_counts"][s]:
            obs[index[tuple(int(x) for x in c)]] += 1
        exp = p * runs
        big = exp >= 5
        o = np.append(obs[big], obs[~big].sum())
        e = np.append(exp[big], exp[~big].sum())
        if e[-1] < 5:
            o, e = o[:-1], e[:-1]
            e *= o.sum() / e.sum()
        stat, pval = stats.power_divergence(o, e, lambda_="log-likelihood")
        assert pval > 1e-4, (t, pval)


def test_lane_clock_closed_form(orc):
    """L+D->2A alone from L = D = m0: T = sum_{m=1}^{m0} Exp(m^2) for every run, over all 32
    runs of each group; the jump chain is the group clock's, step for step."""
    net = orc.Network([[1, 1, 0]], [[0, 0, 2]], [1.0])
    m0, A0, groups = 8, 4, 2000
    mean = sum(1 / m**2 for m in range(1, m0 + 1))
    var = sum(1 / m**4 for m in range(1, m0 + 1))
    lane = orc.run(net, (m0, m0, A0), groups * 32, seed=45, t_end=np.inf, lane_clock=True)
    n = len(lane["t_abs"])
    assert abs(lane["t_abs"].mean() - mean) < 4.5 * math.sqrt(var / n)
    assert abs(lane["t_abs"].var() - var) < 0.05 * var
    grp = orc.run(net, (m0, m0, A0), groups * 32, seed=45, t_end=np.inf)
    assert np.array_equal(lane["steps"], grp["steps"])  # the jump chain does not depend on the clock
    assert np.array_equal(lane["final_counts"], grp["final_counts"])


def test_lane_clock_removes_the_correlation_within_a_group(orc):
    """N = 2 from (1, 1, 0): Z = 1 and the one reaction fires at the first step, so a run's
    absorption time is its first waiting time, Exp(1).  Under the group clock the 32 runs of a
    group share it (correlation 1); under the per-run clock they are independent Exp(1)."""
    groups = 3000
    grp = orc.run(orc.frank(), (1, 1, 0), groups * 32, seed=46, t_end=np.inf)
    tg = grp["t_abs"].reshape(groups, 32)
    assert np.all(tg == tg[:, :1])
    lane = orc.run(orc.frank(), (1, 1, 0), groups * 32, seed=46, t_end=np.inf, lane_clock=True)
    tl = lane["t_abs"].reshape(groups, 32)
    assert stats.kstest(lane["t_abs"], "expon").pvalue > 1e-4
    for a, b in ((0, 1), (5, 31)):
        c = np.corrcoef(tl[:, a], tl[:, b])[0, 1]
        assert abs(c) < 4.5 / math.sqrt(groups), (a, b, c)


def test_lane_clock_stream_layout(orc):
    """The per-run waiting-time words are elements 0 and 1 of Philox4x32-10 with counter
    (j lo 32, s lo 32, s hi 16 | (j >> 32) << 16 | 1 << 24, 0): one step of run j, checked
    against the Philox block function called directly."""
    seed, N = 0x1234_5678_9ABC, 64
    Z = N * (N - 1) // 2
    for j in (0, 31, 32 * 1000 + 7):
        r = orc.run(orc.frank(), (16, 16, 32), run_ids=[j], seed=seed, step_budget=1, check=False, lane_clock=True)
        w = orc.philox4x32_10([j & 0xFFFFFFFF, 0, ((j >> 32) & 0xFF) << 16 | 1 << 24, 0],
                              [seed & 0xFFFFFFFF, seed >> 32])
        u = ((w[1] << 21 | w[0] >> 11) + 1) * 2.0**-53
        assert r["t_last"][0] == pytest.approx(-math.log(u) / Z, rel=1e-15)
