"""Pins of the lattice oracle (Frank's model on a periodic lattice with hops; oracle.h,
orc_lattice): the master equation of the whole lattice on 2 x 1 and 2 x 2 lattices, the
diffusion of one molecule between two sites in closed form, the fast-diffusion limit against
the well-mixed oracle at rates k / M, and conservation."""
import math

import numpy as np
import pytest
from scipy import stats

from tests import _master_equation as me


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def lattice_network(lx, ly, k, d):
    """The lattice as one network of 3M species (L_i, D_i, A_i): Frank's reactions at every site
    and a first-order reaction X_i -> X_j at rate d for every direction from i to a neighbour j
    other than i (two directions to the same site give two reactions)."""
    M = lx * ly
    reac, prod, rates = [], [], []

    def row():
        return [0] * (3 * M)
    for i in range(M):
        L, D, A = 3 * i, 3 * i + 1, 3 * i + 2
        for (a, b), (c, e), kr in (((A, L), (L, L), k[0]), ((A, D), (D, D), k[1]), ((L, D), (A, A), k[2])):
            r, p = row(), row()
            r[a] += 1
            r[b] += 1
            p[c] += 1
            p[e] += 1
            reac.append(r)
            prod.append(p)
            rates.append(kr)
        x, y = i % lx, i // lx
        for nx, ny in (((x + 1) % lx, y), ((x - 1) % lx, y), (x, (y + 1) % ly), (x, (y - 1) % ly)):
            j = nx + lx * ny
            if j == i:
                continue
            for c in range(3):
                r, p = row(), row()
                r[3 * i + c] = 1
                p[3 * j + c] = 1
                reac.append(r)
                prod.append(p)
                rates.append(d)
    return reac, prod, rates


def _g_test(states, index, p, samples):
    obs = np.zeros(len(states))
    for c in samples:
        obs[index[tuple(int(v) for v in c)]] += 1
    exp = p * len(samples)
    big = exp >= 5
    o = np.append(obs[big], obs[~big].sum())
    e = np.append(exp[big], exp[~big].sum())
    if e[-1] < 5:
        o, e = o[:-1], e[:-1]
        e *= o.sum() / e.sum()
    return stats.power_divergence(o, e, lambda_="log-likelihood").pvalue


@pytest.mark.parametrize("lx,ly,init,k,d", [
    (2, 1, [(2, 1, 1), (0, 1, 1)], (1.0, 1.0, 1.0), 0.5),         # rho_r = 2: reaction slots doubled
    (2, 1, [(3, 1, 0), (0, 1, 1)], (1.0, 1.0, 1.0), 3.0),         # rho_h = 3: hop slots tripled
    (2, 2, [(1, 1, 0), (0, 0, 1), (0, 0, 0), (0, 0, 0)], (1.0, 0.5, 1.0), 1.0),  # thinning
    (2, 1, [(4, 3, 2), (1, 0, 0)], (1.0, 1.0, 1.0), 0.5),         # cap 10: 16 molecule slots, 45 pairs
    (2, 1, [(3, 2, 0), (2, 2, 0)], (1.0, 1.0, 1.0), 2.0),         # caps 5, 6, 7, 8, 10 as sites fill up
])
def test_lattice_master_equation(orc, lx, ly, init, k, d):
    """The distribution of the whole lattice's state (every site's counts) at t_end against
    P(t) = p0 expm(Q t) of the lattice's master equation; one run per group (independent
    streams), 20 000 runs per time.  The cases cover slot multiplicities, thinning, a cap that is
    not a power of two, and a cap that grows through several values."""
    init = np.array(init, dtype=np.int64)
    N = int(init.sum())
    reac, prod, rates = lattice_network(lx, ly, k, d)
    st, index, Q = me.generator(reac, prod, rates, N)
    p0 = np.zeros(len(st))
    p0[index[tuple(int(v) for v in init.ravel())]] = 1.0
    runs = 20_000
    for t_end, seed in ((0.1, 3), (0.5, 4)):
        r = orc.lattice_run(lx, ly, init, runs, rates=k, hop=d, seed=seed, t_end=t_end, lanes=1)
        assert np.all(r["final_counts"].sum(axis=(1, 2)) == N)
        pval = _g_test(st, index, me.distribution(Q, p0, t_end), r["final_counts"].reshape(runs, -1))
        assert pval > 1e-4, (t_end, pval)


def test_lattice_diffusion_closed_form(orc):
    """One L molecule on a 2 x 1 lattice, no reaction possible: it changes site at rate 2 d (two of
    its four directions lead to the other site), so P(on its first site at t) = (1 + exp(-4 d t)) / 2."""
    d, t, runs = 0.5, 0.4, 20_000
    init = np.array([(1, 0, 0), (0, 0, 0)], dtype=np.int64)
    r = orc.lattice_run(2, 1, init, runs, hop=d, seed=5, t_end=t, lanes=1)
    p = np.mean(r["final_counts"][:, 0, 0] == 1)
    want = (1 + math.exp(-4 * d * t)) / 2
    assert abs(p - want) < 4.5 * math.sqrt(want * (1 - want) / runs), (p, want)
    assert np.all(r["reactions"] == 0)


def test_lattice_fast_diffusion_is_well_mixed_at_rate_k_over_m(orc):
    """With hops much faster than reactions every molecule's site is uniform and independent, so the
    lattice's reaction rate is k sum_i A_i L_i ~ k A L / M: the well-mixed model at rates k / M.  Time
    to homochirality and the outcome of 2048 runs (hops 32 times the reaction rate constant; runs
    in groups of 32, standard errors over group means) against 4000 well-mixed runs; t_end = 12 is
    past every well-mixed absorption time of this system (the largest is about 7)."""
    M, runs = 4, 2048
    init_sites = np.zeros((M, 3), dtype=np.int64)
    init_sites[0] = (4, 4, 8)
    lat = orc.lattice_run(2, 2, init_sites, runs, rates=(1.0, 1.0, 1.0), hop=32.0, seed=6, t_end=12.0)
    wm = orc.run(orc.frank(0.25, 0.25, 0.25), (4, 4, 8), run_ids=np.arange(4000) * 32, seed=7, t_end=np.inf)
    assert np.all(lat["outcome"] >= 0)
    ga = lat["t_homochiral"].reshape(-1, 32).mean(1)
    b = wm["t_abs"]
    se = math.sqrt(ga.var(ddof=1) / len(ga) + b.var() / len(b))
    assert abs(ga.mean() - b.mean()) < 4.5 * se + 0.04 * b.mean(), (ga.mean(), b.mean(), se)
    for o in (0, 1, 2):
        pa = (lat["outcome"] == o).reshape(-1, 32).mean(1)
        pb = np.mean(wm["outcome"] == o)
        se_o = math.sqrt(pa.var(ddof=1) / len(pa) + pb * (1 - pb) / len(b))
        assert abs(pa.mean() - pb) < 4.5 * se_o + 0.02, (o, pa.mean(), pb, se_o)


def test_lattice_conservation_cap_and_counters(orc):
    """Totals conserved, counts non-negative, the group's cap at or above every site count, the
    snapshot totals and domain counts consistent, and the group's runs sharing their step count."""
    rng = np.random.default_rng(8)
    lx, ly, runs = 4, 4, 64
    init = rng.poisson((8, 8, 16), size=(runs, lx * ly, 3)).astype(np.int64)
    snaps = [0.005, 0.01]
    r = orc.lattice_run(lx, ly, init, runs, hop=0.1, seed=9, t_end=0.02, snap_times=snaps)
    fc = r["final_counts"]
    assert np.all(fc >= 0)
    assert np.array_equal(fc.sum(axis=(1, 2)), init.sum(axis=(1, 2)))
    assert np.all(r["cap"] >= fc.sum(axis=2).max(axis=1))
    assert np.all(r["snap_totals"].sum(axis=2) == init.sum(axis=(1, 2))[:, None])
    assert np.all(r["snap_domains"].sum(axis=2) <= lx * ly)
    assert np.all(r["steps"].reshape(2, 32) == r["steps"].reshape(2, 32)[:, :1])
    assert r["hops"].sum() > 0 and r["reactions"].sum() > 0
