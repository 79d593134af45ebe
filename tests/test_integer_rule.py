"""The general kernels' form of the selection rule (Sec. 4, steps b-c; Eq. equation-changer),
checked exhaustively on small words on the CPU.

The oracle walks the cumulative propensities S_r = h_0 + ... + h_r and fires reaction r where
S_{r-1} <= n < S_r. The general kernels instead take h_0, h_1, ... off n in turn, one K-plane
two's-complement subtraction each, and fire reaction r in the lanes where the r-th subtraction
borrows out of the top plane. While S_R < 2^K the running value n - S_r stays above -2^K, so a lane
borrows at most once, at the reaction whose interval holds n, and a lane with n >= S_R (a ghost or
null event) never borrows. These tests run the plane-wise borrow chain (difference xor3(m, h, b),
borrow maj(~m, h, b)) on 32-lane words and compare it with the interval rule."""
import itertools

import numpy as np

MASK = 0xFFFFFFFF


def _planes(values, K):
    """Bit planes of up to 32 lane values: plane i holds bit i of lane l at bit l."""
    out = []
    for i in range(K):
        w = 0
        for lane, v in enumerate(values):
            w |= ((int(v) >> i) & 1) << lane
        out.append(w)
    return out


def _sub_borrow(m, h):
    """m -= h plane by plane (modulo 2^K); the lanes that borrow out of the top plane."""
    borrow = 0
    for i in range(len(m)):
        mi = m[i]
        m[i] = mi ^ h[i] ^ borrow
        nm = ~mi & MASK
        borrow = (nm & h[i]) | (nm & borrow) | (h[i] & borrow)
    return borrow


def _lanes(word, n):
    return [(word >> lane) & 1 for lane in range(n)]


def _check(K, hs, ns):
    """hs: [lanes][R] propensities, ns: [lanes] draws (at most 32 lanes)."""
    R = len(hs[0])
    m = _planes(ns, K)
    xi = [_sub_borrow(m, _planes([h[r] for h in hs], K)) for r in range(R)]
    for lane, (h, n) in enumerate(zip(hs, ns)):
        S = np.cumsum(h)
        want = [int((S[r] - h[r]) <= n < S[r]) for r in range(R)]
        got = [(xi[r] >> lane) & 1 for r in range(R)]
        assert got == want, (K, h, n, got, want)
    # what is left of n in every lane is n - S_R modulo 2^K
    left = [sum(((m[i] >> lane) & 1) << i for i in range(K)) for lane in range(len(ns))]
    assert left == [(int(n) - int(sum(h))) % (1 << K) for h, n in zip(hs, ns)]


def test_borrow_chain_equals_interval_rule_exhaustive_k4():
    """K = 4, three reactions: every propensity triple with S_R < 16 and every n < 16."""
    K = 4
    cases = [(h, n) for h in itertools.product(range(16), repeat=3) if sum(h) < 16 for n in range(16)]
    for start in range(0, len(cases), 32):
        chunk = cases[start:start + 32]
        _check(K, [c[0] for c in chunk], [c[1] for c in chunk])


def test_borrow_chain_with_zero_propensities_and_ghosts():
    """Zero h_r never fire; n at or above S_R (ghost or null events) fires nothing; n = S_R - 1
    fires the last reaction with a nonzero propensity."""
    K = 5
    hs = [(0, 3, 0, 4), (5, 0, 0, 0), (0, 0, 0, 31), (0, 0, 0, 0), (7, 7, 7, 7), (1, 1, 1, 1)] * 5
    ns = [6, 5, 30, 0, 28, 3] * 5
    ns = [n if k < 6 else (n + k) % 32 for k, n in enumerate(ns)]
    _check(K, hs, ns)


def test_borrow_chain_random_wide_words():
    """K = 19 and K = 31 (the widest propensity a word holds), eight reactions, random
    propensities scaled so that S_R < 2^K, random n below 2^K."""
    rng = np.random.default_rng(2412)
    for K in (19, 31):
        for _ in range(20):
            w = rng.random((32, 8))
            w[rng.random((32, 8)) < 0.2] = 0.0
            tot = rng.integers(1, 1 << K, size=32)
            hs = np.floor(w / np.maximum(w.sum(1, keepdims=True), 1e-300) * tot[:, None]).astype(np.int64)
            assert np.all(hs.sum(1) < (1 << K))
            ns = rng.integers(0, 1 << K, size=32)
            _check(K, hs.tolist(), ns.tolist())
