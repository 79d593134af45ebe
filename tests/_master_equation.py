"""Brute-force chemical master equation for small conserved networks.

Independent of the oracle: it enumerates the states with sum n = N, builds the
dense generator Q[s, s'] = k_r h_r(s) for s -> s + nu_r, and gives
* P(t) = p0 expm(Q t)                       (forward Kolmogorov equation),
* absorption probabilities from the linear system on the transient states,
* mean absorption time from the fundamental matrix.
Used only as a pin for the oracle in the CPU test suite.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg


def states(n_species: int, N: int):
    out = []
    for combo in itertools.product(range(N + 1), repeat=n_species - 1):
        if sum(combo) <= N:
            out.append(tuple(combo) + (N - sum(combo),))
    return out


def propensity(reactants_row, n):
    h = 1
    for m, x in zip(reactants_row, n):
        if m == 1:
            h *= x
        elif m == 2:
            h *= x * (x - 1) // 2
    return h


def generator(reactants, products, rates, N):
    reactants = np.asarray(reactants)
    products = np.asarray(products)
    S = reactants.shape[1]
    st = states(S, N)
    index = {s: i for i, s in enumerate(st)}
    Q = np.zeros((len(st), len(st)))
    for i, s in enumerate(st):
        for r in range(len(rates)):
            a = rates[r] * propensity(reactants[r], s)
            if a == 0:
                continue
            t = tuple(int(x) for x in np.asarray(s) + products[r] - reactants[r])
            Q[i, index[t]] += a
            Q[i, i] -= a
    return st, index, Q


def distribution(Q, p0, t):
    return p0 @ scipy.linalg.expm(Q * t)


def absorption(Q):
    """Absorbing states are those with no outgoing rate.  Returns
    (absorbing indices, B[transient, absorbing] probabilities, mean times[transient],
    transient indices)."""
    absorbing = [i for i in range(Q.shape[0]) if Q[i, i] == 0]
    transient = [i for i in range(Q.shape[0]) if Q[i, i] != 0]
    Qtt = Q[np.ix_(transient, transient)]
    Qta = Q[np.ix_(transient, absorbing)]
    B = np.linalg.solve(-Qtt, Qta)
    T = np.linalg.solve(-Qtt, np.ones(len(transient)))
    return absorbing, B, T, transient
