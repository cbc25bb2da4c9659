"""Exact-chain pin of the oracle on a 4x4 periodic lattice.

The chain is built here from heights alone (a site is a local minimum when its
four neighbours are one higher; it moves by +-2), independently of the oracle's
bond-bit code. One sweep is the product of the two half-sweep kernels, each of
which flips every active minimum with probability P/2^k and every active
maximum with probability Q/2^k, independently. Its stationary law is compared,
by a chi-square test, with the state frequencies of long oracle runs.

At p = q the half-sweep kernels are symmetric (a flipped minimum is a maximum
that flips back with the same probability), so the stationary law is uniform
on the class reachable from the striped start: a closed form.
"""
import itertools

import numpy as np
import pytest
from scipy import stats

L = 4


def _code(h):
    """Bond code of a height array, the layout the oracle records:
    X bit i = [h(x+1,y) - h(x,y) = +1], Y bit i = [h(x,y+1) - h(x,y) = +1], i = y*L + x."""
    sx = np.roll(h, -1, axis=1) - h
    sy = np.roll(h, -1, axis=0) - h
    code = 0
    for i in range(L * L):
        y, x = divmod(i, L)
        code |= int(sx[y, x] == 1) << i
        code |= int(sy[y, x] == 1) << (L * L + i)
    return code


def _normal(h):
    return h - h[0, 0]


def _extrema(h):
    nb = [np.roll(h, 1, 1), np.roll(h, -1, 1), np.roll(h, 1, 0), np.roll(h, -1, 0)]
    is_min = np.all([n == h + 1 for n in nb], axis=0)
    is_max = np.all([n == h - 1 for n in nb], axis=0)
    return is_min, is_max


def _reachable():
    start = np.array([[(x + y) % 2 for x in range(L)] for y in range(L)], np.int64)
    seen = {_code(start): _normal(start)}
    todo = [start]
    while todo:
        h = todo.pop()
        is_min, is_max = _extrema(h)
        for y, x in zip(*np.nonzero(is_min | is_max)):
            g = h.copy()
            g[y, x] += 2 if is_min[y, x] else -2
            c = _code(g)
            if c not in seen:
                seen[c] = _normal(g)
                todo.append(g)
    codes = sorted(seen)
    return codes, [seen[c] for c in codes]


def _halfsweep_kernel(codes, hs, s, pe, qe):
    index = {c: i for i, c in enumerate(codes)}
    n = len(codes)
    K = np.zeros((n, n))
    yy, xx = np.mgrid[0:L, 0:L]
    active = (xx + yy) % 2 == s
    for i, h in enumerate(hs):
        is_min, is_max = _extrema(h)
        sites = [(y, x, 2, pe) for y, x in zip(*np.nonzero(is_min & active))]
        sites += [(y, x, -2, qe) for y, x in zip(*np.nonzero(is_max & active))]
        for flips in itertools.product((0, 1), repeat=len(sites)):
            g = h.copy()
            pr = 1.0
            for f, (y, x, d, pf) in zip(flips, sites):
                if f:
                    g[y, x] += d
                    pr *= pf
                else:
                    pr *= 1.0 - pf
            if pr > 0:
                K[i, index[_code(g)]] += pr
    return K


def _stationary(K):
    w, v = np.linalg.eig(K.T)
    pi = np.real(v[:, np.argmin(np.abs(w - 1.0))])
    pi = pi / pi.sum()
    assert np.all(pi > -1e-12)
    return np.clip(pi, 0, None)


@pytest.fixture(scope="module")
def chain_states():
    return _reachable()


def _chi2_pvalue(counts, expected_prob):
    n = counts.sum()
    exp = expected_prob * n
    big = exp >= 5
    obs_b = list(counts[big]) + [counts[~big].sum()]
    exp_b = list(exp[big]) + [exp[~big].sum()]
    if exp_b[-1] < 5:  # fold a tiny remainder into the smallest bin
        o, e = obs_b.pop(), exp_b.pop()
        obs_b[-1] += o
        exp_b[-1] += e
    exp_b = np.array(exp_b) * (n / np.sum(exp_b))
    return stats.chisquare(obs_b, exp_b).pvalue


@pytest.mark.parametrize("p,q,s_sel,seed", [
    (0.5, 0.5, 0.5, 31),     # p = q: uniform law (closed form), k = 2
    (0.75, 0.25, 0.5, 32),   # p != q, k = 3
    (0.95, 0.05, 0.5, 33),   # non-dyadic, k = 32 (rounded thresholds)
    (1.0, 0.0, 0.5, 34),     # the configs' growth rule
])
def test_stationary_law_4x4(orc, chain_states, p, q, s_sel, seed):
    codes, hs = chain_states
    k, P, Q = orc.thresholds(p, q, s_sel)
    pe, qe = P / 2.0 ** k, Q / 2.0 ** k
    K = _halfsweep_kernel(codes, hs, 0, pe, qe) @ _halfsweep_kernel(codes, hs, 1, pe, qe)
    assert np.allclose(K.sum(axis=1), 1.0)
    pi = _stationary(K)
    if p == q:
        assert np.allclose(K.sum(axis=0), 1.0)           # doubly stochastic
        assert np.allclose(pi, 1.0 / len(codes), atol=1e-9)  # uniform law
    sim = orc.Sim(L, p, q, seed, s_sel=s_sel)
    sim.sweep(100)  # burn-in
    recs = sim.sweep_record(n=4_000_000, thin=40)
    index = {c: i for i, c in enumerate(codes)}
    counts = np.zeros(len(codes))
    for c, n in zip(*np.unique(recs, return_counts=True)):
        assert int(c) in index, "oracle left the reachable class"
        counts[index[int(c)]] += n
    assert _chi2_pvalue(counts, pi) > 0.01
