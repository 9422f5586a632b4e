"""Pins of the oracle's LT sampler (the LT cascade of Sec. 2.2 in its live-edge form: a popped
vertex keeps at most one in-neighbour; integer layer masses n_i floor(p_i 2^32), normalised by
multiply-shift when they sum above 2^32).

* the exact probability that mu keeps nu, counted over all 2^32 words from the brute-force
  layers, gives by enumeration of every keep-one world the exact sigma(S) of Eq. 1; the
  oracle's LT RR sets estimate it within their standard error (three activation settings, one of
  them with masses above 2^32);
* p = 0: the RR set is its root; every LT RR set is a path: its pops keep at most one vertex
  each and the set stops at the first repeat or empty keep.
"""
import itertools
import math

import numpy as np
import pytest

from tests import bruteforce as bf

P32 = 1 << 32
SMALL = [[0, 1, 2], [2, 3], [3, 4], [0, 1]]


def keep_distribution(W, mu, model, uthr):
    """{nu: exact probability that mu keeps nu} (the rest: keeps none)."""
    L, _ = bf.layers(W, mu)
    T = bf.thresholds(W, mu, model, uthr)
    M = sum(len(m) * t for m, t in zip(L, T))
    out = {}
    if M == 0:
        return out
    C = 0
    for members, t in zip(L, T):
        for nu in members:
            lo, hi = C, C + t
            if M <= P32:
                cnt = t
            else:  # y = floor(x M / 2^32) in [lo, hi)  <=>  x in [ceil(lo 2^32 / M), ceil(hi 2^32 / M))
                cnt = (-(-hi * P32 // M)) - (-(-lo * P32 // M))
            out[nu] = cnt / P32
            C = hi
    return out


def exact_lt_spread(n, W, model, uthr, S):
    dists = [keep_distribution(W, mu, model, uthr) for mu in range(n)]
    choices = []
    for d in dists:
        opts = [(nu, p) for nu, p in d.items()]
        rest = 1.0 - sum(p for _, p in opts)
        if rest > 1e-15:
            opts.append((None, rest))
        choices.append(opts)
    S = set(S)
    total = 0.0
    for world in itertools.product(*choices):
        pr = 1.0
        for _, p in world:
            pr *= p
        keep = [nu for nu, _ in world]
        for root in range(n):
            seen = {root}
            x = root
            while True:
                y = keep[x]
                if y is None or y in seen:
                    break
                seen.add(y)
                x = y
            if seen & S:
                total += pr
    return total


@pytest.mark.parametrize("model,uthr", [("uniform_pair", 858993459), ("wc", 0), ("paper_layer", 0)])
def test_lt_exact_spread(oracle, model, uthr):
    n = 5
    W = bf.weights(n, SMALL)
    off, mem = bf.to_csr(SMALL)
    g = oracle.Graph(n, off, mem, model, uthr)
    theta = 200000
    pool = oracle.Pool(g, seed=13, tag=0, roots="plain", strategy="lt")
    pool.grow_theta(theta)
    a = pool.arrays()
    member = np.zeros((theta, n), dtype=bool)
    for i in range(theta):
        member[i, a.mem[a.off[i]:a.off[i + 1]]] = True
    for S in ([0], [2], [4], [1, 3], [0, 4]):
        f = member[:, S].any(axis=1).mean()
        exact = exact_lt_spread(n, W, model, uthr, S)
        se = n * math.sqrt(max(f * (1 - f), 1e-12) / theta)
        assert abs(n * f - exact) < 4.5 * se + 1e-9, (model, S, n * f, exact, se)


def test_lt_special_cases(oracle):
    rng = np.random.default_rng(4)
    n = 60
    hes = [[int(x) for x in rng.choice(n, size=int(rng.integers(2, 6)), replace=False)] for _ in range(40)]
    off, mem = bf.to_csr(hes)
    g0 = oracle.Graph(n, off, mem, "uniform_pair", 0)
    p0 = oracle.Pool(g0, seed=1, tag=0, roots="plain", strategy="lt")
    p0.grow_theta(300)
    a = p0.arrays()
    assert (np.diff(a.off) == 1).all()
    for model, uthr in (("uniform_pair", 1 << 31), ("wc", 0), ("uniform_pair", P32)):
        g = oracle.Graph(n, off, mem, model, uthr)
        W = bf.weights(n, hes)
        for j in range(200):
            st = oracle.Stats()
            R = g.rr_set(7, 0, "plain", 0, j, strategy="lt", stats=st)
            s = st.as_dict()
            assert s["pops"] == len(R)
            # a path: every pop keeps at most one vertex, all but possibly the last keep is new
            assert s["selected"] in (len(R) - 1, len(R))
            # consecutive keeps are neighbours: R is connected in the weight graph
            Rs = set(R)
            comp, stack = {R[0]}, [R[0]]
            while stack:
                x = stack.pop()
                for y in Rs:
                    if y not in comp and W[x, y] > 0:
                        comp.add(y)
                        stack.append(y)
            assert comp == Rs
