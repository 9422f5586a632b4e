"""Pins of the oracle's forward Monte-Carlo influence (the Sec. 2.2 cascade under the IC model).

* the mean activated count against the exact sigma(S) of Eq. 1 (enumeration of every live-edge
  world of the directed IC instance, independent of the oracle), three activation settings;
* special cases: p = 0 activates only the seeds, p = 1 the union of their components;
* every simulation against a plain Python cascade over the brute-force weight matrix and
  thresholds, drawing the same keyed coins (Philox is pinned by its known-answer vectors):
  a wrong layer lookup, threshold or traversal in the oracle changes some count.
"""
import math

import numpy as np
import pytest

from tests import bruteforce as bf

P32 = 1 << 32
SMALL = [[0, 1, 2], [2, 3], [3, 4], [0, 1]]


def graph(oracle, hes, n, model, uthr=0):
    off, mem = bf.to_csr(hes)
    return oracle.Graph(n, off, mem, model, uthr)


@pytest.mark.parametrize("model,uthr", [("uniform_pair", 858993459), ("wc", 0), ("paper_layer", 0)])
def test_forward_mean_is_exact_spread(oracle, model, uthr):
    n = 5
    pairs = bf.directed_pairs(bf.weights(n, SMALL), model, uthr)
    g = graph(oracle, SMALL, n, model, uthr)
    sims = 200000
    for S in ([0], [2], [4], [1, 3], [0, 4]):
        c = g.forward_spread(S, sims, seed=5).astype(np.float64)
        exact = bf.exact_spread(n, pairs, S)
        se = c.std() / math.sqrt(sims)
        assert abs(c.mean() - exact) < 4.5 * se + 1e-9, (model, S, c.mean(), exact, se)


def test_forward_special_cases(oracle):
    rng = np.random.default_rng(2)
    n = 40
    hes = [[int(x) for x in rng.choice(n, size=int(rng.integers(2, 5)), replace=False)] for _ in range(18)]
    comp = bf.components(n, hes)
    S = [0, 7, 7, 21]
    g0 = graph(oracle, hes, n, "uniform_pair", 0)
    assert g0.forward_spread(S, 50, seed=1).tolist() == [3] * 50
    g1 = graph(oracle, hes, n, "uniform_pair", P32)
    reach = set().union(*(comp[s] for s in S))
    assert g1.forward_spread(S, 20, seed=1).tolist() == [len(reach)] * 20
    with pytest.raises(Exception):
        g1.forward_spread([n], 1, seed=1)


def python_cascade(oracle, n, hes, model, uthr, S, r, seed):
    """One simulation written from the definition: u active -> each neighbour v once, live with
    the threshold of u's layer in A(v), coin = word 0 of Philox(r, u, v, 0xFFFFFFFE)."""
    W = bf.weights(n, hes)
    thr = {}
    for v in range(n):
        L, ws = bf.layers(W, v)
        for members, t in zip(L, bf.thresholds(W, v, model, uthr)):
            for u in members:
                thr[(u, v)] = t
    key = (seed & 0xFFFFFFFF, seed >> 32)
    active = []
    for s in S:
        if s not in active:
            active.append(s)
    head = 0
    while head < len(active):
        u = active[head]
        head += 1
        for v in range(n):
            if W[u, v] == 0:
                continue
            t = thr[(u, v)]
            live = t >= P32 or (t > 0 and oracle.philox4x32_10((r, u, v, 0xFFFFFFFE), key)[0] < t)
            if live and v not in active:
                active.append(v)
    return len(active)


@pytest.mark.parametrize("model,uthr", [("uniform_pair", 1288490188), ("wc", 0), ("paper_layer", 0)])
def test_forward_per_simulation(oracle, model, uthr):
    rng = np.random.default_rng(9)
    n = 24
    hes = [[int(x) for x in rng.choice(n, size=int(rng.integers(2, 6)), replace=False)] for _ in range(20)]
    hes += [[0, 1, 2, 3], [0, 1, 2], [0, 1]]  # several layers around 0 and 1
    g = graph(oracle, hes, n, model, uthr)
    S = [0, 5, 5, 17]
    seed = 0x1234_5678_9ABC
    got = g.forward_spread(S, 60, seed=seed)
    want = [python_cascade(oracle, n, hes, model, uthr, S, r, seed) for r in range(60)]
    assert got.tolist() == want
