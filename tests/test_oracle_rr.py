"""Pins of the oracle's RR-set generation (Algorithm 3) and estimator (Eq. 1).

* exact influence sigma(S) by enumerating every live-edge world of the directed IC instance,
  against n * E[coverage fraction] of the oracle's RR sets (Eq. 1);
* Lemma 3: the distribution of the RR set of a fixed root equals the one of independent
  per-neighbour coins (exact enumeration);
* special cases p = 0 (R = {root}) and p = 1 (R = the root's connected component);
* the stratified estimator sum_s |V_s|/n_s Lambda_s is unbiased;
* RR set (s, j) is a pure function of its key (incremental growth == one-shot).
"""
import math

import numpy as np
import pytest

from tests import bruteforce as bf

P32 = 1 << 32
# 5 vertices, w(0,1) = 2 (two layers in A(0) and A(1)), 10 directed pairs
SMALL = [[0, 1, 2], [2, 3], [3, 4], [0, 1]]
SUBSETS = [[0], [2], [4], [1, 3], [0, 4], [2, 3, 4]]


def graph(oracle, hes, n, model, uthr=0):
    off, mem = bf.to_csr(hes)
    return oracle.Graph(n, off, mem, model, uthr)


def pool_sets(pool):
    a = pool.arrays()
    return [a.mem[a.off[i]:a.off[i + 1]].tolist() for i in range(len(a.off) - 1)], a


@pytest.mark.parametrize("model,uthr", [("uniform_pair", 858993459), ("wc", 0),
                                        ("paper_layer", 0)])
def test_eq1_exact_spread(oracle, model, uthr):
    n = 5
    W = bf.weights(n, SMALL)
    pairs = bf.directed_pairs(W, model, uthr)
    g = graph(oracle, SMALL, n, model, uthr)
    theta = 200000
    pool = oracle.Pool(g, seed=11, tag=0, roots="plain", strategy="binomial_only")
    pool.grow_theta(theta)
    sets, _ = pool_sets(pool)
    member = np.zeros((theta, n), dtype=bool)
    for i, R in enumerate(sets):
        member[i, R] = True
    for S in SUBSETS:
        f = member[:, S].any(axis=1).mean()
        est = n * f
        exact = bf.exact_spread(n, pairs, S)
        se = n * math.sqrt(max(f * (1 - f), 1e-12) / theta)
        assert abs(est - exact) < 4.5 * se + 1e-9, (model, S, est, exact, se)
        # the oracle's own estimator agrees with the count
        lam = pool.coverage(S)
        assert abs(pool.estimate(lam) - est) < 1e-9


def test_lemma3_rr_distribution(oracle):
    n = 5
    uthr = 1288490188  # p = 0.3
    W = bf.weights(n, SMALL)
    pairs = bf.directed_pairs(W, "uniform_pair", uthr)
    g = graph(oracle, SMALL, n, "uniform_pair", uthr)
    theta = 150000
    pool = oracle.Pool(g, seed=5, tag=0, roots="plain", strategy="binomial_only")
    pool.grow_theta(theta)
    sets, a = pool_sets(pool)
    roots = np.array([g.root(5, 0, "plain", 0, int(j)) for j in a.j])
    for r in range(n):
        idx = np.nonzero(roots == r)[0]
        emp = {}
        for i in idx:
            key = frozenset(sets[i])
            emp[key] = emp.get(key, 0) + 1
        exact = bf.rr_distribution(n, pairs, r)
        assert set(emp) <= set(exact)
        N = len(idx)
        chi2, dof = 0.0, 0
        for R, p in exact.items():
            e = N * p
            if e < 5:
                continue
            chi2 += (emp.get(R, 0) - e) ** 2 / e
            dof += 1
        # generous: p < 1e-6 for chi-square with dof degrees of freedom
        assert chi2 < dof + 10 * math.sqrt(2 * dof) + 20, (r, chi2, dof)


def test_p0_rr_is_root(oracle):
    rng = np.random.default_rng(0)
    hes = [[int(x) for x in rng.integers(0, 50, size=4)] for _ in range(40)]
    g = graph(oracle, hes, 50, "uniform_pair", 0)
    pool = oracle.Pool(g, seed=3, tag=2, roots="plain")
    pool.grow_theta(20000)
    sets, a = pool_sets(pool)
    assert all(len(R) == 1 for R in sets)
    roots = np.array([R[0] for R in sets])
    for j in range(0, 20000, 997):
        assert roots[j] == g.root(3, 2, "plain", 0, j)
    hist = np.bincount(roots, minlength=50)
    exp = 20000 / 50
    assert ((hist - exp) ** 2 / exp).sum() < 49 + 10 * math.sqrt(98)


def test_p1_rr_is_component(oracle):
    rng = np.random.default_rng(1)
    n = 60
    hes = [[int(x) for x in rng.integers(0, n, size=int(rng.integers(1, 4)))] for _ in range(30)]
    comp = bf.components(n, hes)
    g = graph(oracle, hes, n, "uniform_pair", P32)
    pool = oracle.Pool(g, seed=9, tag=0, roots="plain")
    pool.grow_theta(3000)
    sets, a = pool_sets(pool)
    for i, R in enumerate(sets):
        root = g.root(9, 0, "plain", 0, int(a.j[i]))
        assert set(R) == set(comp[root])


def test_rr_pure_function_of_key(oracle):
    rng = np.random.default_rng(2)
    n = 200
    hes = [[int(x) for x in rng.integers(0, n, size=int(rng.integers(2, 9)))] for _ in range(150)]
    g = graph(oracle, hes, n, "wc")
    p1 = oracle.Pool(g, seed=4, tag=1, roots="stratified")
    p1.grow_theta(100)
    p1.grow_theta(350)
    p2 = oracle.Pool(g, seed=4, tag=1, roots="stratified")
    p2.grow_theta(350)
    a1, a2 = p1.arrays(), p2.arrays()
    assert np.array_equal(a1.off, a2.off) and np.array_equal(a1.mem, a2.mem)
    assert np.array_equal(a1.stratum, a2.stratum) and np.array_equal(a1.j, a2.j)
    # each set is sorted and contains its root
    for i in range(len(a1.off) - 1):
        R = a1.mem[a1.off[i]:a1.off[i + 1]]
        assert np.all(np.diff(R) > 0)
        assert g.root(4, 1, "stratified", int(a1.stratum[i]), int(a1.j[i])) in R
    # a different tag gives a different pool
    p3 = oracle.Pool(g, seed=4, tag=2, roots="stratified")
    p3.grow_theta(350)
    assert not np.array_equal(p3.arrays().mem[:200], a1.mem[:200])


def test_stratified_allocation(oracle):
    rng = np.random.default_rng(4)
    n = 300
    hes = [[int(x) for x in rng.integers(0, n, size=int(rng.integers(2, 7)))] for _ in range(200)]
    g = graph(oracle, hes, n, "wc")
    sizes = [g.stratum_size(s) for s in range(16)]
    for theta in (1, 17, 1000, 12345):
        ns = g.allocate("stratified", theta)
        for s in range(16):
            want = 0 if sizes[s] == 0 else -(-theta * sizes[s] // n)
            assert int(ns[s]) == want
        assert int(ns.sum()) >= theta
        assert int(g.allocate("plain", theta)[0]) == theta


def test_stratified_estimator_unbiased(oracle):
    n = 5
    uthr = 858993459  # p = 0.2
    W = bf.weights(n, SMALL + [[4]])
    hes = SMALL + [[4]]
    pairs = bf.directed_pairs(W, "uniform_pair", uthr)
    g = graph(oracle, hes, n, "uniform_pair", uthr)
    S = [2]
    exact = bf.exact_spread(n, pairs, S)
    est = []
    for seed in range(300):
        pool = oracle.Pool(g, seed=1000 + seed, tag=0, roots="stratified",
                           strategy="binomial_only")
        pool.grow_theta(400)
        est.append(pool.estimate(pool.coverage(S)))
    est = np.array(est)
    se = est.std(ddof=1) / math.sqrt(len(est))
    assert abs(est.mean() - exact) < 4.5 * se


def test_poisson_strategy_close_to_binomial(oracle):
    # a 41-clique hyperedge with small p: layers of 40 members use the Poisson strategy; with
    # p small the RR-size law is close to the Binomial one (Sec. 3.1.3)
    hes = [list(range(41))]
    g = graph(oracle, hes, 41, "uniform_pair", 21474836)  # p = 0.005
    means = {}
    for strat in ("paper", "binomial_only"):
        pool = oracle.Pool(g, seed=21, tag=0, roots="plain", strategy=strat)
        pool.grow_theta(100000)
        a = pool.arrays()
        means[strat] = np.diff(a.off).mean()
    assert abs(means["paper"] - means["binomial_only"]) < 0.01
