"""Pins of the oracle's greedy max coverage (Algorithm 1, Eq. 2) and of the Sec. 4 arithmetic.

Greedy: every round's pick maximises the marginal coverage recomputed from scratch (ties to the
lowest id); coverage >= (1 - 1/e) OPT by exhaustive search; exhausted coverage picks the lowest
unpicked ids. Theta: ln C(n,k) against exact big-integer binomials; theta_0 / i_max invariants.
Bounds: the Sec. 4.2 lower bound is a valid confidence bound (Monte Carlo on binomial counts);
the upper bound of Eq. upper_6 reduces to the coverage itself for k = 1.
"""
import math

import numpy as np
import pytest

from tests import bruteforce as bf


def make_pool(oracle, n, hes, model, uthr, theta, roots, seed=1):
    off, mem = bf.to_csr(hes)
    g = oracle.Graph(n, off, mem, model, uthr)
    pool = oracle.Pool(g, seed=seed, tag=0, roots=roots)
    pool.grow_theta(theta)
    a = pool.arrays()
    sets = [a.mem[a.off[i]:a.off[i + 1]].tolist() for i in range(len(a.off) - 1)]
    return g, pool, sets, a


def weighted_marginal(sets, strata, W, S, v):
    S = set(S)
    return sum(int(W[s]) for R, s in zip(sets, strata) if v in R and not (S & set(R)))


@pytest.mark.parametrize("roots", ["plain", "stratified"])
@pytest.mark.parametrize("seed", range(4))
def test_greedy_marginals_from_scratch(oracle, roots, seed):
    rng = np.random.default_rng(seed)
    n = 40
    hes = [[int(x) for x in rng.integers(0, n, size=int(rng.integers(2, 5)))] for _ in range(30)]
    g, pool, sets, a = make_pool(oracle, n, hes, "uniform_pair", 644245094, 3000, roots, seed)
    ns = pool.counts()
    W = [1] * 16 if roots == "plain" else [
        ((g.stratum_size(s) << 32) // int(ns[s])) if ns[s] else 0 for s in range(16)]
    k = 8
    seeds, lam, gains = pool.greedy(k)
    S = []
    for r in range(k):
        marg = [weighted_marginal(sets, a.stratum, W, S, v) if v not in S else -1 for v in range(n)]
        best = max(marg)
        assert seeds[r] == marg.index(best), r      # argmax, lowest id on ties
        assert int(gains[r]) == best
        S.append(int(seeds[r]))
    assert len(set(S)) == k
    # Lambda per stratum = RR sets of that stratum hit by S
    for s in range(16):
        hit = sum(1 for R, st in zip(sets, a.stratum) if st == s and set(R) & set(S))
        assert int(lam[s]) == hit
    assert list(pool.coverage(S)) == list(lam)


def test_greedy_approximation_ratio(oracle):
    rng = np.random.default_rng(7)
    n = 14
    hes = [[int(x) for x in rng.integers(0, n, size=3)] for _ in range(12)]
    _, pool, sets, _ = make_pool(oracle, n, hes, "uniform_pair", 1288490188, 400, "plain", 3)
    for k in (1, 2, 3):
        seeds, lam, _ = pool.greedy(k)
        opt = bf.best_cover(sets, n, k)
        got = bf.coverage_sets(sets, seeds)
        assert got == int(lam.sum())
        assert got >= (1 - 1 / math.e) * opt
        if k == 1:
            assert got == opt


def test_greedy_exhausted_coverage(oracle):
    # p = 0: every RR set is {root}; once the roots are covered the picks are the lowest ids
    n = 30
    hes = [[i, (i + 1) % n] for i in range(n)]
    _, pool, sets, _ = make_pool(oracle, n, hes, "uniform_pair", 0, 5, "plain")
    roots = sorted({R[0] for R in sets})
    seeds, lam, gains = pool.greedy(12)
    picked = list(seeds)
    assert sorted(picked[:len(roots)]) == roots
    rest = [v for v in range(n) if v not in roots][: 12 - len(roots)]
    assert picked[len(roots):] == rest
    assert all(int(x) == 0 for x in gains[len(roots):])


def test_estimate_formula(oracle):
    rng = np.random.default_rng(9)
    n = 120
    hes = [[int(x) for x in rng.integers(0, n, size=int(rng.integers(2, 6)))] for _ in range(90)]
    g, pool, sets, a = make_pool(oracle, n, hes, "wc", 0, 2000, "stratified")
    S = [3, 17, 55]
    lam = pool.coverage(S)
    ns = pool.counts()
    want = sum(g.stratum_size(s) / int(ns[s]) * int(lam[s]) for s in range(16) if ns[s])
    assert abs(pool.estimate(lam) - want) < 1e-9 * max(1.0, want)
    _, ppool, psets, _ = make_pool(oracle, n, hes, "wc", 0, 2000, "plain")
    plam = ppool.coverage(S)
    assert abs(ppool.estimate(plam) - n * int(plam[0]) / 2000) < 1e-9


# ------------------------------------------------------------------------------------------------
# Sec. 4: theta and the bounds
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n,k", [(1000, 10), (100_000, 50), (2_000_000, 100), (5_000_000, 200),
                                 (64, 63)])
def test_ln_binomial_exact(oracle, n, k):
    plan = oracle.plan_theta(n, k, 0.1, 1.0)
    exact = math.log(math.comb(n, k))
    assert abs(plan["ln_binom"] - exact) <= 1e-12 * exact + 1e-12


@pytest.mark.parametrize("n,k,eps,ell", [(1000, 10, 0.1, 1.0), (100_000, 50, 0.1, 1.0),
                                         (2_000_000, 100, 0.1, 1.0), (5000, 5, 0.3, 2.0)])
def test_theta_invariants(oracle, n, k, eps, ell):
    p = oracle.plan_theta(n, k, eps, ell)
    assert abs(p["delta"] - n ** (-ell)) <= 1e-15 * n ** (-ell)
    t0 = p["theta0"]
    # theta_0 is theta_max eps^2 k / n rounded up, and does not depend on the scale factor n/(eps^2 k)
    assert t0 == math.ceil(p["theta_max"] * eps * eps * k / n)
    assert t0 * 2 ** p["i_max"] >= p["theta_max"] > t0 * 2 ** (p["i_max"] - 1)
    assert p["theta_max_ceil"] == math.ceil(p["theta_max"])
    # monotone: a larger eps needs fewer sets; a larger delta (smaller ell) too
    q = oracle.plan_theta(n, k, eps * 1.5, ell)
    assert q["theta_max"] < p["theta_max"]
    r = oracle.plan_theta(n, k, eps, ell * 0.5)
    assert r["theta_max"] < p["theta_max"]


def test_theta_rejects_bad_arguments(oracle):
    for args in [(10, 0, 0.1, 1.0), (10, 11, 0.1, 1.0), (10, 2, 0.0, 1.0), (10, 2, 1.0, 1.0),
                 (10, 2, 0.1, 0.0)]:
        with pytest.raises(oracle.OracleError):
            oracle.plan_theta(*args)


@pytest.mark.parametrize("delta", [0.05, 0.2])
@pytest.mark.parametrize("f", [0.01, 0.2])
def test_lower_bound_is_a_confidence_bound(oracle, delta, f):
    # Lambda_R2 ~ Binomial(N, f): the lower bound of sigma = n f may exceed it w.p. <= delta
    rng = np.random.default_rng(17)
    n, N, trials = 10000, 2000, 4000
    lam2 = rng.binomial(N, f, size=trials)
    sigma = n * f
    lows = np.array([oracle.lower_bound(float(x), delta, n, N) for x in lam2])
    miss = (lows > sigma).mean()
    assert miss <= delta + 3 * math.sqrt(delta * (1 - delta) / trials)
    # and it is below the point estimate
    assert np.all(lows <= n * lam2 / N + 1e-9)


def test_upper_bound(oracle):
    # k = 1: 1 - (1 - 1/k)^k = 1, the bound is the estimate itself
    assert abs(oracle.upper_bound(37.0, 1, 1000, 500) - 37.0 * 1000 / 500) < 1e-12
    for k in (2, 10, 100):
        u = oracle.upper_bound(37.0, k, 1000, 500)
        ratio = 1 - (1 - 1 / k) ** k
        assert u >= 37.0 * 1000 / 500
        assert abs(u * ratio - 37.0 * 1000 / 500) < 1e-9
        assert ratio > 1 - 1 / math.e  # Eq. upper_6's right-hand bound


def test_brr_schedule(oracle):
    rng = np.random.default_rng(5)
    n = 400
    hes = [[int(x) for x in rng.integers(0, n, size=int(rng.integers(2, 6)))] for _ in range(300)]
    off, mem = bf.to_csr(hes)
    g = oracle.Graph(n, off, mem, "wc")
    k, eps = 5, 0.3
    seeds, res = oracle.brr(g, 1, k, eps, 1.0, 0, "stratified")
    plan = oracle.plan_theta(n, k, eps, 1.0)
    target = 1 - math.exp(-1) - eps
    assert len(set(seeds.tolist())) == k
    assert res["theta"] == plan["theta0"] << (res["rounds"] - 1)
    assert res["alpha"] >= target or res["rounds"] == plan["i_max"] + 1
    assert all(a < target for a in res["alpha_round"][:-1])
    assert res["pool_r1"] == res["pool_r2"] == int(g.allocate("stratified", res["theta"]).sum())
    assert abs(res["alpha"] - res["lower"] / res["upper"]) < 1e-12


@pytest.mark.parametrize("roots", ["plain", "stratified"])
@pytest.mark.parametrize("seed", range(3))
def test_prefix_upper_bound_from_scratch(oracle, roots, seed):
    # Eq. upper_2 with p_max = 1, recomputed from the weighted marginals of every greedy prefix
    rng = np.random.default_rng(100 + seed)
    n = 40
    hes = [[int(x) for x in rng.integers(0, n, size=int(rng.integers(2, 5)))] for _ in range(30)]
    g, pool, sets, a = make_pool(oracle, n, hes, "uniform_pair", 644245094, 2000, roots, seed)
    ns = pool.counts()
    W = [1] * 16 if roots == "plain" else [
        ((g.stratum_size(s) << 32) // int(ns[s])) if ns[s] else 0 for s in range(16)]
    k = 6
    seeds, lam, gains, U = pool.greedy_upper(k)
    best = None
    for i in range(k + 1):
        S = [int(x) for x in seeds[:i]]
        cov = sum(int(W[s]) for R, s in zip(sets, a.stratum) if set(R) & set(S))
        marg = sorted((weighted_marginal(sets, a.stratum, W, S, v) for v in range(n) if v not in S),
                      reverse=True)
        u = cov + sum(marg[:k])
        best = u if best is None else min(best, u)
    assert U == best
    # never looser than the closed form of Lemma 5 (Eq. upper_6 with p_max = 1)
    ck = sum(int(x) for x in gains)
    assert U <= ck / (1 - (1 - 1 / k) ** k) + 1


def test_prefix_upper_bounds_the_optimum(oracle):
    # Lemma 4: the coverage of every k-set is at most the bound (exhaustive search, tiny pools)
    rng = np.random.default_rng(11)
    n = 12
    for trial in range(4):
        hes = [[int(x) for x in rng.integers(0, n, size=3)] for _ in range(10)]
        _, pool, sets, _ = make_pool(oracle, n, hes, "uniform_pair", 1288490188, 300, "plain", trial)
        for k in (1, 2, 3):
            _, lam, _, U = pool.greedy_upper(k)
            opt = bf.best_cover(sets, n, k)
            assert opt <= U, (trial, k, opt, U)
            assert int(lam.sum()) <= U


def test_prefix_upper_in_sigma_units(oracle):
    assert oracle.prefix_upper_sigma(3 << 32, "stratified", 100, 7) == 3.0
    assert oracle.prefix_upper_sigma(21, "plain", 100, 7) == 300.0
    assert oracle.prefix_upper_sigma((1 << 64) + (1 << 32), "stratified", 1, 1) == float(2 ** 32 + 1)


@pytest.mark.parametrize("roots", ["plain", "stratified"])
def test_brr_with_prefix_upper(oracle, roots):
    # the same schedule with Eq. upper_2: every round's bound is at most the closed form's, so the
    # prefix variant stops no later; its last round's bound is the greedy's prefix minimum
    rng = np.random.default_rng(5)
    n = 400
    hes = [[int(x) for x in rng.integers(0, n, size=int(rng.integers(2, 6)))] for _ in range(300)]
    off, mem = bf.to_csr(hes)
    g = oracle.Graph(n, off, mem, "wc")
    k, eps = 5, 0.3
    _, closed = oracle.brr(g, 1, k, eps, 1.0, 0, roots)
    seeds, pref = oracle.brr(g, 1, k, eps, 1.0, 0, roots, upper="prefix")
    assert pref["rounds"] <= closed["rounds"]
    for a_p, a_c in zip(pref["alpha_round"], closed["alpha_round"]):
        # same R1 seeds and R2 lower bound in both: alpha_p / alpha_c = upper_c / upper_p >= 1
        assert a_c == 0.0 or a_p / a_c >= 1 - 1e-12
    # recompute the last round's bound from a pool grown the same way
    p1 = oracle.Pool(g, seed=1, tag=0, roots=roots)
    p1.grow_theta(pref["theta"])
    s2, _, _, U = p1.greedy_upper(k)
    assert s2.tolist() == seeds.tolist()
    assert pref["upper"] == oracle.prefix_upper_sigma(U, roots, n, pref["pool_r1"])


# ------------------------------------------------------------------------------------------------
# Eq. equation-max at high precision and the benchmark workloads' anchors; Eq. upper_6 for k > 1
# ------------------------------------------------------------------------------------------------
def theta_max_mp(n, k, eps, ell):
    """Eq. equation-max, 2n (sqrt(ln(2/delta)) + sqrt(ln C(n,k) + ln(6/delta))) / (eps^2 k) with
    delta = n^-ell, at 50 significant digits; ln C(n,k) from the log-gamma function."""
    mp = pytest.importorskip("mpmath")
    with mp.workdps(50):
        n_, k_, e_, l_ = mp.mpf(n), mp.mpf(k), mp.mpf(eps), mp.mpf(ell)
        delta = n_ ** (-l_)
        lnc = mp.loggamma(n_ + 1) - mp.loggamma(k_ + 1) - mp.loggamma(n_ - k_ + 1)
        t = 2 * n_ * (mp.sqrt(mp.log(2 / delta)) + mp.sqrt(lnc + mp.log(6 / delta))) / (e_ ** 2 * k_)
        return float(t)


@pytest.mark.parametrize("n,k,eps,ell", [(100_000, 50, 0.1, 1.0), (2_000_000, 100, 0.1, 1.0),
                                         (1000, 10, 0.05, 1.0), (5000, 3, 0.3, 2.0),
                                         (160_217, 100, 0.1, 1.0), (4_000_000, 200, 0.2, 1.5)])
def test_theta_max_matches_high_precision(oracle, n, k, eps, ell):
    p = oracle.plan_theta(n, k, eps, ell)
    ref = theta_max_mp(n, k, eps, ell)
    assert abs(p["theta_max"] - ref) <= 1e-12 * ref
    assert p["theta_max_ceil"] == math.ceil(ref)


@pytest.mark.parametrize("n,k,floor_theta_max,theta0,i_max", [
    (100_000, 50, 9_792_352, 49, 18),        # the 100k-vertex workload (p = 0.01, k = 50)
    (2_000_000, 100, 148_467_123, 75, 21),   # the 2M-vertex workload (weighted cascade, k = 100)
])
def test_theta_anchors_of_the_benchmark_workloads(oracle, n, k, floor_theta_max, theta0, i_max):
    # eps = 0.1, ell = 1 (delta = 1/n, as in Sec. 6): theta_max's integer part, theta_0 and the
    # number of doublings; a dropped factor 2, eps in place of eps^2 or ln(2/delta) in place of
    # ln(6/delta) each moves theta_max by far more than one unit
    p = oracle.plan_theta(n, k, 0.1, 1.0)
    assert math.floor(p["theta_max"]) == floor_theta_max
    assert p["theta0"] == theta0 and p["i_max"] == i_max


def test_upper6_closed_values(oracle):
    # (1 - 1/k)^k is 1/4 at k = 2 and 8/27 at k = 3: the bound is 4/3 and 27/19 of the estimate
    # Lambda n / theta; as k grows (1 - 1/k)^k -> 1/e and the bound -> e/(e - 1) of the estimate
    est = 57.0 * 1000 / 500
    assert oracle.upper_bound(57.0, 2, 1000, 500) == pytest.approx(est * 4 / 3, rel=1e-15)
    assert oracle.upper_bound(57.0, 3, 1000, 500) == pytest.approx(est * 27 / 19, rel=1e-15)
    assert oracle.upper_bound(57.0, 10 ** 6, 1000, 500) == pytest.approx(est * math.e / (math.e - 1), rel=1e-6)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("k", [2, 3])
def test_upper6_bounds_the_optimum(oracle, seed, k):
    # greedy covers at least 1 - (1 - 1/k)^k of the best k-set (Lemma 5 / Eq. upper_6), so the
    # closed form applied to the greedy's coverage is never below the optimum found by search
    rng = np.random.default_rng(100 + seed)
    n = 14
    hes = [[int(x) for x in rng.integers(0, n, size=int(rng.integers(2, 5)))] for _ in range(10)]
    g, pool, sets, a = make_pool(oracle, n, hes, "uniform_pair", 1288490188, 60, "plain", seed)
    seeds, lam, _ = pool.greedy(k)
    opt = bf.best_cover(sets, n, k)
    N = len(sets)
    assert oracle.upper_bound(float(lam[0]), k, N, N) >= opt - 1e-9
    assert int(lam[0]) <= opt
