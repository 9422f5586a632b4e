"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle, bit for bit.

Integer results (layer profiles, RR sets, coverage counts, seed sets, work counters) must be
identical; double results (estimates, bounds, theta) agree to 1e-12 relative and integer theta
is identical. Inputs are seeded and steer every kernel path: warp materialisation, block
materialisation on chip, id-bucketed materialisation through global scratch, direct indexing of a
single hyperedge, > 32 layers with draws, > 256 picks, split Poisson draws, p = 1, RR sets larger
than the on-chip sort buffer, degenerate hyperedges.
"""
import numpy as np
import pytest

from tests import gpu_cases as gc

pytestmark = pytest.mark.gpu
P32 = 1 << 32
REL = 1e-12


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_01911_gb300 import build
    build.build()
    import paper_2406_01911_gb300 as H
    return H


def load_both(H, oracle, n, hes, model, uthr=0, seed=1):
    off, mem = gc.csr(hes)
    g = H.Graph(n, off, mem, model, uthr, seed=seed)
    og = oracle.Graph(n, off, mem, model, uthr)
    return g, og


def check_profile(g, og, n):
    prof = g.profile()
    for v in range(n):
        assert prof["deg"][v] == og.deg(v)
        assert prof["nlayers"][v] == og.nlayers(v)
        assert prof["stratum"][v] == og.stratum(v)
        b = prof["prof_off"][v]
        lay = og.layers(v)
        got = list(zip(prof["layer_w"][b:b + len(lay)].tolist(), prof["layer_n"][b:b + len(lay)].tolist(),
                       prof["layer_thr"][b:b + len(lay)].tolist()))
        assert got == lay, v
    st = g.stats()
    assert st["stratum_size"] == [og.stratum_size(s) for s in range(16)]
    assert abs(st["theta_lstar"] - og.theta_lstar()) <= REL * max(1.0, og.theta_lstar())


def check_pool(H, oracle, g, og, theta, roots, strategy="paper", tag=0, seed=1, grow=None):
    p = g.pool(tag=tag, roots=roots, strategy=strategy)
    op = oracle.Pool(og, seed=seed, tag=tag, roots=roots, strategy=strategy)
    for t in (grow or []) + [theta]:
        p.sample(t)
        op.grow_theta(t)
    gc.assert_same_pool(p, op)
    gc.assert_same_counters(p, op)
    return p, op


@pytest.mark.parametrize("model,uthr", [("uniform_pair", 214748364), ("wc", 0), ("paper_layer", 0),
                                        ("uniform_pair", P32)])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_graphs(H, oracle, model, uthr, seed):
    n, hes = gc.random_graph(seed, 300, 260, 9)
    g, og = load_both(H, oracle, n, hes, model, uthr, seed=7)
    check_profile(g, og, n)
    for roots in ("plain", "stratified"):
        for strategy in ("paper", "binomial_only"):
            check_pool(H, oracle, g, og, 700, roots, strategy, seed=7, grow=[50])


def test_degenerate(H, oracle):
    n, hes = gc.degenerate_graph()
    g, og = load_both(H, oracle, n, hes, "uniform_pair", 1 << 31, seed=3)
    check_profile(g, og, n)
    assert g.stats()["nnz"] == og.nnz()
    check_pool(H, oracle, g, og, 500, "plain", seed=3)
    check_pool(H, oracle, g, og, 500, "stratified", seed=3)


def test_single_vertex_and_no_hyperedges(H, oracle):
    for n, hes in ((1, []), (1, [[0]]), (7, [])):
        g, og = load_both(H, oracle, n, hes, "wc", 0, seed=2)
        check_profile(g, og, n)
        check_pool(H, oracle, g, og, 64, "plain", seed=2)
        check_pool(H, oracle, g, og, 64, "stratified", seed=2)


@pytest.mark.parametrize("uthr", [429496729, 1 << 31, P32])
def test_many_layers(H, oracle, uthr):
    n, hes = gc.layered_graph(40)
    g, og = load_both(H, oracle, n, hes, "uniform_pair", uthr, seed=5)
    check_profile(g, og, n)
    assert og.nlayers(0) == 40
    check_pool(H, oracle, g, og, 2000, "plain", seed=5)
    for model in ("wc", "paper_layer"):
        g2, og2 = load_both(H, oracle, n, hes, model, 0, seed=5)
        check_pool(H, oracle, g2, og2, 2000, "stratified", seed=5)


@pytest.mark.parametrize("uthr", [858993459, 42949672, P32])
def test_big_single_hyperedge(H, oracle, uthr):
    # p = 0.2 on a 1999-member layer draws ~400 picks (more than a warp keeps on chip); the
    # Poisson draw is split into parts (lambda > 64)
    n, hes = gc.big_edge_graph()
    g, og = load_both(H, oracle, n, hes, "uniform_pair", uthr, seed=9)
    check_profile(g, og, n)
    check_pool(H, oracle, g, og, 40, "plain", seed=9)


def test_hub_paths(H, oracle):
    n, hes = gc.hub_graph()
    g, og = load_both(H, oracle, n, hes, "uniform_pair", 85899345, seed=11)  # p = 0.02
    check_profile(g, og, n)
    assert og.dh(0) >= 60 and og.dh(1) >= 10
    check_pool(H, oracle, g, og, 12, "plain", seed=11)
    g2, og2 = load_both(H, oracle, n, hes, "wc", 0, seed=11)
    check_pool(H, oracle, g2, og2, 3000, "stratified", seed=11)


def test_greedy_and_spread(H, oracle):
    n, hes = gc.random_graph(4, 2000, 1500, 8)
    g, og = load_both(H, oracle, n, hes, "uniform_pair", 429496729, seed=13)
    for roots in ("plain", "stratified"):
        p, op = check_pool(H, oracle, g, og, 5000, roots, seed=13)
        for k in (1, 7, 40):
            seeds, res = g.select_seeds(p, None, k, mode="fixed")
            oseeds, olam, _ = op.greedy(k)
            assert seeds.tolist() == oseeds.tolist()
            assert res["lambda_r1"].tolist() == olam.tolist()
            est = op.estimate(olam)
            assert abs(res["sigma_r1"] - est) <= REL * max(1.0, est)
        q, oq = check_pool(H, oracle, g, og, 3000, roots, tag=2, seed=13)
        sig, err = g.spread(seeds, q)
        lam = oq.coverage(seeds)
        est = oq.estimate(lam)
        assert abs(sig - est) <= REL * max(1.0, est)
        assert err > 0


def test_theta_plan(H, oracle):
    n, hes = gc.random_graph(5, 5000, 100, 4)
    g, og = load_both(H, oracle, n, hes, "wc")
    for k, eps, ell in ((1, 0.5, 1.0), (50, 0.1, 1.0), (100, 0.05, 2.0), (4999, 0.2, 1.0)):
        a = g.plan_theta(k, eps, ell)
        b = oracle.plan_theta(n, k, eps, ell)
        for key in ("theta_max_ceil", "theta0", "i_max"):
            assert a[key] == b[key]
        for key in ("delta", "ln_binom", "theta_max"):
            assert abs(a[key] - b[key]) <= REL * abs(b[key])


@pytest.mark.parametrize("roots", ["stratified", "plain"])
def test_brr(H, oracle, roots):
    n, hes = gc.random_graph(6, 3000, 2500, 6)
    g, og = load_both(H, oracle, n, hes, "wc", 0, seed=17)
    k, eps = 20, 0.2
    r1, r2 = g.pool(tag=0, roots=roots), g.pool(tag=1, roots=roots)
    seeds, res = g.select_seeds(r1, r2, k, mode="brr", eps=eps, ell=1.0)
    oseeds, ores = oracle.brr(og, 17, k, eps, 1.0, 0, roots)
    assert seeds.tolist() == oseeds.tolist()
    for key in ("rounds", "theta", "pool_r1", "pool_r2"):
        assert res[key] == ores[key], key
    assert res["lambda_r1"].tolist() == ores["lambda_r1"].tolist()
    assert res["lambda_r2"].tolist() == ores["lambda_r2"].tolist()
    for key in ("sigma_r1", "sigma_r2", "upper", "lower", "alpha"):
        assert abs(res[key] - ores[key]) <= REL * max(1.0, abs(ores[key])), key
    assert len(res["alpha_round"]) == len(ores["alpha_round"])


def test_errors(H):
    off, mem = gc.csr([[0, 5]])
    with pytest.raises(H.HyperIMError) as e:
        H.Graph(3, off, mem)
    assert e.value.status == -1
    off, mem = gc.csr([[0, 1], [1, 2]])
    g = H.Graph(3, off, mem)
    with pytest.raises(H.HyperIMError):
        g.plan_theta(4, 0.1)
    with pytest.raises(H.HyperIMError):
        g.plan_theta(1, 1.5)
    p = g.pool(tag=0).sample(10)
    with pytest.raises(H.HyperIMError):
        g.select_seeds(p, None, 4)
    with pytest.raises(H.HyperIMError):
        g.select_seeds(p, p, 1, mode="brr")
    with pytest.raises(H.HyperIMError):
        g.spread([5], p)
    with pytest.raises(H.HyperIMError):
        H.hyperim_sample_rr(g.handle, 300, 5)
    # a device pointer input gives the same graph as a host input
    import torch
    g2 = H.Graph(3, torch.as_tensor(off).cuda(), torch.as_tensor(mem).cuda())
    assert g2.stats()["nnz"] == g.stats()["nnz"] == 4
    # a budget that cannot hold the graph
    with pytest.raises(H.HyperIMError) as e:
        H.Graph(3, off, mem, hbm_budget_bytes=64)
    assert e.value.status == -2
