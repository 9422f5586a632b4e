"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle, bit for bit.

Integer results (layer profiles, RR sets, coverage counts, seed sets, work counters) must be
identical; double results (estimates, bounds, theta) agree to 1e-12 relative and integer theta
is identical. Inputs are seeded and steer every kernel path: warp materialisation, block
materialisation on chip, id-bucketed materialisation through global scratch, the chunk index
path, duplicate-free neighbourhoods, direct indexing of a
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


@pytest.mark.parametrize("uthr,roots,theta", [(4294967, "stratified", 2000), (85899345, "plain", 12),
                                              (P32, "plain", 12)])
def test_hub_paths(H, oracle, uthr, roots, theta):
    # p = 0.001: a few picks per hub pop (chunk index path; the hubs head high strata); p = 0.02:
    # hundreds of picks on vertex 0 (block path, bucketed through global scratch); p = 1: every
    # member (block path)
    n, hes = gc.hub_graph()
    g, og = load_both(H, oracle, n, hes, "uniform_pair", uthr, seed=11)
    check_profile(g, og, n)
    assert og.dh(0) >= 60 and og.dh(1) >= 10
    check_pool(H, oracle, g, og, theta, roots, seed=11)


def test_hub_paths_wc(H, oracle):
    n, hes = gc.hub_graph()
    g2, og2 = load_both(H, oracle, n, hes, "wc", 0, seed=11)
    check_pool(H, oracle, g2, og2, 3000, "stratified", seed=11)
    n3, hes3 = gc.layered_hub_graph()
    g3, og3 = load_both(H, oracle, n3, hes3, "wc", 0, seed=3)
    check_pool(H, oracle, g3, og3, 2000, "stratified", seed=3)
    g4, og4 = load_both(H, oracle, n3, hes3, "uniform_pair", 4294967, seed=3)  # p = 0.001
    check_pool(H, oracle, g4, og4, 2000, "stratified", seed=3)


@pytest.mark.parametrize("uthr", [128849018, 858993459, P32])
def test_distinct_neighbourhoods(H, oracle, uthr):
    # p = 0.03 draws ~27 picks from vertex 0's 894 distinct neighbours, p = 0.2 ~180, p = 1 takes
    # every member
    n, hes = gc.distinct_graph()
    g, og = load_both(H, oracle, n, hes, "uniform_pair", uthr, seed=13)
    assert og.nlayers(0) == 1 and og.deg(0) == 894
    check_pool(H, oracle, g, og, 300, "plain", seed=13)
    g2, og2 = load_both(H, oracle, n, hes, "wc", 0, seed=13)
    check_pool(H, oracle, g2, og2, 1500, "stratified", seed=13)


def expected_chunk_index(og, v, id_bits):
    """(bits, table) the chunk index of v must hold, from the oracle's layers (None: no index).
    With T = members of v's hyperedges besides v (repeats counted) and the expected picks per pop
    sum_i n_i p_i compared with 4 on the integers n_i floor(p_i 2^32): candidates have d_H >= 2,
    1 <= l_v <= 1024 and T > 1024 (fewer than 4 expected picks; chunks of at most 512 members)
    or T > 2048 (chunks of at most 1024); bits = the fewest top id bits (at most 12) for which no
    chunk exceeds that; table[i - 1, k] = members of L_i in chunks < k."""
    lay = og.layers(v)
    if og.dh(v) < 2 or not 1 <= len(lay) <= 1024:
        return None
    T = sum(w * n_i for (w, n_i, _) in lay)
    few = sum(n_i * thr for (_, n_i, thr) in lay) < 4 * P32
    if T <= 1024 or (not few and T <= 2048):
        return None
    target = 512 if few else 1024
    mem = [og.layer_members(v, i) for i in range(1, len(lay) + 1)]
    hb = min(12, id_bits)
    best = None
    for c in range(1, hb + 1):
        occ = np.zeros(1 << c, np.int64)
        for (w, _, _), m in zip(lay, mem):
            np.add.at(occ, m.astype(np.int64) >> (id_bits - c), w)
        if occ.max() <= target:
            best = c
            break
    if best is None:
        return None
    C = 1 << best
    tab = np.zeros((len(lay), C), np.uint32)
    for i, m in enumerate(mem):
        per = np.bincount(m.astype(np.int64) >> (id_bits - best), minlength=C)
        tab[i, 1:] = np.cumsum(per)[:-1]
    return best, tab


def neighbourhood_sizes(n, hes):
    """T(v): members of v's hyperedges other than v, repeats across hyperedges counted (after the
    hyperedges are made sets)."""
    T = np.zeros(n, np.int64)
    for he in hes:
        u = np.unique(np.asarray(he, dtype=np.int64))
        T[u] += len(u) - 1
    return T


def check_chunk_index(g, og, n, vertices):
    id_bits = max(1, int(n - 1).bit_length())
    seen = 0
    for v in vertices:
        want = expected_chunk_index(og, int(v), id_bits)
        bits, tab = g.chunk_index(int(v))
        if want is None:
            assert bits == 0 and tab is None, v
        else:
            assert bits == want[0], v
            assert np.array_equal(tab, want[1]), v
            seen += 1
    return seen


@pytest.mark.parametrize("model,uthr", [("wc", 0), ("uniform_pair", 85899345)])
def test_chunk_index(H, oracle, model, uthr):
    # vertex 0: 60 hyperedges of 250 (about 15K members, repeats across hyperedges); vertex 1:
    # 10 of 300; others sit in a few of those hyperedges. Under WC a pop expects about one pick
    # (chunks of 512 from 1,024 members up); at p = 0.02 the hubs expect hundreds (chunks of 1,024,
    # only above 2,048 members). Every vertex above 1,024 members is checked, plus the first 40.
    n, hes = gc.hub_graph()
    g, og = load_both(H, oracle, n, hes, model, uthr, seed=11)
    T = neighbourhood_sizes(n, hes)
    big = np.nonzero(T > 1024)[0]
    seen = check_chunk_index(g, og, n, sorted(set(range(40)) | set(big.tolist())))
    assert seen == g.stats()["index_vertices"] and seen >= 2
    # many layers on a large neighbourhood
    n2, hes2 = gc.layered_hub_graph()
    g2, og2 = load_both(H, oracle, n2, hes2, "wc", 0, seed=3)
    T2 = neighbourhood_sizes(n2, hes2)
    seen2 = check_chunk_index(g2, og2, n2, sorted(set(range(8)) | set(np.nonzero(T2 > 1024)[0].tolist())))
    assert seen2 == g2.stats()["index_vertices"] and seen2 >= 4


@pytest.mark.parametrize("case", ["layered_small", "deep"])
def test_chunk_index_layers(H, oracle, case):
    # layered_small: hubs of about 4,800 members with six layers (sorted whole on chip while the
    # index is built); deep: a hub of about 22,650 members in 150 layers, so its l x 2^c counts
    # exceed what the build keeps on chip (counted in the table itself, bucketed members)
    if case == "layered_small":
        n, hes = gc.layered_hub_graph(groups=6)
    else:
        n, hes = gc.deep_layered_hub_graph()
    g, og = load_both(H, oracle, n, hes, "wc", 0, seed=5)
    T = neighbourhood_sizes(n, hes)
    seen = check_chunk_index(g, og, n, sorted(set(range(8)) | set(np.nonzero(T > 1024)[0].tolist())))
    assert seen == g.stats()["index_vertices"] and seen >= 1
    if case == "deep":
        bits, tab = g.chunk_index(0)
        assert tab.shape[0] >= 150 and tab.size > 8192


@pytest.mark.parametrize("model,uthr", [("uniform_pair", 858993459), ("wc", 0), ("paper_layer", 0),
                                        ("uniform_pair", P32)])
def test_lt_sampler(H, oracle, model, uthr):
    # the LT cascade's live-edge sampler (one kept in-neighbour per pop); paper_layer and p = 1
    # give layer masses above 2^32 (normalised)
    n, hes = gc.random_graph(5, 500, 420, 9)
    g, og = load_both(H, oracle, n, hes, model, uthr, seed=21)
    for roots in ("plain", "stratified"):
        check_pool(H, oracle, g, og, 3000, roots, "lt", seed=21, grow=[100])


def test_lt_sampler_large_neighbourhoods(H, oracle):
    # hubs (chunk index path), many layers, degenerate hyperedges
    n, hes = gc.hub_graph()
    for model, uthr in (("wc", 0), ("uniform_pair", 85899345)):
        g, og = load_both(H, oracle, n, hes, model, uthr, seed=11)
        check_pool(H, oracle, g, og, 3000, "stratified", "lt", seed=11)
    n2, hes2 = gc.layered_hub_graph()
    g2, og2 = load_both(H, oracle, n2, hes2, "paper_layer", 0, seed=3)
    check_pool(H, oracle, g2, og2, 2000, "stratified", "lt", seed=3)
    n3, hes3 = gc.degenerate_graph()
    g3, og3 = load_both(H, oracle, n3, hes3, "uniform_pair", 1 << 31, seed=3)
    check_pool(H, oracle, g3, og3, 400, "plain", "lt", seed=3)


def test_lt_brr(H, oracle):
    n, hes = gc.random_graph(8, 2000, 1700, 6)
    g, og = load_both(H, oracle, n, hes, "wc", 0, seed=17)
    r1 = g.pool(tag=0, roots="stratified", strategy="lt")
    r2 = g.pool(tag=1, roots="stratified", strategy="lt")
    seeds, res = g.select_seeds(r1, r2, 10, mode="brr", eps=0.2, ell=1.0)
    oseeds, ores = oracle.brr(og, 17, 10, 0.2, 1.0, 0, "stratified", "lt")
    assert seeds.tolist() == oseeds.tolist()
    for key in ("rounds", "theta", "pool_r1", "pool_r2"):
        assert res[key] == ores[key], key
    assert res["lambda_r2"].tolist() == ores["lambda_r2"].tolist()


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


@pytest.mark.parametrize("roots", ["plain", "stratified"])
def test_prefix_upper_fixed(H, oracle, roots):
    # Eq. upper_2 on the device (radix select of the k largest marginals each round) equals the
    # oracle's exact integer bound; includes rounds with fewer unpicked vertices than k
    cases = [(gc.random_graph(12, 3000, 2500, 6), "wc", 0, 4000, 25),
             (gc.random_graph(13, 12, 9, 4), "uniform_pair", 1 << 31, 300, 9),
             (gc.hub_graph(), "wc", 0, 3000, 40)]
    for (n, hes), model, uthr, theta, k in cases:
        g, og = load_both(H, oracle, n, hes, model, uthr, seed=29)
        p = g.pool(tag=0, roots=roots).sample(theta)
        op = oracle.Pool(og, seed=29, tag=0, roots=roots)
        op.grow_theta(theta)
        seeds, res = g.select_seeds(p, None, k, mode="fixed", upper="prefix")
        oseeds, olam, _, U = op.greedy_upper(k)
        assert seeds.tolist() == oseeds.tolist()
        assert res["upper"] == oracle.prefix_upper_sigma(U, roots, n, op.count()), (n, k)


@pytest.mark.parametrize("roots", ["plain", "stratified"])
def test_brr_prefix_upper(H, oracle, roots):
    n, hes = gc.random_graph(6, 3000, 2500, 6)
    g, og = load_both(H, oracle, n, hes, "wc", 0, seed=17)
    k, eps = 20, 0.2
    r1, r2 = g.pool(tag=0, roots=roots), g.pool(tag=1, roots=roots)
    seeds, res = g.select_seeds(r1, r2, k, mode="brr", eps=eps, ell=1.0, upper="prefix")
    oseeds, ores = oracle.brr(og, 17, k, eps, 1.0, 0, roots, upper="prefix")
    assert seeds.tolist() == oseeds.tolist()
    for key in ("rounds", "theta", "pool_r1", "pool_r2"):
        assert res[key] == ores[key], key
    for key in ("sigma_r1", "sigma_r2", "upper", "lower", "alpha"):
        assert abs(res[key] - ores[key]) <= REL * max(1.0, abs(ores[key])), key
    _, closed = oracle.brr(og, 17, k, eps, 1.0, 0, roots)
    assert res["rounds"] <= closed["rounds"]


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


@pytest.mark.parametrize("roots", ["plain", "stratified"])
def test_plain_schedule(H, oracle, roots):
    # the comparison form (one launch per batch, one RR set per block) draws the same sets: pools
    # grown over several batches, and a whole BRR query
    n, hes = gc.hub_graph()
    g, og = load_both(H, oracle, n, hes, "uniform_pair", 85899345, seed=7)
    g.set_schedule("plain")
    check_pool(H, oracle, g, og, 2000, roots, seed=7, grow=[300])
    assert H.lib().hyperim_graph_set_schedule(g._h, 7) == -1
    n2, hes2 = gc.random_graph(6, 3000, 2500, 6)
    g2, og2 = load_both(H, oracle, n2, hes2, "wc", 0, seed=17)
    g2.set_schedule("plain")
    r1, r2 = g2.pool(tag=0, roots=roots), g2.pool(tag=1, roots=roots)
    seeds, res = g2.select_seeds(r1, r2, 20, mode="brr", eps=0.2, ell=1.0)
    oseeds, ores = oracle.brr(og2, 17, 20, 0.2, 1.0, 0, roots)
    assert seeds.tolist() == oseeds.tolist()
    for key in ("rounds", "theta", "pool_r1", "pool_r2"):
        assert res[key] == ores[key], key
    assert res["lambda_r2"].tolist() == ores["lambda_r2"].tolist()
