"""The query server (continuous batching of HyperIM_BRR queries on resident graphs).

* Alone and in the mix: every query served by four workers at once, sharing one R1/R2 pool pair
  per graph with the other queries on that graph, returns exactly what it returns run alone on
  fresh pools (seeds, rounds, theta, the RR sets each round read, Lambda per stratum, estimates
  and bounds), and the smallest graph's queries equal the oracle's HyperIM_BRR.
* Admission: a budget below what the graphs and pools need releases idle pools (evictions) and
  still gives the same results; p50/p99 latency and the counters are reported.
* Shares: a second handle on a graph (own stream) grows and reads the same pools.
"""
import numpy as np
import pytest

from workloads import batch_workload, make_hypergraph

pytestmark = pytest.mark.gpu
REL = 1e-12
SEED = 1


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_01911_gb300 import build
    build.build()
    import paper_2406_01911_gb300 as H
    return H


def _graphs(count=4):
    specs = batch_workload()
    order = sorted(range(len(specs)), key=lambda i: specs[i].n)
    return [(specs[i], *make_hypergraph(specs[i])) for i in order[:count]]


QUERIES = [(0, 10, 0.1), (1, 50, 0.2), (2, 20, 0.1), (0, 50, 0.2), (3, 10, 0.05), (1, 10, 0.1),
           (2, 100, 0.2), (3, 40, 0.1), (0, 100, 0.1), (1, 30, 0.05), (2, 10, 0.2), (3, 70, 0.2)]


def _alone(H, spec, off, mem, k, eps):
    g = H.Graph(spec.n, off, mem, "wc", 0, seed=SEED)
    r1, r2 = g.pool(tag=0, roots="stratified"), g.pool(tag=1, roots="stratified")
    seeds, res = g.select_seeds(r1, r2, k, mode="brr", eps=eps, ell=1.0)
    r1.close()
    r2.close()
    g.close()
    return seeds, res


def _same(a, b):
    (sa, ra), (sb, rb) = a, b
    assert sa.tolist() == sb.tolist()
    for key in ("rounds", "theta", "pool_r1", "pool_r2"):
        assert ra[key] == rb[key], key
    assert ra["lambda_r1"].tolist() == rb["lambda_r1"].tolist()
    assert ra["lambda_r2"].tolist() == rb["lambda_r2"].tolist()
    for key in ("sigma_r1", "sigma_r2", "upper", "lower", "alpha"):
        assert abs(ra[key] - rb[key]) <= REL * max(1.0, abs(rb[key])), key


def _serve(H, graphs, queries, workers, budget=0):
    loaded = [H.Graph(spec.n, off, mem, "wc", 0, seed=SEED) for spec, off, mem in graphs]
    srv = H.Server(workers=workers, hbm_budget_bytes=budget)
    ids = [srv.add_graph(g) for g in loaded]
    tickets = [srv.submit(ids[gi], k, eps) for gi, k, eps in queries]
    out = [srv.wait(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    for g in loaded:
        g.close()
    return out, stats


def test_alone_and_in_the_mix(H, oracle):
    graphs = _graphs()
    alone = [_alone(H, *graphs[gi], k, eps) for gi, k, eps in QUERIES]
    mixed, stats = _serve(H, graphs, QUERIES, workers=4)
    for (gi, k, eps), a, (seeds, res) in zip(QUERIES, alone, mixed):
        assert res["status"] == 0, (gi, k, eps, res.get("message"))
        _same((seeds, res), a)
        assert res["latency_seconds"] >= res["run_seconds"] > 0
    assert stats["completed"] == len(QUERIES) and stats["failed"] == 0
    assert stats["max_running"] >= 2
    assert 0 < stats["p50_latency_seconds"] <= stats["p99_latency_seconds"] <= stats["max_latency_seconds"]
    # the smallest graph's queries against the oracle
    spec, off, mem = graphs[0]
    og = oracle.Graph(spec.n, off, mem, "wc", 0)
    for (gi, k, eps), (seeds, res) in zip(QUERIES, mixed):
        if gi != 0:
            continue
        oseeds, ores = oracle.brr(og, SEED, k, eps, 1.0, 0, "stratified")
        assert seeds.tolist() == oseeds.tolist()
        for key in ("rounds", "theta", "pool_r1", "pool_r2"):
            assert res[key] == ores[key], key
        assert res["lambda_r2"].tolist() == ores["lambda_r2"].tolist()


def test_served_graphs_alone_and_in_the_mix(H):
    # the served configuration's two smallest resident graphs (~10^5 vertices, Zipf(2.0) sizes in
    # [2, 500]) and the stream's first queries on them (k in [10, 200], eps in {0.05, 0.1, 0.2}),
    # four workers sharing one pool pair per graph: each result equals the query run alone
    from workloads import serving_queries, serving_workload
    specs = serving_workload()
    order = sorted(range(len(specs)), key=lambda i: specs[i].n)[:2]
    graphs = [(specs[i], *make_hypergraph(specs[i])) for i in order]
    picked = [q for q in serving_queries() if q.graph in order][:8]
    assert len(picked) == 8
    queries = [(order.index(q.graph), q.k, q.eps) for q in picked]
    alone = [_alone(H, *graphs[gi], k, eps) for gi, k, eps in queries]
    mixed, stats = _serve(H, graphs, queries, workers=4)
    for (gi, k, eps), a, (seeds, res) in zip(queries, alone, mixed):
        assert res["status"] == 0, (gi, k, eps, res.get("message"))
        _same((seeds, res), a)
    assert stats["completed"] == len(queries) and stats["failed"] == 0


def test_budget_admission(H):
    graphs = _graphs()
    queries = QUERIES[:8]
    free, _ = _serve(H, graphs, queries, workers=2)
    tight, stats = _serve(H, graphs, queries, workers=2, budget=1)
    for a, b in zip(free, tight):
        assert b[1]["status"] == 0
        _same(b, a)
    assert stats["evictions"] > 0 and stats["completed"] == len(queries)


def test_server_rejects_bad_queries(H):
    spec, off, mem = _graphs(1)[0]
    g = H.Graph(spec.n, off, mem, "wc", 0, seed=SEED)
    srv = H.Server(workers=1)
    gid = srv.add_graph(g)
    for args in [(gid + 1, 10, 0.1), (gid, 0, 0.1), (gid, spec.n + 1, 0.1), (gid, 10, 1.5)]:
        with pytest.raises(H.HyperIMError):
            srv.submit(*args)
    with pytest.raises(H.HyperIMError):
        srv.wait(12345)
    srv.close()
    g.close()


def test_share_grows_the_same_pools(H, oracle):
    spec, off, mem = _graphs(2)[1]
    g = H.Graph(spec.n, off, mem, "wc", 0, seed=SEED)
    h = g.share()
    p = g.pool(tag=0, roots="stratified").sample(300)
    q = H.Pool(h, tag=0, roots="stratified")  # created through the share, grown through both
    q.sample(150)
    H.hyperim_sample_rr(g.handle, 0, 300, "stratified", "paper", q.handle)
    op = oracle.Pool(oracle.Graph(spec.n, off, mem, "wc", 0), seed=SEED, tag=0, roots="stratified")
    op.grow_theta(300)
    from tests import gpu_cases as gc
    gc.assert_same_pool(p, op)
    gc.assert_same_pool(q, op)
    assert np.array_equal(p.view()["n_s"], q.view()["n_s"])
    seeds_g, _ = g.select_seeds(p, None, 10, mode="fixed")
    seeds_h, _ = h.select_seeds(q, None, 10, mode="fixed")
    assert seeds_g.tolist() == seeds_h.tolist()
    p.close()
    q.close()
    g.close()  # the data stays until the share is freed
    r = H.Pool(h, tag=1, roots="stratified").sample(100)
    seeds_h2, _ = h.select_seeds(r, None, 5, mode="fixed")
    assert len(seeds_h2) == 5
    r.close()
    h.close()


def test_pool_outlives_its_graph_handle(H, oracle):
    # a pool keeps the loaded graph's data alive: freed graph handle first, pool still readable
    spec, off, mem = _graphs(1)[0]
    g = H.Graph(spec.n, off, mem, "wc", 0, seed=SEED)
    p = g.pool(tag=0, roots="stratified").sample(200)
    g.close()
    op = oracle.Pool(oracle.Graph(spec.n, off, mem, "wc", 0), seed=SEED, tag=0, roots="stratified")
    op.grow_theta(200)
    from tests import gpu_cases as gc
    gc.assert_same_pool(p, op)
    p.close()
