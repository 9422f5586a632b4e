"""GPU parity on the batched and served workload shapes (weighted cascade, stratified roots).

* Batched: 64 hypergraphs of uneven size (n log-uniform in [1e3, 2e5], Zipf(2.1) sizes in
  [2, 300]), each queried with k in {10, 50, 100} at eps = 0.1. The whole HyperIM_BRR query
  (every round's pools, seeds, theta, Lambda per stratum, bounds) of the three smallest graphs,
  and for graphs spread over the size range (the largest included) the theta plan, the first
  round's pools set by set, the pools grown to 4 theta_0 (round 2) and greedy on them for every
  k. The oracle spends 1-100 s on one whole query of the larger graphs, so those stop there.
* Served: the resident graphs of the query stream (n log-uniform in [1e5, 5e6], Zipf(2.0) sizes
  in [2, 500]); the smallest graph with the first queries the stream sends it (k in [10, 200],
  eps in {0.05, 0.1, 0.2}): theta plan, the pools of rounds 0 and 2 and greedy.
"""
import pytest

from tests import gpu_cases as gc
from workloads import batch_workload, make_hypergraph, serving_queries, serving_workload

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


def _load(H, oracle, spec):
    off, mem = make_hypergraph(spec)
    g = H.Graph(spec.n, off, mem, "wc", 0, seed=SEED)
    og = oracle.Graph(spec.n, off, mem, "wc", 0)
    return g, og


def _early_rounds(H, oracle, g, og, n, k, eps):
    plan = g.plan_theta(k, eps, 1.0)
    assert plan == pytest.approx(oracle.plan_theta(n, k, eps, 1.0), rel=REL)
    theta0 = int(plan["theta0"])
    for tag in (0, 1):
        p = g.pool(tag=tag, roots="stratified")
        op = oracle.Pool(og, seed=SEED, tag=tag, roots="stratified")
        for theta in (theta0, 4 * theta0):  # rounds 0 and 2 of the doubling schedule
            p.sample(theta)
            op.grow_theta(theta)
            gc.assert_same_pool(p, op)
        gc.assert_same_counters(p, op)
        if tag == 0:
            seeds, res = g.select_seeds(p, None, k, mode="fixed")
            oseeds, olam, _ = op.greedy(k)
            assert seeds.tolist() == oseeds.tolist()
            assert res["lambda_r1"].tolist() == olam.tolist()
        p.close()


def _by_size(specs):
    return sorted(range(len(specs)), key=lambda i: specs[i].n)


@pytest.mark.parametrize("rank", [0, 1, 2])
def test_batched_whole_query(H, oracle, rank):
    specs = batch_workload()
    spec = specs[_by_size(specs)[rank]]
    g, og = _load(H, oracle, spec)
    for k in (10, 50, 100):
        r1, r2 = g.pool(tag=0, roots="stratified"), g.pool(tag=1, roots="stratified")
        seeds, res = g.select_seeds(r1, r2, k, mode="brr", eps=0.1, ell=1.0)
        oseeds, ores = oracle.brr(og, SEED, k, 0.1, 1.0, 0, "stratified")
        assert seeds.tolist() == oseeds.tolist(), k
        for key in ("rounds", "theta", "pool_r1", "pool_r2"):
            assert res[key] == ores[key], (k, key)
        assert res["lambda_r1"].tolist() == ores["lambda_r1"].tolist()
        assert res["lambda_r2"].tolist() == ores["lambda_r2"].tolist()
        for key in ("sigma_r1", "sigma_r2", "upper", "lower", "alpha"):
            assert abs(res[key] - ores[key]) <= REL * max(1.0, abs(ores[key])), (k, key)
        r1.close()
        r2.close()


@pytest.mark.parametrize("rank", [16, 32, 48, 63])
def test_batched_early_rounds(H, oracle, rank):
    specs = batch_workload()
    spec = specs[_by_size(specs)[rank]]
    g, og = _load(H, oracle, spec)
    for k in (10, 50, 100):
        _early_rounds(H, oracle, g, og, spec.n, k, 0.1)


def test_served_early_rounds(H, oracle):
    specs = serving_workload()
    gi = _by_size(specs)[0]
    queries = [q for q in serving_queries() if q.graph == gi][:3]
    assert len(queries) == 3
    g, og = _load(H, oracle, specs[gi])
    for q in queries:
        _early_rounds(H, oracle, g, og, specs[gi].n, q.k, q.eps)
