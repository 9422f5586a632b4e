"""The batched form of HyperIM_BRR (hyperim_select_seeds_batch): all queries advance round by
round, every round's RR growth across graphs is one persistent launch over a device work
counter, and every round's greedy + R2 coverage is one launch with a block per query.

* Against the oracle: the stored whole-query results of tests/golden/brr_*.json (the 100k and 2M
  benchmark workloads, the batched configuration's largest graph with k = 10, 50, 100 sharing one
  pool pair, the served stream's smallest graph) in ONE batch call: rounds, theta, seeds, Lambda
  per stratum, every round's alpha and the bounds.
* The batched configuration itself (64 graphs x k in {10, 50, 100}, queries of a graph sharing
  its pools): every query equals hyperim_select_seeds in BRR mode on fresh pools.
* Edge cases: one query; k = n on a tiny graph; a graph without hyperedges; pools grown further
  beforehand (prefix views); a share handle; plain and stratified roots and the LT sampler in the
  same batch; argument errors.
"""
import glob
import json
import os

import pytest

from tests import gpu_cases as gc
from workloads import HypergraphSpec, batch_workload, make_hypergraph

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
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


def _close(a, b):
    return a == b or abs(a - b) <= REL * max(abs(a), abs(b))


def _same(res, ref, seeds, ref_seeds):
    assert seeds.tolist() == list(ref_seeds)
    for key in ("rounds", "theta", "pool_r1", "pool_r2"):
        assert res[key] == ref[key], key
    assert res["lambda_r1"].tolist() == list(ref["lambda_r1"])
    assert res["lambda_r2"].tolist() == list(ref["lambda_r2"])
    for key in ("sigma_r1", "sigma_r2", "upper", "lower", "alpha"):
        assert _close(res[key], ref[key]), key
    assert len(res["alpha_round"]) == len(ref["alpha_round"])
    for a, b in zip(res["alpha_round"], ref["alpha_round"]):
        assert _close(a, b)


def test_batch_equals_the_oracle_golden_queries(H):
    import torch
    graphs, queries, want = {}, [], []
    for path in sorted(glob.glob(os.path.join(HERE, "golden", "brr_*.json"))):
        doc = json.load(open(path))
        gs, q, res = doc["graph"], doc["query"], doc["result"]
        key = (json.dumps(gs, sort_keys=True), q["model"], q["uniform_threshold"], q["seed"], q["roots"],
               q["strategy"])
        if key not in graphs:
            spec = HypergraphSpec(n=gs["n"], m=gs["m"], size_law=gs["size_law"], size_lo=gs["size_lo"],
                                  size_hi=gs["size_hi"], zipf_alpha=gs["zipf_alpha"],
                                  membership=gs["membership"], gamma=gs["gamma"], seed=gs["seed"])
            off, mem = make_hypergraph(spec)
            g = H.Graph(spec.n, torch.as_tensor(off).cuda(), torch.as_tensor(mem).cuda(), q["model"],
                        q["uniform_threshold"], seed=q["seed"])
            graphs[key] = (g, g.pool(tag=0, roots=q["roots"], strategy=q["strategy"]),
                           g.pool(tag=1, roots=q["roots"], strategy=q["strategy"]))
        g, r1, r2 = graphs[key]
        queries.append((g, r1, r2, q["k"], q["eps"], q["ell"]))
        ref = dict(res)
        for k in ("sigma_r1", "sigma_r2", "upper", "lower", "alpha"):
            ref[k] = float.fromhex(res[k])
        ref["alpha_round"] = [float.fromhex(a) for a in res["alpha_round"]]
        want.append(ref)
    assert len(queries) >= 6 and len(graphs) < len(queries)  # the batched graph's three k share pools
    out = H.hyperim_select_seeds_batch(queries)
    for (seeds, res), ref in zip(out, want):
        _same(res, ref, seeds, ref["seeds"])
    for g, r1, r2 in graphs.values():
        r1.close()
        r2.close()
        g.close()


def test_batched_configuration_equals_single_queries(H):
    import torch
    specs = batch_workload()
    loaded = []
    for sp in specs:
        off, mem = make_hypergraph(sp)
        loaded.append(H.Graph(sp.n, torch.as_tensor(off).cuda(), torch.as_tensor(mem).cuda(), "wc", 0, seed=1))
    pools = [(g.pool(tag=0, roots="stratified"), g.pool(tag=1, roots="stratified")) for g in loaded]
    queries = [(loaded[i], pools[i][0], pools[i][1], k, 0.1, 1.0) for i in range(len(specs)) for k in (10, 50, 100)]
    launches = H.hyperim_kernel_launches()
    out = H.hyperim_select_seeds_batch(queries)
    launches = H.hyperim_kernel_launches() - launches
    rounds = max(res["rounds"] for _, res in out)
    for (g, _, _, k, eps, ell), (seeds, res) in zip(queries, out):
        r1, r2 = g.pool(tag=0, roots="stratified"), g.pool(tag=1, roots="stratified")
        s_ref, ref = g.select_seeds(r1, r2, k, mode="brr", eps=eps, ell=ell)
        _same(res, ref, seeds, s_ref.tolist())
        r1.close()
        r2.close()
    # per round: one RR launch, one greedy launch, and the compaction of each grown pool
    assert launches <= rounds * (2 + 2 * len(specs) * 8), launches
    for (a, b), g in zip(pools, loaded):
        a.close()
        b.close()
        g.close()


def test_batch_edge_cases(H):
    n0, hes0 = gc.random_graph(6, 3000, 2500, 6)
    g0 = H.Graph(n0, *gc.csr(hes0), "wc", 0, seed=17)
    gt = H.Graph(5, *gc.csr([[0, 1], [1, 2, 3]]), "uniform_pair", 1 << 31, seed=4)
    ge = H.Graph(7, *gc.csr([]), "wc", 0, seed=2)
    n1, hes1 = gc.hub_graph(seed=1)
    g1 = H.Graph(n1, *gc.csr(hes1), "uniform_pair", 429496729, seed=9)
    share = g0.share()
    made = []

    def pools(g, roots="stratified", strategy="paper"):
        p = (g.pool(tag=0, roots=roots, strategy=strategy), g.pool(tag=1, roots=roots, strategy=strategy))
        made.extend(p)
        return p

    a = pools(g0)
    a[0].sample(20000)  # grown further than the query needs: the rounds read prefix views
    b = pools(g0, roots="plain")
    c = pools(gt)
    d = pools(ge)
    e = pools(g1, strategy="lt")
    f = pools(g1)
    queries = [(share, a[0], a[1], 20, 0.2, 1.0), (g0, b[0], b[1], 7, 0.3, 1.0), (gt, c[0], c[1], 5, 0.1, 1.0),
               (ge, d[0], d[1], 3, 0.2, 1.0), (g1, e[0], e[1], 30, 0.2, 1.0), (g1, f[0], f[1], 30, 0.2, 1.0)]
    out = H.hyperim_select_seeds_batch(queries)
    for (g, r1, r2, k, eps, ell), (seeds, res) in zip(queries, out):
        x, y = g.pool(tag=0, roots=r1.roots, strategy=r1.strategy), g.pool(tag=1, roots=r1.roots,
                                                                          strategy=r1.strategy)
        s_ref, ref = g.select_seeds(x, y, k, mode="brr", eps=eps, ell=ell)
        _same(res, ref, seeds, s_ref.tolist())
        assert sorted(set(seeds.tolist())) == sorted(seeds.tolist())  # never a vertex twice
        x.close()
        y.close()
    # one query alone
    (seeds, res), = H.hyperim_select_seeds_batch([queries[2]])
    _same(res, out[2][1], seeds, out[2][0].tolist())
    with pytest.raises(H.HyperIMError, match="ESTATE"):
        H.hyperim_select_seeds_batch([(g0, a[0], a[0], 5, 0.2, 1.0)])
    with pytest.raises(H.HyperIMError, match="EINVAL"):
        H.hyperim_select_seeds_batch([(gt, c[0], c[1], 6, 0.2, 1.0)])
    with pytest.raises(H.HyperIMError, match="ESTATE"):
        H.hyperim_select_seeds_batch([(g0, c[0], c[1], 5, 0.2, 1.0)])
    for p in made:
        p.close()
    share.close()
    for g in (g0, gt, ge, g1):
        g.close()


def test_batch_arena_repair_equals_the_oracle(H, oracle):
    # an output arena of one entry per set: every round's batched launch is repaired
    n, hes = gc.random_graph(6, 3000, 2500, 6)
    off, mem = gc.csr(hes)
    g = H.Graph(n, off, mem, "wc", 0, seed=17)
    g.set_tuning(arena_entries_per_set=1)
    og = oracle.Graph(n, off, mem, "wc", 0)
    r1, r2 = g.pool(tag=0, roots="stratified"), g.pool(tag=1, roots="stratified")
    queries = [(g, r1, r2, k, 0.2, 1.0) for k in (5, 10, 20)]
    out = H.hyperim_select_seeds_batch(queries)
    for (_, _, _, k, eps, ell), (seeds, res) in zip(queries, out):
        oseeds, ores = oracle.brr(og, 17, k, eps, ell, 0, "stratified")
        _same(res, ores, seeds, oseeds.tolist())
    r1.close()
    r2.close()
    g.close()
