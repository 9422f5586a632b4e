"""RR-generation scheduling on the GPU: every tuning of hyperim_graph_set_tuning (the warp phase
off or at several set limits, sets beyond the limit built again by a block) produces exactly the
oracle's RR sets and work counters, including sets whose hub pops go to the block path; and the
autotuner applies one of its timed candidates, reuses its choice for a graph of the same degree
profile, and never changes a query's result."""
import numpy as np
import pytest

from tests import gpu_cases as gc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_01911_gb300 import build
    build.build()
    import paper_2406_01911_gb300 as H
    return H


CASES = [
    # hub pops with more than 8,192 members (block path, bucketed) and mid-size ones, p = 0.05
    ("hub", lambda: gc.hub_graph(seed=2), 214748364, "stratified", 400),
    # several layers per hub, chunk-indexed neighbourhoods, p = 0.2
    ("layered", lambda: gc.layered_hub_graph(seed=4), 858993459, "plain", 700),
]


@pytest.mark.parametrize("name,make,thr,roots,theta", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("warp", [0, 1, 16, 64, 128])
def test_tunings_give_the_oracle_sets(H, oracle, name, make, thr, roots, theta, warp):
    n, hes = make()
    off, mem = gc.csr(hes)
    g = H.Graph(n, off, mem, "uniform_pair", thr, seed=9)
    g.set_tuning(warp_set_limit=warp)
    assert g.tuning()["warp_set_limit"] == warp
    og = oracle.Graph(n, off, mem, "uniform_pair", thr)
    op = oracle.Pool(og, seed=9, tag=0, roots=roots)
    op.grow_theta(theta // 2)
    op.grow_theta(theta)
    p = g.pool(tag=0, roots=roots).sample(theta // 2).sample(theta)
    gc.assert_same_pool(p, op)
    gc.assert_same_counters(p, op)
    p.close()
    g.close()


@pytest.mark.parametrize("name,make,thr,roots,theta", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("warp,arena,schedule", [(0, 1, "persistent"), (64, 3, "persistent"), (0, 2, "plain")])
def test_arena_repair_gives_the_oracle_sets(H, oracle, name, make, thr, roots, theta, warp, arena, schedule):
    # an output arena of 1-3 entries per set: nearly every set is built a second time by the
    # repair launch and written to the slot the first launch reserved; sets and work counters
    # (counted once) must still be the oracle's
    n, hes = make()
    off, mem = gc.csr(hes)
    g = H.Graph(n, off, mem, "uniform_pair", thr, seed=9)
    g.set_tuning(warp_set_limit=warp, arena_entries_per_set=arena)
    g.set_schedule(schedule)
    assert g.tuning()["arena_entries_per_set"] == arena
    og = oracle.Graph(n, off, mem, "uniform_pair", thr)
    op = oracle.Pool(og, seed=9, tag=0, roots=roots)
    op.grow_theta(theta // 2)
    op.grow_theta(theta)
    p = g.pool(tag=0, roots=roots).sample(theta // 2).sample(theta)
    gc.assert_same_pool(p, op)
    gc.assert_same_counters(p, op)
    if schedule == "persistent":
        assert p.view()["rr_launches"] > 2  # two growths, at least one of them repaired
    p.close()
    g.close()


def test_autotune_choice_and_cache(H):
    n, hes = gc.hub_graph(seed=6)
    off, mem = gc.csr(hes)
    g = H.Graph(n, off, mem, "uniform_pair", 214748364, seed=3)
    r1, r2 = g.pool(tag=0, roots="stratified"), g.pool(tag=1, roots="stratified")
    seeds_before, res_before = g.select_seeds(r1, r2, 5, mode="brr", eps=0.3)
    t = g.autotune(roots="stratified", strategy="paper", sets=400)
    assert not t["from_cache"] and len(t["candidates"]) == 5
    assert t["warp_set_limit"] in [w for w, _ in t["candidates"]]
    best = min(s for _, s in t["candidates"])
    chosen = [s for w, s in t["candidates"] if w == t["warp_set_limit"]][0]
    assert chosen == best
    assert g.tuning()["warp_set_limit"] == t["warp_set_limit"]
    q1, q2 = g.pool(tag=0, roots="stratified"), g.pool(tag=1, roots="stratified")
    seeds_after, res_after = g.select_seeds(q1, q2, 5, mode="brr", eps=0.3)
    assert seeds_after.tolist() == seeds_before.tolist() and res_after["theta"] == res_before["theta"]
    # a second graph of the same degree profile takes the cached choice
    g2 = H.Graph(n, off, mem, "uniform_pair", 214748364, seed=4)
    t2 = g2.autotune(roots="stratified", strategy="paper", sets=400)
    assert t2["from_cache"] and t2["profile_key"] == t["profile_key"]
    assert t2["warp_set_limit"] == t["warp_set_limit"]
    for p in (r1, r2, q1, q2):
        p.close()
    g.close()
    g2.close()
