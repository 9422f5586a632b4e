"""The boundary's device-memory hooks and its bounded device waits, on the GPU.

* Allocator hooks (hyperim_load_args.dev_alloc / dev_free): a graph loaded with PyTorch's caching
  allocator as its device allocator gets every buffer of the graph, its shares and its pools from
  it (counted), returns every one of them, and computes the same RR sets and seeds as a graph
  using the library's own stream-ordered allocator; a query server on such a graph too.
* Bounded waits (hyperim_graph_set_wait_limit): with a limit of one round the RR kernel's work
  queue waits run out; the launch ends, the call reports HYPERIM_ETIMEDOUT, and the same handle
  (limit restored) and a fresh handle then produce the oracle's RR sets.
"""
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


def _graph_inputs():
    n, hes = gc.hub_graph(seed=3, n=6000, hub_edges=20, hub_size=120, mid_edges=6, mid_size=200, m_rest=2500)
    return n, hes


def test_caching_allocator_hooks(H):
    import torch
    n, hes = _graph_inputs()
    off, mem = gc.csr(hes)
    A = H.torch_caching_allocator()
    base = torch.cuda.memory_allocated()
    g = H.Graph(n, off, mem, "uniform_pair", 214748364, seed=7, allocator=A)
    ref = H.Graph(n, off, mem, "uniform_pair", 214748364, seed=7)
    assert A.allocs > 0 and torch.cuda.memory_allocated() > base
    pa, pb = g.pool(tag=0, roots="stratified").sample(700), ref.pool(tag=0, roots="stratified").sample(700)
    a, b = pa.to_host(), pb.to_host()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    r1, r2 = g.pool(tag=0, roots="stratified"), g.pool(tag=1, roots="stratified")
    q1, q2 = ref.pool(tag=0, roots="stratified"), ref.pool(tag=1, roots="stratified")
    s1, res1 = g.select_seeds(r1, r2, 8, mode="brr", eps=0.3)
    s2, res2 = ref.select_seeds(q1, q2, 8, mode="brr", eps=0.3)
    assert s1.tolist() == s2.tolist() and res1["theta"] == res2["theta"]
    # a share and the query server draw from the same hooks
    sh = g.share()
    p3 = sh.pool(tag=2, roots="plain").sample(300)
    srv = H.Server(workers=2)
    gid = srv.add_graph(g)
    t = srv.submit(gid, 8, 0.3)
    s4, r4 = srv.wait(t)
    assert r4["status"] == 0 and s4.tolist() == s2.tolist()
    srv.close()
    for p in (pa, r1, r2, p3):
        p.close()
    sh.close()
    g.close()
    torch.cuda.synchronize()
    assert A.frees == A.allocs, (A.allocs, A.frees)
    assert torch.cuda.memory_allocated() == base
    for p in (pb, q1, q2):
        p.close()
    ref.close()


def test_wait_limit_runs_out(H, oracle):
    n, hes = gc.random_graph(11, 4000, 3000, 8)
    off, mem = gc.csr(hes)
    thr = 1288490188  # p = 0.3: RR sets of hundreds of members, several warps per set
    g = H.Graph(n, off, mem, "uniform_pair", thr, seed=3)
    g.set_wait_limit(1)
    with pytest.raises(H.HyperIMError) as e:
        g.pool(tag=0, roots="plain").sample(400)
    assert e.value.status == -4  # HYPERIM_ETIMEDOUT
    g.set_wait_limit(0)
    og = oracle.Graph(n, off, mem, "uniform_pair", thr)
    op = oracle.Pool(og, seed=3, tag=0, roots="plain")
    op.grow_theta(400)
    gc.assert_same_pool(g.pool(tag=0, roots="plain").sample(400), op)
    fresh = H.Graph(n, off, mem, "uniform_pair", thr, seed=3)
    gc.assert_same_pool(fresh.pool(tag=0, roots="plain").sample(400), op)
    g.close()
    fresh.close()
