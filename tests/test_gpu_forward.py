"""GPU parity of the forward Monte-Carlo influence (Sec. 2.2 cascade, IC model) with the oracle:
every simulation's activated count identical, on random graphs under the three activation
settings, on hubs whose neighbourhoods are taken id range by id range, on degenerate inputs, and
on the 100k benchmark graph; plus the argument checks and the mean / standard error."""
import math

import numpy as np
import pytest

from tests import gpu_cases as gc
from workloads import make_hypergraph, workload

pytestmark = pytest.mark.gpu
P32 = 1 << 32


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_01911_gb300 import build
    build.build()
    import paper_2406_01911_gb300 as H
    return H


def both(H, oracle, n, hes, model, uthr=0):
    off, mem = gc.csr(hes)
    return H.Graph(n, off, mem, model, uthr, seed=1), oracle.Graph(n, off, mem, model, uthr)


@pytest.mark.parametrize("model,uthr", [("uniform_pair", 429496729), ("wc", 0), ("paper_layer", 0),
                                        ("uniform_pair", P32)])
def test_random_graphs(H, oracle, model, uthr):
    n, hes = gc.random_graph(4, 400, 330, 9)
    g, og = both(H, oracle, n, hes, model, uthr)
    for S in ([3], [0, 1, 2, 2, 399], list(range(0, 400, 37))):
        counts, mean, se = g.forward_spread(S, 300, seed=77)
        want = og.forward_spread(S, 300, seed=77)
        assert counts.tolist() == want.tolist(), (model, S)
        c = want.astype(np.float64)
        assert mean == pytest.approx(c.mean(), rel=1e-12)
        assert se == pytest.approx(c.std(ddof=1) / math.sqrt(len(c)), rel=1e-9)


@pytest.mark.parametrize("model,uthr", [("wc", 0), ("uniform_pair", 4294967)])
def test_hubs(H, oracle, model, uthr):
    # vertex 0 holds ~15K neighbourhood members and vertex 1 ~3K: taken id range by id range
    n, hes = gc.hub_graph()
    g, og = both(H, oracle, n, hes, model, uthr)
    for S in ([0], [1, 5], [0, 1, 2, 3]):
        counts, _, _ = g.forward_spread(S, 64, seed=3)
        assert counts.tolist() == og.forward_spread(S, 64, seed=3).tolist(), (model, S)


def test_degenerate_and_errors(H, oracle):
    n, hes = gc.degenerate_graph()
    g, og = both(H, oracle, n, hes, "uniform_pair", 1 << 31)
    for S in ([0], [4, 4], [], list(range(n))):
        counts, _, _ = g.forward_spread(S, 50, seed=9)
        assert counts.tolist() == og.forward_spread(S, 50, seed=9).tolist(), S
    counts, mean, se = g.forward_spread([6], 1, seed=9)
    assert counts.tolist() == [1] and mean == 1.0 and se == 0.0
    for bad in (([n], 5), ([-1], 5), ([0], 0)):
        with pytest.raises(Exception):
            g.forward_spread(bad[0], bad[1], seed=1)


def test_zipf_100k_graph(H, oracle):
    w = workload("zipf-100k-50k-p001")
    off, mem = make_hypergraph(w.graph)
    q = w.query
    g = H.Graph(w.graph.n, off, mem, q.model, q.uniform_threshold, seed=q.seed)
    og = oracle.Graph(w.graph.n, off, mem, q.model, q.uniform_threshold)
    S = [int(x) for x in np.random.default_rng(5).choice(w.graph.n, size=50, replace=False)]
    counts, _, _ = g.forward_spread(S, 24, seed=11)
    assert counts.tolist() == og.forward_spread(S, 24, seed=11).tolist()
