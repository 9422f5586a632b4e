"""The seeded input generators of the batched and served configurations (no HyperIM arithmetic):
shapes, ranges and the Poisson query stream's statistics."""
import math

import numpy as np

from workloads import batch_workload, make_hypergraph, serving_queries, serving_workload


def test_batch_shapes():
    specs = batch_workload()
    assert len(specs) == 64
    ns = np.array([s.n for s in specs])
    assert ns.min() >= 1000 and ns.max() <= 200_000
    for s in specs:
        assert 0.3 * s.n - 1 <= s.m <= 1.0 * s.n + 1
        assert (s.size_lo, s.size_hi, s.zipf_alpha) == (2, 300, 2.1)
    # log-uniform sizes: both decades represented
    assert (ns < 10_000).sum() >= 10 and (ns > 50_000).sum() >= 10
    # a small one is generated as specified: sizes within range, members distinct per hyperedge
    small = specs[int(np.argmin(ns))]
    off, mem = make_hypergraph(small)
    sizes = np.diff(off)
    assert len(sizes) == small.m and sizes.min() >= 2 and sizes.max() <= 300
    assert mem.min() >= 0 and mem.max() < small.n
    for i in range(small.m):
        he = mem[off[i]:off[i + 1]]
        assert len(np.unique(he)) == len(he)


def test_serving_shapes_and_stream():
    specs = serving_workload()
    assert len(specs) == 16
    for s in specs:
        assert 100_000 <= s.n <= 5_000_000 and s.m == int(min(0.6 * s.n, 3e6))
    q = serving_queries()
    assert len(q) == 2000
    t = np.array([x.arrival for x in q])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    # exponential inter-arrival times of mean 1/200 s: mean and coefficient of variation near 1
    assert abs(gaps.mean() - 1 / 200) < 4 * (1 / 200) / math.sqrt(len(gaps))
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    ks = np.array([x.k for x in q])
    assert ks.min() >= 10 and ks.max() <= 200 and len(np.unique(ks)) > 150
    assert {x.eps for x in q} == {0.05, 0.1, 0.2}
    assert {x.graph for x in q} == set(range(16))
    # seeded: the same stream twice
    assert serving_queries()[:50] == q[:50]
