"""Seeded hypergraphs that steer the CUDA kernels through each of their paths, plus helpers
that compare a GPU pool with the oracle's pool set by set (no HyperIM arithmetic here)."""
import numpy as np

P32 = 1 << 32


def csr(hyperedges):
    off = np.zeros(len(hyperedges) + 1, dtype=np.int32)
    for i, he in enumerate(hyperedges):
        off[i + 1] = off[i] + len(he)
    mem = np.array([v for he in hyperedges for v in he], dtype=np.int32)
    return off, mem


def hub_graph(seed=0, n=20000, hub_edges=60, hub_size=250, mid_edges=10, mid_size=300, m_rest=3000):
    """Vertex 0 sits in hub_edges hyperedges of hub_size members (sum of sizes > 8192: bucketed
    block path); vertex 1 in mid_edges of mid_size (on-chip block path); the rest is sparse."""
    rng = np.random.default_rng(seed)
    hes = []
    for _ in range(hub_edges):
        hes.append([0] + [int(x) for x in rng.integers(2, n, size=hub_size - 1)])
    for _ in range(mid_edges):
        hes.append([1] + [int(x) for x in rng.integers(2, n, size=mid_size - 1)])
    for _ in range(m_rest):
        hes.append([int(x) for x in rng.integers(0, n, size=int(rng.integers(2, 6)))])
    return n, hes


def layered_hub_graph(seed=0, n=30000, groups=12, group_edges=(1, 2, 3, 5, 8, 13), size=120,
                      m_rest=4000):
    """Vertices 0..3 share group_edges[i] hyperedges with groups of co-members of varying size, so
    their neighbourhoods (several thousand members) have one layer per multiplicity in
    group_edges, plus sparse random hyperedges: chunk index with several layers."""
    rng = np.random.default_rng(seed)
    hes = []
    for hub in range(4):
        for gi in range(groups):
            w = group_edges[gi % len(group_edges)]
            common = [int(x) for x in rng.integers(4, n, size=size)]
            for _ in range(w):
                extra = [int(x) for x in rng.integers(4, n, size=size // 4)]
                hes.append([hub] + common + extra)
    for _ in range(m_rest):
        hes.append([int(x) for x in rng.integers(0, n, size=int(rng.integers(2, 6)))])
    return n, hes


def deep_layered_hub_graph(seed=0, n=40000, layers=150, per_layer=2, m_rest=3000):
    """Vertex 0 sits in `layers` hyperedges; for w = 1..layers, `per_layer` random co-members sit
    in exactly w of them (hyperedges 0..w-1), so A(0) has one layer per w and about
    per_layer * layers^2 / 2 members (repeats counted): many layers times many chunks, more
    (layer, chunk) counts than the index build keeps on chip. Plus sparse random hyperedges."""
    rng = np.random.default_rng(seed)
    ids = rng.choice(np.arange(1, n), size=layers * per_layer, replace=False)
    hes = [[0] for _ in range(layers)]
    for w in range(1, layers + 1):
        for v in ids[(w - 1) * per_layer:w * per_layer]:
            for j in range(w):
                hes[j].append(int(v))
    for _ in range(m_rest):
        hes.append([int(x) for x in rng.integers(0, n, size=int(rng.integers(2, 6)))])
    return n, hes


def layered_graph(depth=40, pad=100):
    """Vertex 0 shares exactly i hyperedges with vertex i (i = 1..depth): depth distinct layers."""
    hes = []
    for j in range(1, depth + 1):
        hes.append([0] + [i for i in range(j, depth + 1)])
    n = depth + 1 + pad
    for v in range(depth + 1, n - 1):
        hes.append([v, v + 1])
    return n, hes


def big_edge_graph(size=2000, n=2500):
    """One hyperedge of `size` members (A(mu) is one layer for each member: direct indexing)."""
    return n, [list(range(size))] + [[size + i, size + i + 1] for i in range(n - size - 1)]


def degenerate_graph():
    """Empty, single-member and repeated-member hyperedges and isolated vertices."""
    return 12, [[], [3], [2, 2, 5], [5, 2, 7, 7], [1, 1], [9, 10, 11, 9], [], [0, 4]]


def distinct_graph(seed=0, n=6000, edges=6, size=150, m_rest=2500):
    """Vertex 0 sits in `edges` disjoint hyperedges of `size` members: its neighbourhood has no
    repeated member (one layer of w = 1) and about (size - 1) * edges members; the rest is sparse
    with distinct members per hyperedge, so many small neighbourhoods have one layer too."""
    rng = np.random.default_rng(seed)
    pool = rng.permutation(np.arange(1, n))
    hes = [[0] + [int(x) for x in pool[i * (size - 1):(i + 1) * (size - 1)]] for i in range(edges)]
    for _ in range(m_rest):
        hes.append([int(x) + 1 for x in rng.choice(n - 1, size=int(rng.integers(2, 8)), replace=False)])
    return n, hes


def random_graph(seed, n, m, smax):
    rng = np.random.default_rng(seed)
    return n, [[int(x) for x in rng.integers(0, n, size=int(rng.integers(0, smax + 1)))]
               for _ in range(m)]


def gpu_sets(pool):
    off, mem, st, j = pool.to_host()
    order = np.lexsort((j, st))
    sets = [mem[off[i]:off[i + 1]].tolist() for i in order]
    return sets, st[order], j[order]


def oracle_sets(opool):
    a = opool.arrays()
    return [a.mem[a.off[i]:a.off[i + 1]].tolist() for i in range(len(a.off) - 1)], a.stratum, a.j


def assert_same_pool(gpu_pool, oracle_pool):
    gs, gst, gj = gpu_sets(gpu_pool)
    os_, ost, oj = oracle_sets(oracle_pool)
    assert len(gs) == len(os_), (len(gs), len(os_))
    assert np.array_equal(gst, ost) and np.array_equal(gj, oj)
    for i, (a, b) in enumerate(zip(gs, os_)):
        assert a == b, f"RR set {i} (stratum {gst[i]}, j {gj[i]}): gpu {a[:20]}... oracle {b[:20]}..."
    assert np.array_equal(gpu_pool.view()["n_s"], oracle_pool.counts())


def algorithmic_bytes(view):
    """Cost-model bytes of RR generation from a GPU pool's counters (see hyperim_pool_view_t):
    32 per sector touched, 8 per hyperedge of a materialising pop, 4 per output id, 8 per set."""
    return 32 * view["sectors"] + 8 * view["mat_he"] + 4 * view["total"] + 8 * view["count"]


def assert_same_counters(gpu_pool, oracle_pool):
    c = gpu_pool.counters()
    o = oracle_pool.stats()
    for k in ("pops", "layers_seen", "draws", "mats", "mat_he", "mat_members", "selected"):
        assert c[k] == o[k], (k, c[k], o[k])
    b = algorithmic_bytes(gpu_pool.view())
    assert b == o["bytes_rr"], ("algorithmic bytes", b, o["bytes_rr"])
