"""Pins of the oracle's cost-model byte counter (or_stats.bytes_rr, the algorithmic bytes of RR
generation at 32-byte-sector granularity): recomputed from scratch, in Python, from the
normalised incidence lists and a brute-force layer profile, in the two cases where the pops and
their materialisations are fixed by the probabilities alone: p = 0 (every RR set is its root,
which never materialises A(mu)) and p = 1 (every RR set is the root's connected component, and
every vertex with a neighbour materialises)."""
import numpy as np
import pytest

from tests import bruteforce as bf
from tests import gpu_cases as gc


def sector_bytes(a, length):
    return 0 if length == 0 else 32 * ((a + length - 1) // 32 - a // 32 + 1)


def layout(n, hes):
    """normalised hyperedges, their offsets, each vertex's hyperedges and offsets, and the
    profile's entry offsets (layers counted from the brute-force weight matrix)"""
    norm = [sorted(set(he)) for he in hes]
    he_off = np.zeros(len(norm) + 1, np.int64)
    for i, he in enumerate(norm):
        he_off[i + 1] = he_off[i] + len(he)
    v_he = [[e for e, he in enumerate(norm) if v in he] for v in range(n)]
    v_off = np.zeros(n + 1, np.int64)
    for v in range(n):
        v_off[v + 1] = v_off[v] + len(v_he[v])
    W = bf.weights(n, hes)
    nl = [len(bf.layers(W, v)[1]) for v in range(n)]
    prof_off = np.zeros(n + 1, np.int64)
    for v in range(n):
        prof_off[v + 1] = prof_off[v] + nl[v]
    return norm, he_off, v_he, v_off, prof_off, nl


def pop_bytes(L, mu, materialises):
    norm, he_off, v_he, v_off, prof_off, nl = L
    b = sector_bytes(12 * int(prof_off[mu]), 12 * nl[mu])
    if materialises:
        b += sector_bytes(4 * int(v_off[mu]), 4 * len(v_he[mu]))
        for e in v_he[mu]:
            b += 8 + sector_bytes(4 * int(he_off[e]), 4 * len(norm[e]))
    return b


GRAPHS = [gc.random_graph(3, 40, 30, 6), gc.random_graph(4, 60, 25, 9), gc.degenerate_graph(),
          gc.layered_graph(depth=12, pad=20)]


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
@pytest.mark.parametrize("roots", ["plain", "stratified"])
def test_bytes_p0(oracle, gi, roots):
    n, hes = GRAPHS[gi]
    L = layout(n, hes)
    off, mem = bf.to_csr(hes)
    g = oracle.Graph(n, off, mem, "uniform_pair", 0)
    pool = oracle.Pool(g, seed=5, tag=0, roots=roots)
    pool.grow_theta(300)
    a = pool.arrays()
    want = 0
    for i in range(len(a.off) - 1):
        R = a.mem[a.off[i]:a.off[i + 1]].tolist()
        assert len(R) == 1
        want += pop_bytes(L, R[0], False) + 4 * len(R) + 8
    assert pool.stats()["bytes_rr"] == want


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
@pytest.mark.parametrize("roots", ["plain", "stratified"])
def test_bytes_p1(oracle, gi, roots):
    n, hes = GRAPHS[gi]
    L = layout(n, hes)
    comp = bf.components(n, hes)
    off, mem = bf.to_csr(hes)
    g = oracle.Graph(n, off, mem, "uniform_pair", 1 << 32)
    pool = oracle.Pool(g, seed=6, tag=0, roots=roots)
    pool.grow_theta(200)
    a = pool.arrays()
    want = 0
    for i in range(len(a.off) - 1):
        R = a.mem[a.off[i]:a.off[i + 1]].tolist()
        assert set(R) == set(comp[R[0]])  # every member lies in the root's component
        want += sum(pop_bytes(L, mu, L[5][mu] > 0) for mu in R) + 4 * len(R) + 8
    assert pool.stats()["bytes_rr"] == want


def test_sector_arithmetic():
    # byte ranges against 32-byte sectors: empty, inside one sector, straddling, aligned
    assert sector_bytes(0, 0) == 0 and sector_bytes(31, 0) == 0
    assert sector_bytes(0, 1) == 32 and sector_bytes(0, 32) == 32 and sector_bytes(0, 33) == 64
    assert sector_bytes(28, 8) == 64 and sector_bytes(32, 32) == 32 and sector_bytes(12, 12) == 32
