"""Seeded synthetic hypergraphs and IM query workloads.

This module is the one piece of code that both the CUDA path's tests/benchmarks and the CPU oracle
consume. It only produces inputs: hyperedge member lists and the query parameters that go with
them. It holds none of HyperIM's arithmetic (no layers, no thresholds, no sampling, no greedy).

Shapes stand in for the real hypergraphs of the paper's evaluation (Table 3: 1,005 to 1,261,129
vertices, 10,273 to 1,204,704 hyperedges), which are not available here.

Recipe (deterministic for a given seed):

* Random stream: numpy's PCG64 bit generator seeded through ``SeedSequence((seed, salt))``; only
  raw 64-bit outputs are used and turned into doubles in [0, 1) as ``(x >> 11) * 2**-53``, so the
  stream does not depend on numpy's distribution code.
* Hyperedge sizes: either uniform integers in [lo, hi] or a Zipf law P(s) ~ s^-alpha truncated to
  [lo, hi], drawn by inverting the exact discrete CDF.
* Membership: "uniform" draws members uniformly from V; "preferential" draws them with Chung-Lu
  weights pi_v ~ (v + i0)^(-1/(gamma-1)) (gamma = 2.5), where the offset i0 >= 1 is the smallest
  power of two for which the largest expected vertex degree stays below sqrt(nnz), the
  admissibility condition of the Chung-Lu model (w_max^2 <= sum w). Members of one hyperedge are
  distinct: duplicates are redrawn up to 8 times and any left after that are dropped.
* A random permutation of vertex ids is applied last, so that id order (the tie-break used
  throughout HyperIM's greedy) is not correlated with degree.
* Member lists are emitted in draw order (unsorted), which exercises the normalisation that the
  incidence store performs.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = [
    "HypergraphSpec", "QuerySpec", "Workload", "make_hypergraph", "WORKLOADS", "workload",
    "batch_workload", "serving_workload", "serving_queries", "ServingQuery", "uniform01",
]

_TWO_M53 = 2.0 ** -53


class _Stream:
    """Raw PCG64 stream -> doubles in [0,1) and bounded integers (platform independent)."""

    def __init__(self, seed: int, salt: int):
        ss = np.random.SeedSequence([int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF,
                                     int(salt) & 0xFFFFFFFF])
        self._bg = np.random.PCG64(ss)

    def uniform(self, size: int) -> np.ndarray:
        raw = self._bg.random_raw(size)
        return (raw >> np.uint64(11)).astype(np.float64) * _TWO_M53

    def below(self, bound: int, size: int) -> np.ndarray:
        """Integers in [0, bound) by multiply-shift of the top 32 bits (bound < 2^32)."""
        raw = self._bg.random_raw(size) >> np.uint64(32)
        return ((raw * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)


def uniform01(seed: int, salt: int, size: int) -> np.ndarray:
    """Seeded doubles in [0,1) for test inputs (same recipe as the graph generator)."""
    return _Stream(seed, salt).uniform(size)


@dataclasses.dataclass(frozen=True)
class HypergraphSpec:
    n: int                      # |V|
    m: int                      # |HE|
    size_law: str               # "uniform" or "zipf"
    size_lo: int
    size_hi: int
    zipf_alpha: float = 0.0
    membership: str = "uniform"  # "uniform" or "preferential"
    gamma: float = 2.5          # Chung-Lu exponent for preferential membership
    seed: int = 1


@dataclasses.dataclass(frozen=True)
class QuerySpec:
    model: str                  # "uniform_pair" | "wc" | "paper_layer"
    uniform_threshold: int      # floor(p * 2^32) for "uniform_pair" (2^32 means p = 1)
    k: int
    theta: Optional[int]        # fixed number of RR sets, or None for the adaptive schedule
    eps: float
    ell: float
    roots: str                  # "plain" | "stratified"
    seed: int = 1
    strategy: str = "paper"     # "paper" | "binomial_only" (IC) | "lt" (the LT cascade)


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    graph: HypergraphSpec
    query: QuerySpec
    description: str


def _sizes(spec: HypergraphSpec, st: _Stream) -> np.ndarray:
    lo, hi = spec.size_lo, spec.size_hi
    if spec.size_law == "uniform":
        return lo + st.below(hi - lo + 1, spec.m)
    if spec.size_law == "zipf":
        s = np.arange(lo, hi + 1, dtype=np.float64)
        pmf = s ** (-spec.zipf_alpha)
        cdf = np.cumsum(pmf)
        cdf /= cdf[-1]
        u = st.uniform(spec.m)
        idx = np.searchsorted(cdf, u, side="right")
        return lo + np.minimum(idx, hi - lo).astype(np.int64)
    raise ValueError(f"unknown size law {spec.size_law!r}")


def _chung_lu_cdf(n: int, gamma: float, nnz: int) -> np.ndarray:
    expo = 1.0 / (gamma - 1.0)
    cap = math.sqrt(max(nnz, 1))
    i0 = 1
    while True:
        w = (np.arange(n, dtype=np.float64) + i0) ** (-expo)
        tot = w.sum()
        if nnz * w[0] / tot <= cap or i0 > n:
            break
        i0 *= 2
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    return cdf


def make_hypergraph(spec: HypergraphSpec):
    """Return (he_off int32[m+1], he_mem int32[nnz]) for the spec."""
    st = _Stream(spec.seed, 0xF0)
    sizes = np.minimum(_sizes(spec, st), spec.n)
    nnz = int(sizes.sum())
    he_idx = np.repeat(np.arange(spec.m, dtype=np.int64), sizes)
    if spec.membership == "uniform":
        def draw(count):
            return st.below(spec.n, count)
    elif spec.membership == "preferential":
        cdf = _chung_lu_cdf(spec.n, spec.gamma, nnz)

        def draw(count):
            u = st.uniform(count)
            return np.minimum(np.searchsorted(cdf, u, side="right"), spec.n - 1).astype(np.int64)
    else:
        raise ValueError(f"unknown membership {spec.membership!r}")
    mem = draw(nnz)
    keep = np.ones(nnz, dtype=bool)
    for _ in range(9):
        key = he_idx * spec.n + mem
        order = np.argsort(key, kind="stable")
        sk = key[order]
        dup_sorted = np.zeros(nnz, dtype=bool)
        dup_sorted[1:] = sk[1:] == sk[:-1]
        dup = np.zeros(nnz, dtype=bool)
        dup[order] = dup_sorted
        if not dup.any():
            break
        if _ == 8:
            keep = ~dup
            break
        mem[dup] = draw(int(dup.sum()))
    perm = np.argsort(st.uniform(spec.n), kind="stable")   # random relabelling of vertex ids
    mem = perm[mem]
    mem = mem[keep]
    he_idx = he_idx[keep]
    counts = np.bincount(he_idx, minlength=spec.m)
    he_off = np.zeros(spec.m + 1, dtype=np.int64)
    np.cumsum(counts, out=he_off[1:])
    return he_off.astype(np.int32), mem.astype(np.int32)


# ------------------------------------------------------------------------------------------------
# Named workloads. Thresholds are floor(p * 2^32): p = 0.05 -> 214748364, p = 0.01 -> 42949672.
# ------------------------------------------------------------------------------------------------
WORKLOADS = {
    "tiny-1k-u2to6-p005": Workload(
        name="tiny-1k-u2to6-p005",
        graph=HypergraphSpec(n=1000, m=500, size_law="uniform", size_lo=2, size_hi=6,
                             membership="uniform", seed=1),
        query=QuerySpec(model="uniform_pair", uniform_threshold=214748364, k=10, theta=10000,
                        eps=0.1, ell=1.0, roots="plain", seed=1),
        description="1,000 vertices, 500 hyperedges of size U[2,6], uniform members; IC with "
                    "p=0.05 per co-member pair; k=10; fixed theta=10,000; plain roots"),
    "zipf-100k-50k-p001": Workload(
        name="zipf-100k-50k-p001",
        graph=HypergraphSpec(n=100_000, m=50_000, size_law="zipf", size_lo=2, size_hi=200,
                             zipf_alpha=2.1, membership="preferential", seed=1),
        query=QuerySpec(model="uniform_pair", uniform_threshold=42949672, k=50, theta=None,
                        eps=0.1, ell=1.0, roots="stratified", seed=1),
        description="100k vertices, 50k hyperedges, Zipf(2.1) sizes in [2,200], preferential "
                    "membership; IC with p=0.01; k=50; eps=0.1, delta=1/n; adaptive theta; "
                    "stratified roots"),
    "zipf-100k-50k-paper": Workload(
        name="zipf-100k-50k-paper",
        graph=HypergraphSpec(n=100_000, m=50_000, size_law="zipf", size_lo=2, size_hi=200,
                             zipf_alpha=2.1, membership="preferential", seed=1),
        query=QuerySpec(model="paper_layer", uniform_threshold=0, k=50, theta=None,
                        eps=0.1, ell=1.0, roots="stratified", seed=1),
        description="100k vertices, 50k hyperedges, Zipf(2.1) sizes in [2,200], preferential "
                    "membership (the zipf-100k-50k-p001 graph); the paper's layer probabilities "
                    "p_i = 1/(i ln(l+1)) / n_i; k=50; eps=0.1, delta=1/n; adaptive theta; "
                    "stratified roots"),
    "zipf-2m-1m-lt": Workload(
        name="zipf-2m-1m-lt",
        graph=HypergraphSpec(n=2_000_000, m=1_000_000, size_law="zipf", size_lo=2, size_hi=1000,
                             zipf_alpha=1.9, membership="preferential", seed=1),
        query=QuerySpec(model="wc", uniform_threshold=0, k=100, theta=None, eps=0.1, ell=1.0,
                        roots="stratified", seed=1, strategy="lt"),
        description="the zipf-2m-1m-wc graph under the LT cascade (live-edge form, one kept "
                    "in-neighbour per pop) with weighted-cascade weights p=1/deg; k=100; eps=0.1, "
                    "delta=1/n; adaptive theta; stratified roots"),
    "zipf-2m-1m-wc": Workload(
        name="zipf-2m-1m-wc",
        graph=HypergraphSpec(n=2_000_000, m=1_000_000, size_law="zipf", size_lo=2, size_hi=1000,
                             zipf_alpha=1.9, membership="preferential", seed=1),
        query=QuerySpec(model="wc", uniform_threshold=0, k=100, theta=None, eps=0.1, ell=1.0,
                        roots="stratified", seed=1),
        description="2M vertices, 1M hyperedges, Zipf(1.9) sizes in [2,1000], preferential "
                    "membership; weighted cascade p=1/deg; k=100; eps=0.1, delta=1/n; adaptive "
                    "theta; stratified roots"),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def batch_workload(count: int = 64, seed: int = 1):
    """Many hypergraphs of uneven size: n log-uniform in [1e3, 2e5], m/n in [0.3, 1.0],
    Zipf(2.1) sizes in [2,300], preferential membership; each queried with k in {10, 50, 100}."""
    st = _Stream(seed, 0xB0)
    u = st.uniform(2 * count)
    out = []
    for g in range(count):
        n = int(round(math.exp(math.log(1e3) + u[2 * g] * (math.log(2e5) - math.log(1e3)))))
        m = max(2, int(round(n * (0.3 + 0.7 * u[2 * g + 1]))))
        spec = HypergraphSpec(n=n, m=m, size_law="zipf", size_lo=2, size_hi=300, zipf_alpha=2.1,
                              membership="preferential", seed=seed * 1000 + g)
        out.append(spec)
    return out


def serving_workload(count: int = 16, seed: int = 1):
    """Resident hypergraphs for a query stream: n log-uniform in [1e5, 5e6],
    m = min(0.6 n, 3e6), Zipf(2.0) sizes in [2,500], preferential membership."""
    st = _Stream(seed, 0x5E)
    u = st.uniform(count)
    out = []
    for g in range(count):
        n = int(round(math.exp(math.log(1e5) + u[g] * (math.log(5e6) - math.log(1e5)))))
        m = int(min(0.6 * n, 3e6))
        out.append(HypergraphSpec(n=n, m=m, size_law="zipf", size_lo=2, size_hi=500,
                                  zipf_alpha=2.0, membership="preferential",
                                  seed=seed * 2000 + g))
    return out


@dataclasses.dataclass(frozen=True)
class ServingQuery:
    arrival: float              # seconds from the start of the stream
    graph: int                  # index into serving_workload()
    k: int
    eps: float


def serving_queries(count: int = 2000, rate: float = 200.0, graphs: int = 16, seed: int = 1):
    """A Poisson stream of IM queries over the resident graphs: exponential inter-arrival times
    of mean 1/rate (inversion of seeded uniforms), graph uniform over `graphs`, k uniform in
    [10, 200], eps uniform over {0.05, 0.1, 0.2}."""
    st = _Stream(seed, 0x5F)
    u = st.uniform(4 * count)
    out, t = [], 0.0
    for i in range(count):
        t += -math.log1p(-float(u[4 * i])) / rate
        out.append(ServingQuery(arrival=t, graph=min(int(u[4 * i + 1] * graphs), graphs - 1),
                                k=10 + min(int(u[4 * i + 2] * 191), 190),
                                eps=(0.05, 0.1, 0.2)[min(int(u[4 * i + 3] * 3), 2)]))
    return out

