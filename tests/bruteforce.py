"""Brute-force references for tiny hypergraphs, written directly from the definitions
(Sec. 2.1: G_w, w(mu,nu), deg; Sec. 3.1.1: layers; IC live-edge semantics; Eq. 1).
Independent of both the oracle and the CUDA library; only usable on tiny inputs."""
import itertools

import numpy as np

P32 = 1 << 32


def incidence(n, hyperedges):
    B = np.zeros((n, len(hyperedges)), dtype=np.int64)
    for e, he in enumerate(hyperedges):
        for v in set(he):
            B[v, e] = 1
    return B


def weights(n, hyperedges):
    """w[mu, nu] = number of hyperedges containing both (0 on the diagonal)."""
    B = incidence(n, hyperedges)
    W = B @ B.T
    np.fill_diagonal(W, 0)
    return W


def layers(W, mu):
    """Layers of A(mu): lists of neighbour ids (ascending) by descending w."""
    row = W[mu]
    ws = sorted({int(x) for x in row if x > 0}, reverse=True)
    return [[int(v) for v in np.nonzero(row == w)[0]] for w in ws], ws


def thresholds(W, mu, model, uthr=0):
    """floor(p 2^32) per layer of A(mu) (2^32 means p = 1)."""
    L, ws = layers(W, mu)
    deg = sum(len(x) for x in L)
    out = []
    for i, members in enumerate(L, start=1):
        if model == "uniform_pair":
            out.append(uthr)
        elif model == "wc":
            out.append(P32 if deg <= 1 else P32 // deg)
        else:
            import math
            pl = 1.0 / (i * math.log(len(L) + 1.0))
            pd = pl / len(members)
            out.append(P32 if pd >= 1.0 else int(pd * P32))
    return out


def directed_pairs(W, model, uthr=0):
    """[(nu, mu, p)]: nu can activate mu with probability p (live edge nu -> mu)."""
    n = W.shape[0]
    out = []
    for mu in range(n):
        L, _ = layers(W, mu)
        thr = thresholds(W, mu, model, uthr)
        for members, t in zip(L, thr):
            for nu in members:
                out.append((nu, mu, t / P32))
    return out


def reach_backward(n, live, root):
    """Vertices that reach root through live edges (the RR set of root in that world)."""
    into = [[] for _ in range(n)]
    for nu, mu in live:
        into[mu].append(nu)
    seen = {root}
    stack = [root]
    while stack:
        x = stack.pop()
        for y in into[x]:
            if y not in seen:
                seen.add(y)
                stack.append(y)
    return frozenset(seen)


def rr_distribution(n, pairs, root):
    """Exact distribution of the RR set of `root` by enumerating all live-edge worlds."""
    dist = {}
    m = len(pairs)
    assert m <= 22, "too many directed pairs to enumerate"
    probs = np.array([p for _, _, p in pairs])
    for mask in range(1 << m):
        pr = 1.0
        live = []
        for b in range(m):
            if mask >> b & 1:
                pr *= probs[b]
                live.append(pairs[b][:2])
            else:
                pr *= 1.0 - probs[b]
        if pr == 0.0:
            continue
        R = reach_backward(n, live, root)
        dist[R] = dist.get(R, 0.0) + pr
    return dist


def exact_spread(n, pairs, S):
    """sigma(S) = sum_root P(S meets RR(root)) (Eq. 1 with the exact RR distribution)."""
    S = set(S)
    total = 0.0
    for r in range(n):
        for R, pr in rr_distribution(n, pairs, r).items():
            if S & R:
                total += pr
    return total


def components(n, hyperedges):
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for he in hyperedges:
        he = list(set(he))
        for v in he[1:]:
            a, b = find(he[0]), find(v)
            if a != b:
                parent[a] = b
    comp = {}
    for v in range(n):
        comp.setdefault(find(v), set()).add(v)
    return {v: frozenset(comp[find(v)]) for v in range(n)}


def to_csr(hyperedges):
    off = np.zeros(len(hyperedges) + 1, dtype=np.int32)
    for i, he in enumerate(hyperedges):
        off[i + 1] = off[i] + len(he)
    mem = np.array([v for he in hyperedges for v in he], dtype=np.int32)
    return off, mem


def coverage_sets(pool_sets, S):
    S = set(S)
    return sum(1 for R in pool_sets if S & set(R))


def best_cover(pool_sets, n, k):
    best = 0
    for combo in itertools.combinations(range(n), k):
        best = max(best, coverage_sets(pool_sets, combo))
    return best
