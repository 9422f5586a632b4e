"""Pins of the oracle's incidence store and layer profile (Sec. 2.1, Sec. 3.1.1) against a dense
brute-force w(mu,nu) matrix, the paper's Fig. 3 text facts, Lemma 1 and its l = 1 counterexample."""
import json
import math
import os

import numpy as np
import pytest

from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
P32 = 1 << 32


def random_hypergraph(rng, n, m, smax, repeat=True):
    hes = []
    for _ in range(m):
        s = int(rng.integers(0, smax + 1))
        he = [int(x) for x in rng.integers(0, n, size=s)]
        if repeat and he and rng.random() < 0.3:
            he.append(he[0])  # a repeated id (collapsed on load)
        hes.append(he)
    return hes


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("model", ["uniform_pair", "wc", "paper_layer"])
def test_profile_matches_bruteforce(oracle, seed, model):
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(3, 40)), int(rng.integers(1, 30))
    hes = random_hypergraph(rng, n, m, 8)
    W = bf.weights(n, hes)
    off, mem = bf.to_csr(hes)
    uthr = 214748364
    g = oracle.Graph(n, off, mem, model, uthr)
    for mu in range(n):
        L, ws = bf.layers(W, mu)
        assert g.deg(mu) == int((W[mu] > 0).sum())
        assert g.nlayers(mu) == len(L)
        assert g.stratum(mu) == min(len(L), 15)
        thr = bf.thresholds(W, mu, model, uthr)
        got = g.layers(mu)
        assert [x[0] for x in got] == ws
        assert [x[1] for x in got] == [len(x) for x in L]
        assert [x[2] for x in got] == thr
        for i in range(1, len(L) + 1):
            assert g.layer_members(mu, i).tolist() == L[i - 1]
    for s in range(16):
        assert g.stratum_size(s) == sum(1 for mu in range(n) if min(g.nlayers(mu), 15) == s)


def test_fig3_set_division(oracle):
    spec = json.load(open(os.path.join(GOLDEN, "fig3_set_division.json")))
    off, mem = bf.to_csr(spec["hyperedges"])
    g = oracle.Graph(spec["n"], off, mem, "paper_layer")
    exp = spec["expect"]
    assert g.nlayers(1) == 4
    assert [g.layer_members(1, i).tolist() for i in range(1, 5)] == exp["layers_of_1"]
    assert g.deg(5) == exp["deg_5"]
    assert g.deg(9) == exp["deg_9"]
    for v in exp["isolated"]:
        assert g.nlayers(v) == 0 and g.deg(v) == 0 and g.stratum(v) == 0
    # Lemma 1 (first half): P(L_i) = n_i p_i is strictly decreasing in i
    lay = g.layers(1)
    mass = [n_i * thr / P32 for (_, n_i, thr) in lay]
    assert all(a > b for a, b in zip(mass, mass[1:]))
    assert abs(mass[0] - 1.0 / math.log(5.0)) < 1e-9  # l = 4: P(L_1) = 1/ln 5


def test_lemma1_sum_exceeds_one_is_clamped(oracle):
    # Lemma 1 claims sum_i P(L_i) <= 1, but for l = 1 P(L_1) = 1/ln 2 > 1: the single member's
    # probability is clamped to 1 (reading of the paper recorded with the oracle).
    off, mem = bf.to_csr([[0, 1]])
    g = oracle.Graph(2, off, mem, "paper_layer")
    assert g.layers(0) == [(1, 1, P32)]
    assert 1.0 / math.log(2.0) > 1.0
    # and for l >= 2 the sum H_l / ln(l+1) is still above 1 (H_2 / ln 3 = 1.365)
    assert sum(1.0 / i for i in range(1, 3)) / math.log(3.0) > 1.0


def test_normalisation_and_degenerate_hyperedges(oracle):
    hes = [[3, 3, 1], [], [2], [1, 3], [0, 0]]
    off, mem = bf.to_csr(hes)
    g = oracle.Graph(5, off, mem, "uniform_pair", 0)
    assert g.nnz() == 2 + 0 + 1 + 2 + 1
    assert g.layers(1) == [(2, 1, 0)]          # w(1,3) = 2
    assert g.layers(2) == [] and g.layers(4) == [] and g.layers(0) == []
    assert g.dh(3) == 2 and g.dh(2) == 1 and g.dh(4) == 0


def test_invalid_member_rejected(oracle):
    off, mem = bf.to_csr([[0, 5]])
    with pytest.raises(oracle.OracleError):
        oracle.Graph(3, off, mem)


def test_theta_lstar(oracle):
    rng = np.random.default_rng(3)
    hes = random_hypergraph(rng, 25, 20, 6)
    W = bf.weights(25, hes)
    off, mem = bf.to_csr(hes)
    g = oracle.Graph(25, off, mem)
    want = 0.0
    for mu in range(25):
        l = len(bf.layers(W, mu)[0])
        if l:
            want += l / math.log(l + 1)
    assert abs(g.theta_lstar() - want / 25) < 1e-12
