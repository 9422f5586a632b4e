"""Whole-query GPU parity at full size: HyperIM_BRR (Alg. 4) through the C ABI on the benchmark
workloads (100k vertices / p = 0.01; 2M vertices / weighted cascade), on the batched
configuration's largest graph (k = 10, 50, 100) and on the first query of the served stream's
smallest graph, against the oracle's complete result stored in tests/golden/brr_*.json (written
by tests/golden/make_brr_golden.py, which calls only the oracle).

Every round's alpha, the final theta, pool sizes, seed set and per-stratum coverage must be
identical; the estimates and bounds are the same IEEE double sequences on both sides (compared
to 1e-12 relative). In the final round, 200 RR sets drawn at random (pool, stratum, index) are
compared with the oracle's by size and SHA-256 of their ids, and when the pools hold exactly the
final round's sets the work counters and the cost-model bytes of both pools must equal the
oracle's."""
import glob
import hashlib
import json
import os

import numpy as np
import pytest

from tests import gpu_cases as gc
from workloads import HypergraphSpec, make_hypergraph

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = sorted(glob.glob(os.path.join(HERE, "golden", "brr_*.json")))


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
    return abs(a - b) <= 1e-12 * max(abs(a), abs(b)) or a == b


@pytest.mark.parametrize("path", CASES, ids=[os.path.basename(p)[4:-5] for p in CASES])
def test_brr_whole_query(H, path):
    import torch
    doc = json.load(open(path))
    gs, q, want = doc["graph"], doc["query"], doc["result"]
    spec = HypergraphSpec(n=gs["n"], m=gs["m"], size_law=gs["size_law"], size_lo=gs["size_lo"],
                          size_hi=gs["size_hi"], zipf_alpha=gs["zipf_alpha"], membership=gs["membership"],
                          gamma=gs["gamma"], seed=gs["seed"])
    off, mem = make_hypergraph(spec)
    g = H.Graph(spec.n, torch.as_tensor(off).cuda(), torch.as_tensor(mem).cuda(), q["model"],
                q["uniform_threshold"], seed=q["seed"])
    r1 = g.pool(tag=0, roots=q["roots"], strategy=q["strategy"])
    r2 = g.pool(tag=1, roots=q["roots"], strategy=q["strategy"])
    seeds, res = g.select_seeds(r1, r2, q["k"], mode="brr", eps=q["eps"], ell=q["ell"])
    assert res["rounds"] == want["rounds"]
    assert res["theta"] == want["theta"]
    assert res["pool_r1"] == want["pool_r1"] and res["pool_r2"] == want["pool_r2"]
    assert seeds.tolist() == want["seeds"]
    assert res["lambda_r1"].tolist() == want["lambda_r1"]
    assert res["lambda_r2"].tolist() == want["lambda_r2"]
    for key in ("sigma_r1", "sigma_r2", "upper", "lower", "alpha"):
        assert _close(res[key], float.fromhex(want[key])), key
    assert len(res["alpha_round"]) == len(want["alpha_round"])
    for a, b in zip(res["alpha_round"], want["alpha_round"]):
        assert _close(a, float.fromhex(b))
    # sampled RR sets of the final round, by (pool tag, stratum, index)
    pools = {0: r1, 1: r2}
    host = {}
    for t, p in pools.items():
        poff, pmem, pst, pj = p.to_host()
        index = {(int(s), int(j)): i for i, (s, j) in enumerate(zip(pst.tolist(), pj.tolist()))}
        host[t] = (poff, pmem, index)
    for e in doc["sampled_sets"]:
        poff, pmem, index = host[e["tag"]]
        i = index[(e["stratum"], e["j"])]
        R = np.ascontiguousarray(pmem[poff[i]:poff[i + 1]], dtype="<i4")
        assert len(R) == e["size"], e
        assert hashlib.sha256(R.tobytes()).hexdigest() == e["sha256"], e
    # work counters and cost-model bytes of both pools when they hold exactly the final round
    v1, v2 = r1.view(), r2.view()
    if v1["count"] == want["pool_r1"] and v2["count"] == want["pool_r2"]:
        st = doc["oracle_stats"]
        for key in ("pops", "layers_seen", "draws", "mats", "mat_he", "mat_members", "selected"):
            assert v1[key] + v2[key] == st[key], key
        assert gc.algorithmic_bytes(v1) + gc.algorithmic_bytes(v2) == st["bytes_rr"]
    r1.close()
    r2.close()
    g.close()
