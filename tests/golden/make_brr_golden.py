"""Writes tests/golden/brr_*.json: the CPU oracle's complete HyperIM_BRR result (Alg. 4 with the
Sec. 4.2 bounds and the Eq. equation-max budget) on full-size workloads, for the GPU parity test
tests/test_gpu_brr_fullsize.py.

Calls only the oracle (oracle/) and the seeded input generators (workloads/): no value here comes
from the CUDA library. The pools are grown by the oracle's multi-threaded driver (or_pool_grow_mt:
the same single-threaded RR-set routine over disjoint (stratum, j) ranges, identical pools).

Per case the file holds the query, every round's alpha, the final round's theta, pool sizes,
seed set, per-stratum coverage of R1 and R2, the two estimates and bounds, the oracle's work
counters (both pools), and the SHA-256 of 200 RR sets of the final round drawn at random (pool
tag, stratum, index), each with its size.

    python tests/golden/make_brr_golden.py [case ...]      # default: every case
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from workloads import (batch_workload, make_hypergraph, serving_queries, serving_workload,  # noqa: E402
                       workload)

HERE = os.path.dirname(os.path.abspath(__file__))
SAMPLED_SETS = 200


def cases():
    """name -> (graph spec, model, uniform threshold, k, eps, ell, roots, strategy, seed)"""
    out = {}
    for name in ("zipf-100k-50k-p001", "zipf-2m-1m-wc"):
        w = workload(name)
        q = w.query
        out[name] = (w.graph, q.model, q.uniform_threshold, q.k, q.eps, q.ell, q.roots, q.strategy, q.seed)
    # the batched configuration's largest graph, queried with each of its k values
    specs = batch_workload()
    gi = max(range(len(specs)), key=lambda i: specs[i].n)
    for k in (10, 50, 100):
        out[f"batched-largest-k{k}"] = (specs[gi], "wc", 0, k, 0.1, 1.0, "stratified", "paper", 1)
    # the served configuration: the first query of the stream on its smallest resident graph
    sspecs = serving_workload()
    si = min(range(len(sspecs)), key=lambda i: sspecs[i].n)
    sq = next(q for q in serving_queries() if q.graph == si)
    out["served-smallest-first"] = (sspecs[si], "wc", 0, sq.k, sq.eps, 1.0, "stratified", "paper", 1)
    return out


def set_digest(members):
    a = np.ascontiguousarray(members, dtype="<i4")
    return hashlib.sha256(a.tobytes()).hexdigest()


def run(name, spec, model, uthr, k, eps, ell, roots, strategy, seed, threads):
    t0 = time.time()
    off, mem = make_hypergraph(spec)
    og = oracle.Graph(spec.n, off, mem, model, uthr)
    t1 = time.time()
    seeds, res = oracle.brr(og, seed, k, eps, ell, roots=roots, strategy=strategy, threads=threads)
    t2 = time.time()
    ns = og.allocate(roots, res["theta"])
    keys = [(tag, s, j) for tag in (0, 1) for s in range(16) for j in range(int(ns[s]))]
    rng = np.random.default_rng(20240602)
    pick = rng.choice(len(keys), size=min(SAMPLED_SETS, len(keys)), replace=False)
    sampled = []
    for i in sorted(int(x) for x in pick):
        tag, s, j = keys[i]
        R = og.rr_set(seed, tag, roots, s, j, strategy=strategy)
        sampled.append({"tag": tag, "stratum": s, "j": j, "size": int(len(R)), "sha256": set_digest(R)})
    t3 = time.time()
    doc = {
        "case": name,
        "source": "oracle (tests/golden/make_brr_golden.py); HyperIM_BRR, Alg. 4",
        "graph": {"n": spec.n, "m": spec.m, "size_law": spec.size_law, "size_lo": spec.size_lo,
                  "size_hi": spec.size_hi, "zipf_alpha": spec.zipf_alpha, "membership": spec.membership,
                  "gamma": spec.gamma, "seed": spec.seed},
        "query": {"model": model, "uniform_threshold": int(uthr), "k": int(k), "eps": eps, "ell": ell,
                  "roots": roots, "strategy": strategy, "seed": int(seed)},
        "result": {"rounds": int(res["rounds"]), "theta": int(res["theta"]),
                   "pool_r1": int(res["pool_r1"]), "pool_r2": int(res["pool_r2"]),
                   "seeds": [int(x) for x in seeds],
                   "lambda_r1": [int(x) for x in res["lambda_r1"]],
                   "lambda_r2": [int(x) for x in res["lambda_r2"]],
                   "sigma_r1": res["sigma_r1"].hex(), "sigma_r2": res["sigma_r2"].hex(),
                   "upper": res["upper"].hex(), "lower": res["lower"].hex(), "alpha": res["alpha"].hex(),
                   "alpha_round": [float(a).hex() for a in res["alpha_round"]]},
        "n_s_final": [int(x) for x in ns],
        "oracle_stats": {k2: int(v) for k2, v in res["stats"].items()},
        "sampled_sets": sampled,
        "seconds": {"build": round(t1 - t0, 1), "brr": round(t2 - t1, 1), "sampled": round(t3 - t2, 1),
                    "threads": threads},
    }
    path = os.path.join(HERE, f"brr_{name}.json")
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    print(f"{name}: rounds {res['rounds']} theta {res['theta']} ({t2 - t1:.0f} s BRR) -> {path}", flush=True)


def main():
    want = sys.argv[1:]
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    for name, args in cases().items():
        if want and name not in want:
            continue
        run(name, *args, threads=threads)


if __name__ == "__main__":
    main()
