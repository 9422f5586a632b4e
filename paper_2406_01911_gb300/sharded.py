"""HyperIM_BRR (Algorithm 4) with the RR pools split over several ranks (GPUs or processes).

The path shards naturally: RR set (s, j) is a pure function of (seed, pool tag, stratum, index),
so rank r of W generates the sets with j = r (mod W) of every growth's allocation
(hyperim_sample_rr_shard) and the union over ranks is exactly the single-GPU pool -- no exchange.
Greedy max coverage (Algorithm 1) then needs one exchange per round: the all-reduce (sum) of the
n-length integer score vector of Eq. 2, after which every rank picks the same vertex (integer
weights, ties to the lowest id) and retires the sets of its own shard that it covers. The
per-stratum coverages of R1 (the greedy's) and R2 (the lower bound's) are all-reduced once per
round (16 integers each), and the round's bounds and stop test are the host arithmetic of
hyperim_brr_round. The result equals hyperim_select_seeds in BRR mode on one GPU: same rounds,
theta, seeds, coverages and bounds.

`sharded_brr` is written against a small engine interface, so the same driver runs the shards of
this process's GPU (`GpuShards`, through the C ABI) with NCCL between processes, or any other
engine that computes the same quantities.
"""
from __future__ import annotations

from typing import Callable, Optional, Sequence

import numpy as np

from . import GreedyRounds, ShardPool, hyperim_brr_round, hyperim_coverage_view, hyperim_plan_theta

NSTRATA = 16


class GpuShards:
    """The R1 and R2 shards (ranks `ranks` of `world`) that this process holds on its GPU.

    Scores and coverages are returned as int64 CUDA tensors (uint64 values; an all-reduce sum in
    int64 wraps exactly like uint64), so NCCL can all-reduce them in place."""

    def __init__(self, graph, ranks: Sequence[int], world: int, roots="stratified", strategy="paper"):
        import torch
        self.torch = torch
        self.g = graph
        self.n = graph.n
        self.roots = roots
        self.r1 = [ShardPool(graph, 0, r, world, roots, strategy) for r in ranks]
        self.r2 = [ShardPool(graph, 1, r, world, roots, strategy) for r in ranks]
        self._total = torch.zeros(self.n, dtype=torch.int64, device="cuda")
        self._buf = torch.zeros(self.n, dtype=torch.int64, device="cuda")
        self._states = []

    def plan(self, k, eps, ell):
        return hyperim_plan_theta(self.g.handle, k, eps, ell)

    def grow(self, theta):
        for p in self.r1 + self.r2:
            p.sample(theta)

    def greedy_begin(self, theta):
        self._states = [GreedyRounds(self.g, p, theta) for p in self.r1]

    def local_scores(self):
        """The summed scores of this process's R1 shards (a CUDA tensor it may all-reduce)."""
        self._total.zero_()
        for st in self._states:
            st.scores_into(self._buf.data_ptr())
            self._total += self._buf
        return self._total

    def pick(self, total) -> int:
        picks = {st.pick(total.data_ptr()) for st in self._states}
        if len(picks) != 1:
            raise RuntimeError(f"shards of one process picked different vertices: {sorted(picks)}")
        return picks.pop()

    def greedy_end(self):
        lam = sum((st.end().astype(np.int64) for st in self._states), np.zeros(NSTRATA, np.int64))
        self._states = []
        return self.torch.as_tensor(lam, device="cuda")

    def coverage(self, seeds, theta):
        lam = sum((hyperim_coverage_view(self.g, p, theta, seeds).astype(np.int64) for p in self.r2),
                  np.zeros(NSTRATA, np.int64))
        return self.torch.as_tensor(lam, device="cuda")

    def round(self, k, eps, ell, i, lam1, lam2):
        a = np.asarray(lam1.cpu() if hasattr(lam1, "cpu") else lam1).astype(np.uint64)
        b = np.asarray(lam2.cpu() if hasattr(lam2, "cpu") else lam2).astype(np.uint64)
        return hyperim_brr_round(self.g, k, eps, ell, self.roots, i, a, b)

    def close(self):
        for p in self.r1 + self.r2:
            p.close()


def sharded_brr(engine, k: int, eps: float, ell: float = 1.0,
                all_reduce: Optional[Callable] = None):
    """HyperIM_BRR over sharded pools. `engine` holds this process's shards (see GpuShards);
    `all_reduce(x)` sums a tensor over every process in place (None: this process holds all the
    shards). Returns (seeds, result) with the fields of hyperim_select_seeds' BRR result that the
    rounds determine: rounds, theta, lambda_r1 / lambda_r2 (summed over the shards), sigma_r1,
    sigma_r2, upper, lower, alpha and alpha_round."""
    plan = engine.plan(k, eps, ell)
    alphas = []
    for i in range(63):
        theta = int(plan["theta0"]) << i
        engine.grow(theta)
        engine.greedy_begin(theta)
        seeds = []
        for _ in range(k):
            total = engine.local_scores()
            if all_reduce is not None:
                all_reduce(total)
            seeds.append(engine.pick(total))
        lam1 = engine.greedy_end()
        lam2 = engine.coverage(seeds, theta)
        if all_reduce is not None:
            all_reduce(lam1)
            all_reduce(lam2)
        r = engine.round(k, eps, ell, i, lam1, lam2)
        alphas.append(r["alpha"])
        if r["stop"]:
            break
    to_np = lambda x: np.asarray(x.cpu() if hasattr(x, "cpu") else x).astype(np.uint64)
    res = {"rounds": i + 1, "theta": r["theta"], "lambda_r1": to_np(lam1), "lambda_r2": to_np(lam2),
           "sigma_r1": r["sigma_r1"], "sigma_r2": r["sigma_r2"], "upper": r["upper"], "lower": r["lower"],
           "alpha": r["alpha"], "alpha_round": alphas}
    return np.asarray(seeds, dtype=np.int32), res
