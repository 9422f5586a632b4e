"""Multi-rank HyperIM_BRR (paper_2406_01911_gb300.sharded): the RR pools split over ranks by
(stratum, j) ranges, one all-reduce of the integer score vector per greedy round, the coverages of
R1 and R2 all-reduced per BRR round.

On the CPU: two `gloo` ranks run the product's driver (`sharded_brr`) with a test engine whose
shards are the CPU oracle's RR sets (j = rank mod 2 of the oracle's own pools) and whose greedy
state is a plain numpy restatement of Algorithm 1 on them; the result must equal the oracle's
single-process HyperIM_BRR (rounds, theta, seeds, coverages, bounds). A failing rank (an
exception before its first collective) is reported by the other rank's process-group timeout,
not by a hang. On the GPU (marked gpu): one process holds both shards of each pool through the C
ABI (`GpuShards`), and the result equals hyperim_select_seeds in BRR mode.
"""
import math
import os
import socket

import numpy as np
import pytest

from tests import bruteforce as bf

NSTRATA = 16


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def graph_inputs(seed=3, n=160, m=140):
    rng = np.random.default_rng(seed)
    hes = [[int(x) for x in rng.integers(0, n, size=int(rng.integers(2, 6)))] for _ in range(m)]
    return n, hes


class OracleShards:
    """Test engine: this rank's shards of R1 and R2 as the CPU oracle builds them, and Algorithm 1
    restated in numpy over the shard (weights floor(|V_s| 2^32 / n_s), ties to the lowest id)."""

    def __init__(self, O, og, seed, rank, world, roots="stratified"):
        import torch
        self.torch, self.O, self.og = torch, O, og
        self.rank, self.world, self.roots = rank, world, roots
        self.pools = {t: O.Pool(og, seed=seed, tag=t, roots=roots) for t in (0, 1)}

    def plan(self, k, eps, ell):
        return self.O.plan_theta(self.og.n, k, eps, ell)

    def grow(self, theta):
        for p in self.pools.values():
            p.grow_theta(theta)

    def _shard(self, tag, theta):
        ns = self.og.allocate(self.roots, theta)
        a = self.pools[tag].arrays()
        keep = [i for i in range(len(a.off) - 1)
                if a.j[i] < ns[a.stratum[i]] and a.j[i] % self.world == self.rank]
        return [a.mem[a.off[i]:a.off[i + 1]] for i in keep], [int(a.stratum[i]) for i in keep], ns

    def greedy_begin(self, theta):
        self.sets, self.strata, ns = self._shard(0, theta)
        self.W = [((self.og.stratum_size(s) << 32) // int(ns[s])) if ns[s] else 0 for s in range(NSTRATA)]
        if self.roots == "plain":
            self.W = [1] * NSTRATA
        self.score = np.zeros(self.og.n, np.int64)
        for R, s in zip(self.sets, self.strata):
            self.score[R] += self.W[s]
        self.covered = np.zeros(len(self.sets), bool)
        self.picked = np.zeros(self.og.n, bool)
        self.lam = np.zeros(NSTRATA, np.int64)

    def local_scores(self):
        return self.torch.as_tensor(self.score.copy())

    def pick(self, total):
        t = total.numpy().copy()
        t[self.picked] = -1
        v = int(np.argmax(t))  # first maximum: the lowest id on ties
        self.picked[v] = True
        for r, (R, s) in enumerate(zip(self.sets, self.strata)):
            if not self.covered[r] and v in R:
                self.covered[r] = True
                self.lam[s] += 1
                self.score[R] -= self.W[s]
        return v

    def greedy_end(self):
        return self.torch.as_tensor(self.lam.copy())

    def coverage(self, seeds, theta):
        sets, strata, _ = self._shard(1, theta)
        lam = np.zeros(NSTRATA, np.int64)
        S = set(seeds)
        for R, s in zip(sets, strata):
            if S.intersection(R.tolist()):
                lam[s] += 1
        return self.torch.as_tensor(lam)

    def round(self, k, eps, ell, i, lam1, lam2):
        plan = self.plan(k, eps, ell)
        theta = int(plan["theta0"]) << i
        ns = self.og.allocate(self.roots, theta)
        N = int(ns.sum())
        n = self.og.n
        vs = [self.og.stratum_size(s) if self.roots == "stratified" else n for s in range(NSTRATA)]
        est = lambda lam: sum((vs[s] / int(ns[s])) * int(lam[s]) for s in range(NSTRATA) if ns[s])
        s1, s2 = est(lam1.numpy()), est(lam2.numpy())
        up = self.O.upper_bound(s1 * N / n, k, n, N)
        lo = self.O.lower_bound(s2 * N / n, plan["delta"], n, N)
        return {"theta": theta, "sigma_r1": s1, "sigma_r2": s2, "upper": up, "lower": lo, "alpha": lo / up,
                "stop": int(lo / up >= 1 - math.exp(-1) - eps or i >= plan["i_max"])}


def _rank_main(rank, world, port, out_dir, fail_rank):
    import datetime

    import torch
    import torch.distributed as dist

    import oracle as O
    from paper_2406_01911_gb300.sharded import sharded_brr

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    try:
        if rank == fail_rank:
            raise RuntimeError("this rank fails before its first collective")
        n, hes = graph_inputs()
        off, mem = bf.to_csr(hes)
        og = O.Graph(n, off, mem, "uniform_pair", 858993459)
        eng = OracleShards(O, og, seed=5, rank=rank, world=world)
        seeds, res = sharded_brr(eng, k=4, eps=0.3, ell=1.0, all_reduce=lambda t: dist.all_reduce(t))
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), seeds=seeds, lam1=res["lambda_r1"], lam2=res["lambda_r2"],
                 scal=np.array([res["rounds"], res["theta"], res["sigma_r1"], res["sigma_r2"], res["upper"],
                                res["lower"]], dtype=np.float64))
    except Exception as e:  # reported through a file: the parent checks who failed and why
        with open(os.path.join(out_dir, f"rank{rank}.err"), "w") as f:
            f.write(f"{type(e).__name__}: {e}")
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _spawn(world, fail_rank, tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(world, free_port(), str(tmp_path), fail_rank), nprocs=world,
                       start_method="spawn", join=True)


def test_two_gloo_ranks_equal_the_oracle(oracle, tmp_path):
    _spawn(2, -1, tmp_path)
    errs = [p for p in os.listdir(tmp_path) if p.endswith(".err")]
    assert not errs, [open(tmp_path / p).read() for p in errs]
    n, hes = graph_inputs()
    off, mem = bf.to_csr(hes)
    og = oracle.Graph(n, off, mem, "uniform_pair", 858993459)
    seeds, res = oracle.brr(og, 5, 4, 0.3, 1.0, roots="stratified")
    for rank in range(2):
        d = np.load(tmp_path / f"rank{rank}.npz")
        assert d["seeds"].tolist() == seeds.tolist()
        assert d["lam1"].tolist() == res["lambda_r1"].tolist()
        assert d["lam2"].tolist() == res["lambda_r2"].tolist()
        rounds, theta, s1, s2, up, lo = d["scal"].tolist()
        assert int(rounds) == res["rounds"] and int(theta) == res["theta"]
        for a, b in ((s1, res["sigma_r1"]), (s2, res["sigma_r2"]), (up, res["upper"]), (lo, res["lower"])):
            assert a == pytest.approx(b, rel=1e-12)


def test_a_failing_rank_ends_the_other_by_timeout(tmp_path):
    # rank 1 raises before any collective; rank 0's first all-reduce ends with an error (the
    # process group's timeout), so both ranks return and report, nothing hangs
    _spawn(2, 1, tmp_path)
    assert "fails before" in open(tmp_path / "rank1.err").read()
    assert os.path.exists(tmp_path / "rank0.err")


@pytest.mark.gpu
def test_gpu_shards_equal_the_single_pool_query():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_01911_gb300 import build
    build.build()
    import paper_2406_01911_gb300 as H
    from paper_2406_01911_gb300.sharded import GpuShards, sharded_brr
    from workloads import make_hypergraph, workload
    w = workload("zipf-100k-50k-paper")
    q = w.query
    off, mem = make_hypergraph(w.graph)
    g = H.Graph(w.graph.n, off, mem, q.model, q.uniform_threshold, seed=q.seed)
    for world in (2, 3):
        eng = GpuShards(g, ranks=range(world), world=world, roots=q.roots)
        seeds, res = sharded_brr(eng, q.k, q.eps, q.ell)
        r1, r2 = g.pool(tag=0, roots=q.roots), g.pool(tag=1, roots=q.roots)
        s_ref, ref = g.select_seeds(r1, r2, q.k, mode="brr", eps=q.eps, ell=q.ell)
        assert seeds.tolist() == s_ref.tolist()
        assert res["rounds"] == ref["rounds"] and res["theta"] == ref["theta"]
        assert res["lambda_r1"].tolist() == ref["lambda_r1"].tolist()
        assert res["lambda_r2"].tolist() == ref["lambda_r2"].tolist()
        for key in ("sigma_r1", "sigma_r2", "upper", "lower", "alpha"):
            assert res[key] == pytest.approx(ref[key], rel=1e-12)
        # the shards together hold exactly the single pool's sets
        v = sum(p.view()["count"] for p in eng.r1)
        assert v == r1.view()["count"] or ref["theta"] < r1.view()["count"]
        eng.close()
        r1.close()
        r2.close()
    g.close()
