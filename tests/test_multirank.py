"""The benchmark's multi-rank path on CPU ranks (gloo, world size 2): every rank runs its own
query with its own seed (replicas, no collective on the data path); the job's time is the
slowest rank's and its RR sets the sum over ranks. The RR sets each rank counts here come from
the oracle on a tiny workload, so the test needs no GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    from workloads import make_hypergraph, workload

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        w = workload("tiny-1k-u2to6-p005")
        off, mem = make_hypergraph(w.graph)
        g = oracle.Graph(w.graph.n, off, mem, w.query.model, w.query.uniform_threshold)
        seed = bench.rank_seed(w.query.seed, rank)
        pool = oracle.Pool(g, seed=seed, tag=0, roots=w.query.roots)
        pool.grow_theta(200 * (rank + 1))
        sets = pool.count()
        first = pool.arrays().mem[:50].tolist()
        t_local = 1.0 + rank  # stand-ins for the timed durations of the ranks
        res = bench.reduce_over_ranks(torch, dist, [t_local, 2.0 * t_local], [float(sets)], "cpu")
        gathered = [None] * world
        dist.all_gather_object(gathered, (sets, first))
        if rank == 0:
            out.put((res, gathered))
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction():
    ctx = mp.get_context("spawn")
    out = ctx.SimpleQueue()
    world = 2
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    res, gathered = out.get()
    counts = [c for c, _ in gathered]
    assert counts == [200, 400]
    # slowest rank's durations, summed RR sets
    assert res == pytest.approx([2.0, 4.0, 600.0])
    # independent queries: the two ranks' pools differ
    assert gathered[0][1] != gathered[1][1]
