#!/usr/bin/env python
"""Benchmark of HyperIM's hot path on GB300.

One step = one whole influence-maximisation query through the C ABI: load the hypergraph
(incidence store + layer profile), plan theta, then HyperIM_BRR (grow the R1/R2 RR pools round
by round, greedy max coverage on R1, coverage on R2, bounds) until the stop test passes -- or, for
workloads with a fixed theta, one pool of theta RR sets and greedy. The metric is RR sets
generated per second over the whole job; seed-selection seconds are reported beside it.

Timing: W untimed warm-up steps, then K timed steps, each bracketed by CUDA events on the stream
the library launches on; L2 is flushed (256 MiB write) before every step, outside the events.
The inputs (CSR) are resident in HBM before the timed region; the e2e figure repeats the steps
from pinned host buffers (host->device copy inside the timed call, seeds copied back).

With torchrun (N > 1) every rank runs its own query (its own seed) on its GPU: the queries are
independent problems, so there is no collective on the data path (weak scaling); rank 0 prints.
``--impl reference`` times the CPU oracle on a bounded sample of the same workload, on every host
core (one thread and one oracle graph per core, disjoint RR ids).
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import make_hypergraph, workload  # noqa: E402

DEFAULT_WORKLOAD = "zipf-2m-1m-wc"
METRIC = "RR sets/sec + seed-selection seconds at fixed eps vs plain GPU form; % HBM roofline"
UNIT = "RR sets/s"
L2_FLUSH_BYTES = 256 << 20


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def rr_algorithmic_bytes(v):
    """Algorithmic bytes of RR generation (the cost model of Thms 2-3, at 32-byte-sector
    granularity; the oracle counts the same figure independently): per pop the sectors of mu's
    layer profile (12-byte entries), per materialising pop also the sectors of v_he(mu) and, for
    every hyperedge of mu, its two offsets (8) and the sectors of its member ids -- what
    materialising A(mu) from the incidence lists reads, whatever this design reads instead --
    plus 4 bytes per output id and 8 per RR set (root draw, offset)."""
    return 32 * v["sectors"] + 8 * v["mat_he"] + 4 * v["total"] + 8 * v["count"]


def rr_design_bytes(v):
    """The bytes this design's RR kernel reads and writes by its own counters: per pop the vertex
    record (8) and one 32-byte entry per layer of A(mu); per materialising pop the hyperedge spans
    (8 + 4 per hyperedge) and the record and sum of sizes (12); the member ids gathered (4 each:
    all of mu's hyperedges in one pass, or only the id slices of the chunks that hold picks when mu
    has a chunk index) and the words read to locate those slices (4 each); per member of R its
    queue write, queue read and output write (12); per RR set its root (4)."""
    return (8 * v["pops"] + 32 * v["layers_seen"] + 12 * v["mats"] + 12 * v["mat_he"]
            + 4 * v["gathered"] + 4 * v["search_words"] + 12 * v["total"] + 4 * v["count"])


def source_hash():
    h = hashlib.sha256()
    for f in ("rr.cu", "mat.cuh", "device_math.cuh", "index.cu"):
        h.update(open(os.path.join(ROOT, "paper_2406_01911_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_ratio_for(name):
    """DRAM bytes per algorithmic byte of the RR kernel, from the committed ncu capture of one
    launch of known size (``--profile-batch``), if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"k_rr_{name}.json")
    try:
        d = json.load(open(path))
    except OSError:
        return None
    if d.get("source_hash") != source_hash():
        return None
    return d.get("dram_bytes_per_algorithmic_byte")


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        else:
            self.lines = []

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_query(H, torch, w, off, mem, seed, host_inputs=False, upper="closed", schedule="persistent",
              tune=True):
    """One whole IM query through the C ABI; returns counters of the work done. With `tune`, the
    graph takes the autotuner's RR scheduling for its degree profile (measured once per process,
    on the first query; a cache lookup afterwards)."""
    q = w.query
    g = H.Graph(w.graph.n, off, mem, q.model, q.uniform_threshold, seed=seed)
    tuning = g.autotune(roots=q.roots, strategy=q.strategy) if tune else g.tuning()
    if schedule != "persistent":
        g.set_schedule(schedule)
    r1 = g.pool(tag=0, roots=q.roots, strategy=q.strategy)
    r2 = g.pool(tag=1, roots=q.roots, strategy=q.strategy)
    if q.theta is not None:
        r1.sample(q.theta)
        seeds, res = g.select_seeds(r1, None, q.k, mode="fixed")
    else:
        seeds, res = g.select_seeds(r1, r2, q.k, mode="brr", eps=q.eps, ell=q.ell, upper=upper)
    v1, v2 = r1.view(), r2.view()
    # RR sets the query read (its last round's prefix of R1 and R2); sets generated ahead of a
    # round and never read would not count (none on the benchmark workloads)
    out = {"rr_sets": int(res["pool_r1"] + res["pool_r2"]), "rr_generated": v1["count"] + v2["count"],
           "rr_kernel_seconds": v1["rr_kernel_seconds"] + v2["rr_kernel_seconds"],
           "rr_launches": v1["rr_launches"] + v2["rr_launches"],
           "bytes": rr_algorithmic_bytes(v1) + rr_algorithmic_bytes(v2),
           "design_bytes": rr_design_bytes(v1) + rr_design_bytes(v2),
           "edges": sum(v["mat_he"] + v["gathered"] for v in (v1, v2)),
           "select_seconds": res["seconds_select"], "sample_seconds": res["seconds_sample"],
           "rounds": res["rounds"], "theta": res["theta"] or (q.theta or 0), "sigma": res["sigma_r1"],
           "sigma_r2": res["sigma_r2"], "seeds": seeds,
           "tuning": {k: tuning[k] for k in ("warp_set_limit", "early_sets_per_block")}}
    r1.close()
    r2.close()
    g.close()
    return out


def reduce_over_ranks(torch, dist, times, units, device):
    """Whole-job figures of a multi-rank run: each timed duration is the slowest rank's (max over
    ranks), each unit count the sum over ranks. Returns the reduced times followed by the sums."""
    tmax = torch.tensor(times, dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tot = torch.tensor(units, dtype=torch.float64, device=device)
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return [float(x) for x in tmax.tolist()] + [float(x) for x in tot.tolist()]


def rank_seed(base, rank):
    """Each rank's query seed: the ranks run independent queries (distinct Philox keys)."""
    return base + 1000 * rank


def bench_gpu(args):
    import torch
    import torch.distributed as dist
    import paper_2406_01911_gb300 as H

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2406_01911_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
        build.build()

    w = workload(args.workload)
    off, mem = make_hypergraph(w.graph)
    d_off = torch.as_tensor(off).cuda()
    d_mem = torch.as_tensor(mem).cuda()
    p_off = torch.as_tensor(off).pin_memory()
    p_mem = torch.as_tensor(mem).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    seed = rank_seed(w.query.seed, rank)

    def sync_all():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for i in range(args.warmup):
        run_query(H, torch, w, d_off, d_mem, seed)
    stream = torch.cuda.current_stream()
    times, stats = [], []
    launches0 = H.hyperim_kernel_launches()
    sync_all()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats.append(run_query(H, torch, w, d_off, d_mem, seed))
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        sync_all()
        t_wall = time.perf_counter() - t_wall
    launches = H.hyperim_kernel_launches() - launches0
    # end to end from pinned host buffers
    e2e_times = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = run_query(H, torch, w, p_off, p_mem, seed)
        e1.record(stream)
        e1.synchronize()
        e2e_times.append(e0.elapsed_time(e1) / 1e3)
    rr_local = sum(s["rr_sets"] for s in stats)
    t_local = sum(times)
    e2e_local = sum(e2e_times)
    if world > 1:
        t_all, e2e_all, rr_all = reduce_over_ranks(torch, dist, [t_local, e2e_local], [float(rr_local)], "cuda")
    else:
        t_all, e2e_all, rr_all = t_local, e2e_local, float(rr_local)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    peak_note = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    kbytes = sum(s["bytes"] for s in stats)
    dbytes = sum(s["design_bytes"] for s in stats)
    ksec = sum(s["rr_kernel_seconds"] for s in stats)
    klaunch = sum(s["rr_launches"] for s in stats)
    achieved = kbytes / ksec / 1e9 if ksec > 0 else 0.0
    ratio = traffic_ratio_for(args.workload)
    traffic = ratio * kbytes / max(klaunch, 1) if ratio is not None else None
    line = {
        "metric": METRIC,
        "value": rr_all / t_all,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_all / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": w.name, "description": w.description, "n": w.graph.n, "m": w.graph.m,
                   "k": w.query.k, "eps": w.query.eps, "ell": w.query.ell, "roots": w.query.roots,
                   "theta": w.query.theta or "adaptive (HyperIM_BRR)",
                   "rr_sets_per_step": rr_local / args.steps,
                   "rr_sets_generated_per_step": sum(x["rr_generated"] for x in stats) / args.steps,
                   "brr_rounds": stats[-1]["rounds"], "theta_final": stats[-1]["theta"],
                   "parallelism": f"replicas x{world} (independent queries)",
                   "rr_tuning": stats[-1]["tuning"],
                   "l2": "flushed between steps (256 MiB write), inputs resident in HBM"},
        "seed_selection_seconds": sum(s["select_seconds"] for s in stats) / args.steps,
        # incidence entries the RR generator read (hyperedge ids of materialising pops plus the
        # member ids gathered), per second of the timed region (this rank)
        "edge_traversals_per_s": sum(s["edges"] for s in stats) / t_local,
        "rr_sampling_seconds": sum(s["sample_seconds"] for s in stats) / args.steps,
        # RR generation alone (sets per second of RR-kernel time): the quantity the oracle's timed
        # sample measures (the reference arm and cpu_baseline time RR generation only)
        "rr_generation_sets_per_s": rr_local / ksec if ksec > 0 else None,
        "wall_seconds_timed_region": t_wall,
        "e2e": {"value": rr_all / e2e_all, "unit": UNIT,
                "h2d_bytes_per_step": int(off.nbytes + mem.nbytes),
                "d2h_bytes_per_step": int(4 * w.query.k)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": "k_rr (RR generation)", "achieved": achieved,
                     "peak": hbm, "peak_source": peak_note, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "algorithmic_bytes_per_launch": kbytes / max(klaunch, 1),
                     "launches": klaunch, "kernel_seconds": ksec,
                     "sm_mhz_x_seconds": None,
                     "design_bytes_per_launch": dbytes / max(klaunch, 1),
                     "design_gbs": dbytes / ksec / 1e9 if ksec > 0 else 0.0,
                     "design_frac": (dbytes / ksec / 1e9) / hbm if ksec > 0 else 0.0},
        "clocks": clk.summary(),
    }
    mhz = line["clocks"]["sm_mhz"]
    # the RR kernel's time in SM clock cycles at the median clock sampled under load
    line["roofline"]["sm_mhz_x_seconds"] = mhz * ksec if mhz else None
    if args.forward_sims > 0:
        line["forward_mc"] = forward_check(H, torch, w, d_off, d_mem, stats[-1], args.forward_sims)
    if not args.no_plain_form:
        line["plain_form"] = plain_form(H, torch, w, d_off, d_mem, seed, flush, stream, line["value"])
    if w.query.theta is None and not args.no_prefix_query:
        line["brr_prefix_upper"] = prefix_query(H, torch, w, d_off, d_mem, seed, flush, stream)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, off, mem, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def plain_form(H, torch, w, off, mem, seed, flush, stream, value, steps=2):
    """Outside the timed region: the same query with RR generation in the plain form (one launch
    per batch of as many sets as blocks fit, one set per block, instead of the persistent grid
    with its device work counter); the RR sets, seeds and theta are identical."""
    run_query(H, torch, w, off, mem, seed, schedule="plain")
    times, stats = [], []
    for i in range(steps):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats.append(run_query(H, torch, w, off, mem, seed, schedule="plain"))
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    rr = sum(s["rr_sets"] for s in stats)
    plain = rr / sum(times)
    return {"value": plain, "unit": UNIT, "ms_per_query": 1e3 * sum(times) / steps,
            "rr_kernel_seconds_per_query": sum(s["rr_kernel_seconds"] for s in stats) / steps,
            "rr_kernel_launches_per_query": sum(s["rr_launches"] for s in stats) / steps,
            "seed_selection_seconds": sum(s["select_seconds"] for s in stats) / steps,
            "persistent_over_plain": value / plain}


def prefix_query(H, torch, w, off, mem, seed, flush, stream, steps=3):
    """Outside the timed region: the same query with BRR's upper bound taken as Eq. upper_2
    (the prefix minimum) instead of the closed form of Alg. 4; fewer rounds, same guarantee."""
    run_query(H, torch, w, off, mem, seed, upper="prefix")
    times, stats = [], []
    for i in range(steps):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats.append(run_query(H, torch, w, off, mem, seed, upper="prefix"))
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    last = stats[-1]
    return {"ms_per_query": 1e3 * sum(times) / steps, "rr_sets_per_query": last["rr_sets"],
            "rr_sets_per_s": sum(s["rr_sets"] for s in stats) / sum(times),
            "brr_rounds": last["rounds"], "theta_final": last["theta"],
            "seed_selection_seconds": sum(s["select_seconds"] for s in stats) / steps,
            "sigma_rr_r2": last["sigma_r2"]}


def forward_check(H, torch, w, off, mem, last, sims):
    """Outside the timed region: forward Monte-Carlo influence (Sec. 2.2 cascade) of the last
    query's seeds on the GPU, beside the RR estimates of that query (R1: the pool greedy chose
    on, biased upward; R2: the independent pool of the lower bound)."""
    q = w.query
    g = H.Graph(w.graph.n, off, mem, q.model, q.uniform_threshold, seed=q.seed)
    torch.cuda.synchronize()
    t = time.perf_counter()
    _, mean, se = g.forward_spread(last["seeds"], sims, seed=0xF0F0 + q.seed)
    dt = time.perf_counter() - t
    g.close()
    return {"simulations": sims, "seconds": dt, "simulations_per_s": sims / dt, "sigma": mean,
            "std_err": se, "sigma_rr_r1": last["sigma"], "sigma_rr_r2": last["sigma_r2"]}


def profile_batch(args):
    """Grow four fresh pools by the same theta, one after the other; the last growth is a single
    RR-kernel launch of known size. Prints its RR sets, algorithmic bytes and its index among the
    RR-kernel launches of this process (the -s of an ncu capture filtered on k_rr)."""
    import torch
    import paper_2406_01911_gb300 as H
    from paper_2406_01911_gb300 import build
    torch.cuda.set_device(0)
    build.build()
    w = workload(args.workload)
    q = w.query
    off, mem = make_hypergraph(w.graph)
    g = H.Graph(w.graph.n, torch.as_tensor(off).cuda(), torch.as_tensor(mem).cuda(), q.model,
                q.uniform_threshold, seed=q.seed)
    before = 0
    for i in range(4):
        p = g.pool(tag=10 + i, roots=q.roots, strategy=q.strategy)
        p.sample(args.profile_batch)
        v = p.view()
        if i == 3:
            print(json.dumps({"workload": w.name, "theta": args.profile_batch, "rr_sets": v["count"],
                              "k_rr_launch_index": before, "k_rr_launches": v["rr_launches"],
                              "algorithmic_bytes": rr_algorithmic_bytes(v),
                              "kernel_seconds": v["rr_kernel_seconds"], "source_hash": source_hash()}),
                  flush=True)
        before += v["rr_launches"]
        p.close()
    torch.cuda.synchronize()


def oracle_graph(w, off, mem):
    """The CPU oracle's graph of the workload (built once; its build is never timed)."""
    import oracle as O
    return O.Graph(w.graph.n, off, mem, w.query.model, w.query.uniform_threshold)


def oracle_rate(w, og, seconds, seed, tag=0):
    """RR sets per second of the CPU oracle on the same graph: grows a pool of the workload's root
    mode set by set until `seconds` have passed (graph build excluded)."""
    import oracle as O
    q = w.query
    pool = O.Pool(og, seed=seed, tag=tag, roots=q.roots, strategy=q.strategy)
    t0 = time.perf_counter()
    theta = 1
    while True:
        pool.grow_theta(theta)
        el = time.perf_counter() - t0
        if el >= seconds:
            break
        theta += max(1, pool.count() // 8)
    return pool.count(), el


def oracle_rate_threads(w, og, seconds, seed, threads, tag=0):
    """The oracle driven by `threads` host threads over disjoint RR ids of one pool (one oracle
    graph, one worker view of it per thread; the ctypes calls release the GIL). The (stratum, j)
    ids of a stratified allocation are interleaved in proportion to the strata, so any prefix of
    the work list has the pool's mix. Returns (sets done, wall seconds)."""
    import threading
    import oracle
    q = w.query
    workers = oracle.Workers(og, threads)
    n_s = og.allocate(q.roots, 1 << 16)
    work = sorted(((j + 0.5) / int(c), s, j) for s, c in enumerate(n_s) if c for j in range(int(c)))
    lock = threading.Lock()
    state = {"next": 0, "done": 0}
    t0 = time.perf_counter()

    def run(t):
        while time.perf_counter() - t0 < seconds:
            with lock:
                i = state["next"]
                state["next"] += 1
            if i >= len(work):
                return
            _, s, j = work[i]
            workers.rr_set(t, seed, tag, q.roots, s, j, strategy=q.strategy)
            with lock:
                state["done"] += 1

    ts = [threading.Thread(target=run, args=(t,)) for t in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    el = time.perf_counter() - t0
    workers.close()
    return state["done"], el


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(w, off, mem, seconds):
    """The oracle on the host: every core (the baseline) and one core (beside it)."""
    cores = host_cores()
    og = oracle_graph(w, off, mem)
    count, el = oracle_rate_threads(w, og, seconds, w.query.seed, cores)
    c1, e1 = oracle_rate(w, og, seconds, w.query.seed)
    return {"value": count / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{count} RR sets of one pool (tag 0, {w.query.roots} roots, ids interleaved "
                      f"across strata) on the same graph, {el:.1f} s of oracle work on {cores} "
                      "threads, one worker view of the oracle graph per thread; graph build excluded",
            "single_core": {"value": c1 / e1, "cores": 1,
                            "sample": f"first {c1} RR sets of pool tag 0, {e1:.1f} s on one thread"}}


def bench_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.workload)
    off, mem = make_hypergraph(w.graph)
    per_step = args.reference_seconds
    cores = host_cores()
    t_build = time.perf_counter()
    og = oracle_graph(w, off, mem)
    t_build = time.perf_counter() - t_build
    for i in range(args.warmup):
        oracle_rate_threads(w, og, min(per_step / 4, 2.0), w.query.seed + 7 + i, cores, tag=3)
    counts, times = [], []
    for i in range(args.steps):
        c, el = oracle_rate_threads(w, og, per_step, w.query.seed + 100 + i, cores)
        counts.append(c)
        times.append(el)
    value = sum(counts) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": w.name, "description": w.description, "n": w.graph.n, "m": w.graph.m,
                   "k": w.query.k, "eps": w.query.eps, "roots": w.query.roots},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} steps of ~{per_step:.0f} s each: "
                                   f"RR sets of one pool per step ({w.query.roots} roots, a new "
                                   f"seed each step) on the same graph, {cores} threads with one "
                                   "worker view of the oracle graph each, graph build excluded"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        # the oracle's graph build (incidence lists and layer profile, one thread), outside the steps
        "oracle_graph_build_seconds": t_build,
    }
    print(json.dumps(line), flush=True)


def _sequential(H, torch, loaded, queries, schedule):
    """Each query alone on fresh pools, one after the other (wall seconds, results)."""
    out = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for gi, k, eps in queries:
        g = loaded[gi]
        g.set_schedule(schedule)
        r1, r2 = g.pool(tag=0, roots="stratified"), g.pool(tag=1, roots="stratified")
        seeds, res = g.select_seeds(r1, r2, k, mode="brr", eps=eps, ell=1.0)
        out.append((time.perf_counter() - t0, seeds, res, r1.view()["count"] + r2.view()["count"]))
        r1.close()
        r2.close()
    torch.cuda.synchronize()
    for g in loaded:
        g.set_schedule("persistent")
    return time.perf_counter() - t0, out


def _served(H, torch, loaded, queries, workers, budget, arrivals=None):
    """The same queries through the server (continuous batching, shared pools); submitted all at
    once, or at their arrival times (seconds from the start) when given."""
    srv = H.Server(workers=workers, hbm_budget_bytes=budget)
    ids = [srv.add_graph(g) for g in loaded]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tickets = []
    for i, (gi, k, eps) in enumerate(queries):
        if arrivals is not None:
            delay = arrivals[i] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
        tickets.append(srv.submit(ids[gi], k, eps))
    res = [srv.wait(t) for t in tickets]
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    return wall, res, st


def _batch(H, torch, loaded, queries):
    """All queries in one hyperim_select_seeds_batch call on fresh pools (one R1/R2 pair per graph,
    shared by its queries): per BRR round one RR launch over every graph and one greedy launch."""
    pools = {}
    for gi, _, _ in queries:
        if gi not in pools:
            g = loaded[gi]
            pools[gi] = (g.pool(tag=0, roots="stratified"), g.pool(tag=1, roots="stratified"))
    batch = [(loaded[gi], pools[gi][0], pools[gi][1], k, eps, 1.0) for gi, k, eps in queries]
    launches = H.hyperim_kernel_launches()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = H.hyperim_select_seeds_batch(batch)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = H.hyperim_kernel_launches() - launches
    views = [p.view() for pair in pools.values() for p in pair]
    stat = {"rounds": max(res["rounds"] for _, res in out), "kernel_launches": launches,
            "rr_launches": max(v["rr_launches"] for v in views),
            "rr_sets_generated": sum(v["count"] for v in views),
            "rr_kernel_seconds": sum(v["rr_kernel_seconds"] for v in views)}
    stat["rr_sets_per_s"] = stat["rr_sets_generated"] / wall
    for pair in pools.values():
        for p in pair:
            p.close()
    return wall, out, stat


def _same_seeds(a, b):
    return all(x.tolist() == y.tolist() for x, y in zip(a, b))


def bench_batched(args):
    """The batched configuration: 64 hypergraphs of uneven size (n log-uniform in [1e3, 2e5],
    Zipf(2.1) sizes in [2, 300]), each queried with k in {10, 50, 100} at eps = 0.1 (weighted
    cascade, stratified roots), resident in HBM. Four forms, same GPU, same queries, identical
    seeds: the plain form (one query at a time, fresh pools, RR sets one launch per batch of one
    set per block), one query at a time with the persistent RR kernel, the server (all 192
    queries submitted at once to `--workers` workers; queries on one graph share its pools), and
    the batch (all 192 in one hyperim_select_seeds_batch call: per BRR round one RR launch over
    every graph's pools and one greedy launch over every query; the line's value)."""
    import torch
    import paper_2406_01911_gb300 as H
    from workloads import batch_workload
    specs = batch_workload()
    loaded = []
    for sp in specs:
        off, mem = make_hypergraph(sp)
        loaded.append(H.Graph(sp.n, torch.as_tensor(off).cuda(), torch.as_tensor(mem).cuda(), "wc", 0, seed=1))
    queries = [(gi, k, 0.1) for gi in range(len(specs)) for k in (10, 50, 100)]
    _sequential(H, torch, loaded, queries[:6], "persistent")  # warm-up
    t_plain, plain = _sequential(H, torch, loaded, queries, "plain")
    t_seq, seq = _sequential(H, torch, loaded, queries, "persistent")
    t_srv, srv, st = _served(H, torch, loaded, queries, args.workers, int(args.budget_gb * 2**30))
    _batch(H, torch, loaded, queries)  # warm-up: the first call pays for lazy setup
    t_bat, bat, bstat = _batch(H, torch, loaded, queries)
    same = _same_seeds([x[1] for x in plain], [x[1] for x in seq]) and \
        _same_seeds([x[1] for x in seq], [x[0] for x in srv]) and \
        _same_seeds([x[1] for x in seq], [x[0] for x in bat])
    sets_fresh = sum(x[3] for x in seq)
    line = {"metric": "batched IM queries per second (64 graphs x k in {10, 50, 100}, eps = 0.1)",
            "value": len(queries) / t_bat, "unit": "queries/s", "n_gpus": 1, "higher_is_better": True,
            "config": {"workload": "batched-64-graphs", "graphs": len(specs), "queries": len(queries),
                       "workers": args.workers, "model": "wc", "roots": "stratified"},
            "batch": dict(bstat, wall_seconds=t_bat, queries_per_s=len(queries) / t_bat),
            "served": {"wall_seconds": t_srv, "queries_per_s": len(queries) / t_srv,
                       "rr_sets_generated": st["rr_sets_generated"],
                       "rr_sets_per_s": st["rr_sets_generated"] / t_srv,
                       "p50_latency_seconds": st["p50_latency_seconds"],
                       "p99_latency_seconds": st["p99_latency_seconds"], "max_running": st["max_running"]},
            "sequential_persistent": {"wall_seconds": t_seq, "queries_per_s": len(queries) / t_seq,
                                      "rr_sets": sets_fresh, "rr_sets_per_s": sets_fresh / t_seq},
            "plain_form": {"wall_seconds": t_plain, "queries_per_s": len(queries) / t_plain,
                           "rr_sets_per_s": sets_fresh / t_plain},
            "served_over_plain": t_plain / t_srv, "served_over_sequential": t_seq / t_srv,
            "batch_over_plain": t_plain / t_bat, "batch_over_served": t_srv / t_bat,
            "identical_seeds": same, "failed": st["failed"]}
    print(json.dumps(line), flush=True)
    for g in loaded:
        g.close()


def bench_served(args):
    """The served configuration: 16 resident hypergraphs (n log-uniform in [1e5, 5e6],
    m = min(0.6 n, 3e6), Zipf(2.0) sizes in [2, 500]) and a Poisson stream of queries (mean 200
    per second; k uniform in [10, 200]; eps in {0.05, 0.1, 0.2}); the first `--queries` of the
    stream are submitted at their arrival times. Latency is submit to completion. The same stream
    is served again by one worker (one query at a time, same persistent kernels and shared pools,
    latencies measured alike). The plain form
    (one query at a time on fresh pools, RR sets one launch per batch) runs the first
    `--plain-queries` of them; its latencies follow from its measured durations under the same
    arrivals with one query in service at a time (FIFO)."""
    import torch
    import paper_2406_01911_gb300 as H
    from workloads import serving_queries, serving_workload
    specs = serving_workload()
    loaded = []
    t_load = time.perf_counter()
    for sp in specs:
        off, mem = make_hypergraph(sp)
        loaded.append(H.Graph(sp.n, torch.as_tensor(off).cuda(), torch.as_tensor(mem).cuda(), "wc", 0, seed=1))
    torch.cuda.synchronize()
    t_load = time.perf_counter() - t_load
    stream = serving_queries()[:args.queries]
    queries = [(q.graph, q.k, q.eps) for q in stream]
    arrivals = [q.arrival for q in stream]
    t_srv, srv, st = _served(H, torch, loaded, queries, args.workers, int(args.budget_gb * 2**30), arrivals)
    t_one, one, st1 = _served(H, torch, loaded, queries, 1, int(args.budget_gb * 2**30), arrivals)
    npl = min(args.plain_queries, len(queries))
    t_plain, plain = _sequential(H, torch, loaded, queries[:npl], "plain")
    done, prev, lat = 0.0, 0.0, []
    for i, (t_end, *_rest) in enumerate(plain):
        dur = t_end - prev
        prev = t_end
        done = max(done, arrivals[i]) + dur
        lat.append(done - arrivals[i])
    lat.sort()
    pct = lambda q: lat[max(0, min(len(lat), math.ceil(q * len(lat))) - 1)]
    same = _same_seeds([x[1] for x in plain], [x[0] for x in srv[:npl]])
    line = {"metric": "served IM queries: throughput and p50/p99 latency", "value": st["queries_per_second"],
            "unit": "queries/s", "n_gpus": 1, "higher_is_better": True,
            "config": {"workload": "served-16-graphs-poisson-200qps", "graphs": len(specs),
                       "queries": len(queries), "workers": args.workers,
                       "hbm_budget_gb": args.budget_gb, "load_seconds": t_load},
            "served": {"queries_per_s": st["queries_per_second"], "p50_latency_seconds": st["p50_latency_seconds"],
                       "p99_latency_seconds": st["p99_latency_seconds"], "mean_latency_seconds": st["mean_latency_seconds"],
                       "span_seconds": st["span_seconds"], "rr_sets_generated": st["rr_sets_generated"],
                       "evictions": st["evictions"], "max_running": st["max_running"], "failed": st["failed"],
                       "device_gb": st["device_bytes"] / 2**30},
            "one_worker": {"queries_per_s": st1["queries_per_second"],
                           "p50_latency_seconds": st1["p50_latency_seconds"],
                           "p99_latency_seconds": st1["p99_latency_seconds"],
                           "mean_latency_seconds": st1["mean_latency_seconds"],
                           "rr_sets_generated": st1["rr_sets_generated"], "failed": st1["failed"]},
            "plain_form": {"queries": npl, "busy_seconds": t_plain, "queries_per_s": npl / t_plain,
                           "p50_latency_seconds": pct(0.5), "p99_latency_seconds": pct(0.99),
                           "latency": "from the measured durations, FIFO with one query in service"},
            "identical_seeds": same and _same_seeds([x[0] for x in srv], [x[0] for x in one])}
    print(json.dumps(line), flush=True)
    for g in loaded:
        g.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--forward-sims", type=int, default=256,
                    help="forward Monte-Carlo simulations of the last query's seeds (0: skip)")
    ap.add_argument("--reference-seconds", type=float, default=5.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain-form", action="store_true",
                    help="skip the plain-schedule comparison query (outside the timed region)")
    ap.add_argument("--no-prefix-query", action="store_true",
                    help="skip the extra measurement of BRR with the Eq. upper_2 bound")
    ap.add_argument("--profile-batch", type=int, default=0,
                    help="profiling aid: one RR-kernel launch growing a fresh pool by this theta")
    ap.add_argument("--batched", action="store_true",
                    help="the 64-graph batched configuration (its own JSON line) instead of the bench")
    ap.add_argument("--served", action="store_true",
                    help="the 16-graph served configuration (its own JSON line) instead of the bench")
    ap.add_argument("--workers", type=int, default=8, help="server workers (--batched, --served)")
    ap.add_argument("--budget-gb", type=float, default=0.0, help="server HBM budget, GiB (0: none)")
    ap.add_argument("--queries", type=int, default=200, help="queries of the stream (--served)")
    ap.add_argument("--plain-queries", type=int, default=24, help="of them run in the plain form (--served)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.profile_batch:
        profile_batch(args)
    elif args.batched and args.impl == "ours":
        bench_batched(args)
    elif args.served and args.impl == "ours":
        bench_served(args)
    elif args.impl == "reference":
        bench_reference(args)
    else:
        bench_gpu(args)


if __name__ == "__main__":
    main()
