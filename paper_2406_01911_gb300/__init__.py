"""HyperIM on GB300: Python binding of the C ABI in include/hyperim.h.

Argument marshalling only: every step of the hot path (incidence store, layer profile, RR-set
generation, compaction, greedy max coverage, coverage of a seed set) runs in the CUDA kernels of
``libhyperim.so``. Module-level functions carry the C names (``hyperim_load``,
``hyperim_plan_theta``, ``hyperim_sample_rr``, ``hyperim_select_seeds``, ``hyperim_spread``,
...); ``Graph`` and ``Pool`` wrap the handles. PyTorch only supplies the CUDA stream (and, when
the caller passes CUDA tensors, the device pointers of the input CSR).

There is no CPU fallback: importing works anywhere, but the first call raises if the compiled
library is missing or no GPU is present.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhyperim.so")

NSTRATA = 16
P_ONE = 1 << 32
NOALLOC_MAX_N = 1 << 24
MODELS = {"uniform_pair": 0, "wc": 1, "paper_layer": 2}
ROOTS = {"plain": 0, "stratified": 1}
SCHEDULES = {"persistent": 0, "plain": 1}
STRATEGIES = {"paper": 0, "binomial_only": 1, "lt": 2}
SELECT_MODES = {"fixed": 0, "brr": 1}
STATUS = {0: "HYPERIM_OK", -1: "HYPERIM_EINVAL", -2: "HYPERIM_ENOMEM", -3: "HYPERIM_EOVERFLOW",
          -4: "HYPERIM_ETIMEDOUT", -5: "HYPERIM_ECUDA", -6: "HYPERIM_ESTATE"}


class HyperIMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


# the caller's device allocator (hyperim_load_args.dev_alloc / dev_free)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class LoadArgs(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("he_off", C.c_void_p), ("he_mem", C.c_void_p),
                ("ptrs_on_device", C.c_int32), ("model", C.c_int32),
                ("uniform_threshold", C.c_uint64), ("seed", C.c_uint64),
                ("cuda_stream", C.c_void_p), ("hbm_budget_bytes", C.c_size_t),
                ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_ctx", C.c_void_p)]


class GraphStats(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("nnz", C.c_int64),
                ("profile_entries", C.c_int64), ("max_layers", C.c_int32), ("max_dh", C.c_int32),
                ("max_deg", C.c_int64), ("stratum_size", C.c_int64 * NSTRATA),
                ("theta_lstar", C.c_double), ("device_bytes", C.c_size_t),
                ("index_vertices", C.c_int32), ("index_entries", C.c_int64)]


class ThetaPlan(C.Structure):
    _fields_ = [("delta", C.c_double), ("ln_binom", C.c_double), ("theta_max", C.c_double),
                ("theta_max_ceil", C.c_uint64), ("theta0", C.c_uint64), ("i_max", C.c_int32)]


class PoolView(C.Structure):
    _fields_ = [("count", C.c_int64), ("total", C.c_int64), ("rr_off", C.c_void_p),
                ("rr_mem", C.c_void_p), ("rr_stratum", C.c_void_p), ("rr_j", C.c_void_p),
                ("n_s", C.c_uint64 * NSTRATA), ("pool_tag", C.c_uint32), ("root_mode", C.c_int32),
                ("strategy", C.c_int32), ("pops", C.c_uint64), ("layers_seen", C.c_uint64),
                ("draws", C.c_uint64), ("mats", C.c_uint64), ("mat_he", C.c_uint64),
                ("mat_members", C.c_uint64), ("selected", C.c_uint64),
                ("gathered", C.c_uint64), ("search_words", C.c_uint64),
                ("rr_launches", C.c_uint64), ("rr_kernel_seconds", C.c_double),
                ("sectors", C.c_uint64)]


class Tuning(C.Structure):
    _fields_ = [("warp_set_limit", C.c_int32), ("early_sets_per_block", C.c_int32),
                ("arena_entries_per_set", C.c_int32)]


class AutotuneResult(C.Structure):
    _fields_ = [("chosen", Tuning), ("from_cache", C.c_int32), ("candidates", C.c_int32),
                ("warp_set_limit", C.c_int32 * 8), ("seconds", C.c_double * 8),
                ("profile_key", C.c_uint64)]


class SelectOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("eps", C.c_double), ("ell", C.c_double),
                ("theta_cap", C.c_uint64), ("root_mode", C.c_int32), ("strategy", C.c_int32),
                ("upper_mode", C.c_int32)]


class SelectResult(C.Structure):
    _fields_ = [("rounds", C.c_int32), ("theta", C.c_uint64), ("pool_r1", C.c_uint64),
                ("pool_r2", C.c_uint64), ("lambda_r1", C.c_uint64 * NSTRATA),
                ("lambda_r2", C.c_uint64 * NSTRATA), ("sigma_r1", C.c_double),
                ("sigma_r2", C.c_double), ("upper", C.c_double), ("lower", C.c_double),
                ("alpha", C.c_double), ("alpha_round", C.c_double * 64),
                ("seconds_sample", C.c_double), ("seconds_select", C.c_double)]


class BatchQuery(C.Structure):
    _fields_ = [("graph", C.c_void_p), ("r1", C.c_void_p), ("r2", C.c_void_p), ("k", C.c_int32),
                ("eps", C.c_double), ("ell", C.c_double), ("seeds_host", C.c_void_p),
                ("result", C.POINTER(SelectResult))]


class BrrRound(C.Structure):
    _fields_ = [("theta", C.c_uint64), ("sigma_r1", C.c_double), ("sigma_r2", C.c_double), ("upper", C.c_double),
                ("lower", C.c_double), ("alpha", C.c_double), ("stop", C.c_int32)]


class ServerArgs(C.Structure):
    _fields_ = [("workers", C.c_int32), ("hbm_budget_bytes", C.c_size_t)]


class Query(C.Structure):
    _fields_ = [("graph_id", C.c_int32), ("k", C.c_int32), ("eps", C.c_double), ("ell", C.c_double),
                ("upper_mode", C.c_int32)]


class QueryResult(C.Structure):
    _fields_ = [("status", C.c_int), ("k", C.c_int32), ("result", SelectResult),
                ("queued_seconds", C.c_double), ("run_seconds", C.c_double),
                ("latency_seconds", C.c_double), ("worker", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("evictions", C.c_uint64), ("p50_latency_seconds", C.c_double),
                ("p99_latency_seconds", C.c_double), ("mean_latency_seconds", C.c_double),
                ("max_latency_seconds", C.c_double), ("span_seconds", C.c_double),
                ("queries_per_second", C.c_double), ("rr_sets_generated", C.c_uint64),
                ("device_bytes", C.c_size_t), ("max_running", C.c_int32)]


_lib = None
_vp = C.c_void_p
_SIGNATURES = {
    "hyperim_load": (C.c_int, [C.POINTER(LoadArgs), C.POINTER(_vp)]),
    "hyperim_graph_free": (None, [_vp]),
    "hyperim_graph_stats": (C.c_int, [_vp, C.POINTER(GraphStats)]),
    "hyperim_graph_profile": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "hyperim_graph_set_schedule": (C.c_int, [_vp, C.c_int32]),
    "hyperim_graph_set_wait_limit": (C.c_int, [_vp, C.c_uint32]),
    "hyperim_graph_set_tuning": (C.c_int, [_vp, C.POINTER(Tuning)]),
    "hyperim_graph_get_tuning": (C.c_int, [_vp, C.POINTER(Tuning)]),
    "hyperim_graph_autotune": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(AutotuneResult)]),
    "hyperim_graph_share": (C.c_int, [_vp, _vp, C.POINTER(_vp)]),
    "hyperim_server_create": (C.c_int, [C.POINTER(ServerArgs), C.POINTER(_vp)]),
    "hyperim_server_add_graph": (C.c_int, [_vp, _vp, C.POINTER(C.c_int32)]),
    "hyperim_server_submit": (C.c_int, [_vp, C.POINTER(Query), C.POINTER(C.c_uint64)]),
    "hyperim_server_wait": (C.c_int, [_vp, C.c_uint64, _vp, C.POINTER(QueryResult)]),
    "hyperim_server_stats": (C.c_int, [_vp, C.POINTER(ServerStats)]),
    "hyperim_server_free": (None, [_vp]),
    "hyperim_graph_chunk_index": (C.c_int, [_vp, C.c_int32, C.POINTER(C.c_int32), _vp, C.c_int64,
                                            C.POINTER(C.c_int64)]),
    "hyperim_forward_spread": (C.c_int, [_vp, _vp, C.c_int32, C.c_uint64, C.c_uint64, _vp,
                                         C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "hyperim_plan_theta": (C.c_int, [_vp, C.c_int32, C.c_double, C.c_double, C.POINTER(ThetaPlan)]),
    "hyperim_sample_rr": (C.c_int, [_vp, C.c_uint32, C.c_uint64, C.c_int32, C.c_int32,
                                    C.POINTER(_vp)]),
    "hyperim_pool_free": (None, [_vp]),
    "hyperim_sample_rr_shard": (C.c_int, [_vp, C.c_uint32, C.c_uint64, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                          C.POINTER(_vp)]),
    "hyperim_greedy_begin": (C.c_int, [_vp, _vp, C.c_uint64, C.POINTER(_vp)]),
    "hyperim_greedy_scores": (C.c_int, [_vp, _vp]),
    "hyperim_greedy_pick": (C.c_int, [_vp, _vp, C.POINTER(C.c_int32)]),
    "hyperim_greedy_end": (C.c_int, [_vp, _vp]),
    "hyperim_coverage_view": (C.c_int, [_vp, _vp, C.c_uint64, _vp, C.c_int32, _vp]),
    "hyperim_brr_round": (C.c_int, [_vp, C.c_int32, C.c_double, C.c_double, C.c_int32, C.c_int32, _vp, _vp,
                                    C.POINTER(BrrRound)]),
    "hyperim_pool_view": (C.c_int, [_vp, C.POINTER(PoolView)]),
    "hyperim_pool_copy": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "hyperim_select_seeds": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.POINTER(SelectOpts), _vp,
                                       C.POINTER(SelectResult)]),
    "hyperim_select_seeds_batch": (C.c_int, [C.POINTER(BatchQuery), C.c_int32]),
    "hyperim_spread": (C.c_int, [_vp, _vp, C.c_int32, _vp, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double)]),
    "hyperim_coverage_noalloc": (C.c_int, [C.c_int32, _vp, _vp, _vp, C.c_int64, _vp, C.c_int32, _vp,
                                           _vp]),
    "hyperim_kernel_launches": (C.c_uint64, []),
    "hyperim_last_error": (C.c_char_p, []),
}


def lib():
    """The loaded libhyperim.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with paper_2406_01911_gb300.build.build() "
                "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGNATURES)


def _check(status: int):
    if status != 0:
        raise HyperIMError(status, lib().hyperim_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def current_stream():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("HyperIM needs a CUDA device (no CPU fallback)")
    return torch.cuda.current_stream().cuda_stream


# ------------------------------------------------------------------------------------------------
# C-named entry points (thin wrappers)
# ------------------------------------------------------------------------------------------------
class DeviceAllocator:
    """A device allocator handed to hyperim_load: ``alloc(nbytes, stream) -> int`` (a device
    pointer, 0 on failure) and ``free(ptr, stream)``, called by the library for every device
    buffer of the graph, its shares and its pools (stream: the cudaStream_t of the calling
    handle, as an int). The C callbacks are kept alive for the life of the process, since pools
    and shares may outlive the Graph object."""

    _alive = []

    def __init__(self, alloc, free):
        self.allocs = 0
        self.frees = 0

        def _a(nbytes, stream, ctx):
            self.allocs += 1
            try:
                return int(alloc(int(nbytes), int(stream or 0))) or None
            except Exception:
                return None

        def _f(ptr, stream, ctx):
            self.frees += 1
            free(int(ptr), int(stream or 0))

        self.c_alloc = ALLOC_FN(_a)
        self.c_free = FREE_FN(_f)
        DeviceAllocator._alive.append(self)


def torch_caching_allocator(device=None):
    """A DeviceAllocator backed by PyTorch's CUDA caching allocator."""
    import torch
    dev = torch.cuda.current_device() if device is None else int(device)
    return DeviceAllocator(lambda nbytes, stream: torch.cuda.caching_allocator_alloc(nbytes, dev, stream),
                           lambda ptr, stream: torch.cuda.caching_allocator_delete(ptr))


def hyperim_load(n, he_off, he_mem, model="uniform_pair", uniform_threshold=0, seed=1,
                 stream=None, hbm_budget_bytes=0, allocator: Optional[DeviceAllocator] = None):
    """Returns a graph handle. he_off/he_mem: int32 numpy arrays (host) or CUDA tensors.
    allocator: None (the library's stream-ordered cudaMallocAsync) or a DeviceAllocator."""
    keep = []
    on_dev = 0
    if hasattr(he_off, "is_cuda") and he_off.is_cuda:
        import torch
        he_off = he_off.to(torch.int32).contiguous()
        he_mem = he_mem.to(torch.int32).contiguous()
        keep += [he_off, he_mem]
        p_off, p_mem, on_dev = he_off.data_ptr(), he_mem.data_ptr() if he_mem.numel() else None, 1
    else:
        he_off = np.ascontiguousarray(he_off, dtype=np.int32)
        he_mem = np.ascontiguousarray(he_mem, dtype=np.int32)
        keep += [he_off, he_mem]
        p_off, p_mem = he_off.ctypes.data, (he_mem.ctypes.data if he_mem.size else None)
    args = LoadArgs(int(n), len(he_off) - 1, p_off, p_mem, on_dev, MODELS[model],
                    int(uniform_threshold), int(seed),
                    stream if stream is not None else current_stream(), int(hbm_budget_bytes),
                    allocator.c_alloc if allocator is not None else ALLOC_FN(),
                    allocator.c_free if allocator is not None else FREE_FN(), None)
    h = C.c_void_p()
    _check(lib().hyperim_load(C.byref(args), C.byref(h)))
    return h


def hyperim_kernel_launches():
    return int(lib().hyperim_kernel_launches())


def hyperim_graph_free(h):
    lib().hyperim_graph_free(h)


def hyperim_plan_theta(h, k, eps, ell=1.0):
    p = ThetaPlan()
    _check(lib().hyperim_plan_theta(h, int(k), float(eps), float(ell), C.byref(p)))
    return {f: getattr(p, f) for f, _ in ThetaPlan._fields_}


def hyperim_sample_rr(h, pool_tag, theta, root_mode="plain", strategy="paper", pool=None):
    ph = pool if pool is not None else C.c_void_p()
    _check(lib().hyperim_sample_rr(h, int(pool_tag), int(theta), ROOTS[root_mode],
                                   STRATEGIES[strategy], C.byref(ph)))
    return ph


UPPER_MODES = {"closed": 0, "prefix": 1}


def hyperim_select_seeds(h, r1, r2, k, mode="fixed", eps=0.1, ell=1.0, theta_cap=0,
                         root_mode="stratified", strategy="paper", upper="closed"):
    opts = SelectOpts(SELECT_MODES[mode], float(eps), float(ell), int(theta_cap), ROOTS[root_mode],
                      STRATEGIES[strategy], UPPER_MODES[upper])
    seeds = np.zeros(int(k), dtype=np.int32)
    res = SelectResult()
    _check(lib().hyperim_select_seeds(h, r1, r2, int(k), C.byref(opts), _ptr(seeds), C.byref(res)))
    return seeds, _select_result(res)


def hyperim_select_seeds_batch(queries):
    """HyperIM_BRR for many queries in one call (one RR launch and one greedy launch per round).
    queries: sequence of (graph, r1, r2, k, eps, ell) with Graph / Pool objects. Returns a list of
    (seeds, result) in query order, each as hyperim_select_seeds in BRR mode returns it."""
    qs = (BatchQuery * len(queries))()
    seeds, results = [], []
    for i, (g, r1, r2, k, eps, ell) in enumerate(queries):
        sd = np.zeros(int(k), dtype=np.int32)
        res = SelectResult()
        seeds.append(sd)
        results.append(res)
        qs[i] = BatchQuery(g.handle, r1.handle, r2.handle, int(k), float(eps), float(ell), _ptr(sd),
                           C.pointer(res))
    _check(lib().hyperim_select_seeds_batch(qs, len(queries)))
    return [(sd, _select_result(res)) for sd, res in zip(seeds, results)]


def _select_result(res):
    out = {f: getattr(res, f) for f, _ in SelectResult._fields_
           if f not in ("lambda_r1", "lambda_r2", "alpha_round")}
    out["lambda_r1"] = np.array(res.lambda_r1, dtype=np.uint64)
    out["lambda_r2"] = np.array(res.lambda_r2, dtype=np.uint64)
    out["alpha_round"] = list(res.alpha_round)[: res.rounds]
    return out


def hyperim_spread(h, seeds, pool):
    s = np.ascontiguousarray(seeds, dtype=np.int32)
    sig, err = C.c_double(), C.c_double()
    _check(lib().hyperim_spread(h, _ptr(s) if s.size else None, len(s), pool, C.byref(sig),
                                C.byref(err)))
    return sig.value, err.value


# ------------------------------------------------------------------------------------------------
# handle classes
# ------------------------------------------------------------------------------------------------
class Graph:
    """A hypergraph loaded on the device (incidence store + layer profile)."""

    def __init__(self, n, he_off, he_mem, model="uniform_pair", uniform_threshold=0, seed=1,
                 stream=None, hbm_budget_bytes=0, allocator=None):
        self.n = int(n)
        self.model = model
        self._h = hyperim_load(n, he_off, he_mem, model, uniform_threshold, seed, stream,
                               hbm_budget_bytes, allocator)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().hyperim_graph_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self):
        s = GraphStats()
        _check(lib().hyperim_graph_stats(self._h, C.byref(s)))
        out = {f: getattr(s, f) for f, _ in GraphStats._fields_ if f != "stratum_size"}
        out["stratum_size"] = list(s.stratum_size)
        return out

    def profile(self):
        st = self.stats()
        n, L = self.n, st["profile_entries"]
        deg = np.zeros(n, np.int32)
        nl = np.zeros(n, np.int32)
        strat = np.zeros(n, np.int32)
        poff = np.zeros(n + 1, np.int64)
        lw = np.zeros(max(L, 1), np.uint32)
        ln = np.zeros(max(L, 1), np.uint32)
        lt = np.zeros(max(L, 1), np.uint64)
        _check(lib().hyperim_graph_profile(self._h, _ptr(deg), _ptr(nl), _ptr(strat), _ptr(poff),
                                           _ptr(lw), _ptr(ln), _ptr(lt)))
        return {"deg": deg, "nlayers": nl, "stratum": strat, "prof_off": poff,
                "layer_w": lw[:L], "layer_n": ln[:L], "layer_thr": lt[:L]}

    def chunk_index(self, v):
        """(bits, table[l_v, 2^bits]) of vertex v's chunk index, or (0, None) if it has none."""
        bits, entries = C.c_int32(), C.c_int64()
        _check(lib().hyperim_graph_chunk_index(self._h, int(v), C.byref(bits), None, 0, C.byref(entries)))
        if entries.value == 0:
            return 0, None
        tab = np.zeros(entries.value, np.uint32)
        _check(lib().hyperim_graph_chunk_index(self._h, int(v), C.byref(bits), _ptr(tab), entries.value,
                                               C.byref(entries)))
        return bits.value, tab.reshape(-1, 1 << bits.value)

    def share(self, stream=None):
        """A second handle on this graph (hyperim_graph_share): same device data and pools, its own
        stream (a cudaStream_t as int; default: the current torch stream) and scratch, for use
        from another host thread at the same time."""
        h = C.c_void_p()
        _check(lib().hyperim_graph_share(self._h, stream if stream is not None else current_stream(),
                                         C.byref(h)))
        g = Graph.__new__(Graph)
        g.n, g.model, g._h, g.parent = self.n, self.model, h, self
        return g

    def tuning(self):
        t = Tuning()
        _check(lib().hyperim_graph_get_tuning(self._h, C.byref(t)))
        return {"warp_set_limit": t.warp_set_limit, "early_sets_per_block": t.early_sets_per_block,
                "arena_entries_per_set": t.arena_entries_per_set}

    def set_tuning(self, warp_set_limit=None, early_sets_per_block=None, arena_entries_per_set=None):
        """RR-generation scheduling (hyperim_graph_set_tuning); the results never change."""
        cur = self.tuning()
        pick = lambda v, k: int(cur[k] if v is None else v)
        t = Tuning(pick(warp_set_limit, "warp_set_limit"), pick(early_sets_per_block, "early_sets_per_block"),
                   pick(arena_entries_per_set, "arena_entries_per_set"))
        _check(lib().hyperim_graph_set_tuning(self._h, C.byref(t)))

    def autotune(self, roots="stratified", strategy="paper", sets=0):
        """hyperim_graph_autotune: measure the RR-scheduling candidates (or reuse the process's
        choice for an equal degree profile) and apply the fastest; returns what was chosen."""
        r = AutotuneResult()
        _check(lib().hyperim_graph_autotune(self._h, ROOTS[roots], STRATEGIES[strategy], int(sets), C.byref(r)))
        return {"warp_set_limit": r.chosen.warp_set_limit,
                "early_sets_per_block": r.chosen.early_sets_per_block, "from_cache": bool(r.from_cache),
                "candidates": [(r.warp_set_limit[i], r.seconds[i]) for i in range(r.candidates)],
                "profile_key": r.profile_key}

    def set_wait_limit(self, iterations):
        """Bound of the device-side waits of this handle's kernels (0: the default, 2^24 rounds);
        a wait that runs out makes the call raise HYPERIM_ETIMEDOUT."""
        _check(lib().hyperim_graph_set_wait_limit(self._h, int(iterations)))

    def set_schedule(self, schedule):
        """RR generation schedule: "persistent" (default) or "plain" (one launch per batch of one
        set per block, the comparison form); the RR sets are the same under both."""
        _check(lib().hyperim_graph_set_schedule(self._h, SCHEDULES[schedule]))

    def forward_spread(self, seeds, simulations, seed):
        """(counts[simulations], mean, std_err) of forward IC cascades from `seeds` (Sec. 2.2)."""
        s = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32))
        counts = np.zeros(int(simulations), np.uint32)
        mean, se = C.c_double(), C.c_double()
        _check(lib().hyperim_forward_spread(self._h, _ptr(s), len(s), int(simulations), int(seed),
                                            _ptr(counts), C.byref(mean), C.byref(se)))
        return counts, mean.value, se.value

    def plan_theta(self, k, eps, ell=1.0):
        return hyperim_plan_theta(self._h, k, eps, ell)

    def pool(self, tag=0, roots="plain", strategy="paper"):
        return Pool(self, tag, roots, strategy)

    def select_seeds(self, r1, r2, k, mode="fixed", eps=0.1, ell=1.0, theta_cap=0, upper="closed"):
        return hyperim_select_seeds(self._h, r1.handle, r2.handle if r2 is not None else None, k,
                                    mode, eps, ell, theta_cap, r1.roots, r1.strategy, upper)

    def spread(self, seeds, pool):
        return hyperim_spread(self._h, seeds, pool.handle)


class Pool:
    """An RR-set pool of a graph (grown with sample())."""

    def __init__(self, graph: Graph, tag=0, roots="plain", strategy="paper"):
        self.graph = graph
        self.tag = int(tag)
        self.roots = roots
        self.strategy = strategy
        self._h = C.c_void_p()
        # an empty pool: theta = 0 creates the handle without sampling
        self._h = hyperim_sample_rr(graph.handle, self.tag, 0, roots, strategy, self._h)

    @property
    def handle(self):
        return self._h

    def sample(self, theta):
        self._h = hyperim_sample_rr(self.graph.handle, self.tag, theta, self.roots, self.strategy,
                                    self._h)
        return self

    def view(self):
        v = PoolView()
        _check(lib().hyperim_pool_view(self._h, C.byref(v)))
        out = {f: getattr(v, f) for f, _ in PoolView._fields_ if f != "n_s"}
        out["n_s"] = np.array(v.n_s, dtype=np.uint64)
        return out

    def counters(self):
        v = self.view()
        return {k: v[k] for k in ("pops", "layers_seen", "draws", "mats", "mat_he", "mat_members",
                                  "selected")}

    def to_host(self):
        v = self.view()
        N, T = v["count"], v["total"]
        off = np.zeros(N + 1, np.int64)
        mem = np.zeros(max(T, 1), np.int32)
        st = np.zeros(max(N, 1), np.uint8)
        j = np.zeros(max(N, 1), np.uint32)
        _check(lib().hyperim_pool_copy(self._h, _ptr(off), _ptr(mem), _ptr(st), _ptr(j)))
        return off, mem[:T], st[:N], j[:N]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().hyperim_pool_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ShardPool(Pool):
    """One shard of an RR pool split over `world` ranks (hyperim_sample_rr_shard): the sets
    (s, j) with j = rank (mod world) of each growth's allocation."""

    def __init__(self, graph: Graph, tag=0, rank=0, world=1, roots="stratified", strategy="paper"):
        self.graph = graph
        self.tag = int(tag)
        self.roots = roots
        self.strategy = strategy
        self.rank, self.world = int(rank), int(world)
        self._h = C.c_void_p()
        self.sample(0)

    def sample(self, theta):
        _check(lib().hyperim_sample_rr_shard(self.graph.handle, self.tag, int(theta), ROOTS[self.roots],
                                             STRATEGIES[self.strategy], self.rank, self.world, C.byref(self._h)))
        return self


class GreedyRounds:
    """Greedy max coverage one round at a time on a pool's prefix view (hyperim_greedy_*)."""

    def __init__(self, graph: Graph, pool: Pool, theta=0):
        self._h = C.c_void_p()
        _check(lib().hyperim_greedy_begin(graph.handle, pool.handle, int(theta), C.byref(self._h)))

    def scores_into(self, dev_ptr: int):
        """Copies the n current scores (uint64) to caller-owned device memory."""
        _check(lib().hyperim_greedy_scores(self._h, C.c_void_p(int(dev_ptr))))

    def pick(self, dev_total=None) -> int:
        """Argmax of the summed scores at dev_total (device pointer; None: this pool's own), then
        the retirement of this pool's sets that contain it; returns the vertex."""
        v = C.c_int32()
        _check(lib().hyperim_greedy_pick(self._h, C.c_void_p(int(dev_total)) if dev_total else None, C.byref(v)))
        return v.value

    def end(self):
        lam = np.zeros(NSTRATA, np.uint64)
        _check(lib().hyperim_greedy_end(self._h, _ptr(lam)))
        self._h = None
        return lam


def hyperim_coverage_view(graph: Graph, pool: Pool, theta, seeds):
    s = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32))
    lam = np.zeros(NSTRATA, np.uint64)
    _check(lib().hyperim_coverage_view(graph.handle, pool.handle, int(theta), _ptr(s) if s.size else None, len(s),
                                       _ptr(lam)))
    return lam


def hyperim_brr_round(graph: Graph, k, eps, ell, roots, i, lambda_r1, lambda_r2):
    a = np.ascontiguousarray(lambda_r1, dtype=np.uint64)
    b = np.ascontiguousarray(lambda_r2, dtype=np.uint64)
    r = BrrRound()
    _check(lib().hyperim_brr_round(graph.handle, int(k), float(eps), float(ell), ROOTS[roots], int(i), _ptr(a), _ptr(b),
                                   C.byref(r)))
    return {f: getattr(r, f) for f, _ in BrrRound._fields_}


class Server:
    """Query server over resident graphs (hyperim_server_*): continuous batching of BRR queries
    on `workers` host threads, each with its own CUDA stream; admission by HBM budget."""

    def __init__(self, workers=4, hbm_budget_bytes=0):
        self._h = C.c_void_p()
        _check(lib().hyperim_server_create(C.byref(ServerArgs(int(workers), int(hbm_budget_bytes))),
                                           C.byref(self._h)))
        self.graphs = []
        self._k = {}

    def add_graph(self, graph):
        gid = C.c_int32()
        _check(lib().hyperim_server_add_graph(self._h, graph.handle, C.byref(gid)))
        self.graphs.append(graph)
        return gid.value

    def submit(self, graph_id, k, eps=0.1, ell=1.0, upper="closed"):
        t = C.c_uint64()
        _check(lib().hyperim_server_submit(self._h, C.byref(Query(int(graph_id), int(k), float(eps), float(ell),
                                                                  UPPER_MODES[upper])), C.byref(t)))
        self._k[t.value] = int(k)
        return t.value

    def wait(self, ticket):
        """(seeds, result dict with status, latency_seconds, ...) of a submitted query."""
        seeds = np.zeros(self._k.pop(ticket, 1), np.int32)
        r = QueryResult()
        _check(lib().hyperim_server_wait(self._h, C.c_uint64(ticket), _ptr(seeds), C.byref(r)))
        out = _select_result(r.result)
        out.update(status=r.status, queued_seconds=r.queued_seconds, run_seconds=r.run_seconds,
                   latency_seconds=r.latency_seconds, worker=r.worker)
        if r.status != 0:
            out["message"] = lib().hyperim_last_error().decode(errors="replace")
        return seeds[:r.k], out

    def stats(self):
        st = ServerStats()
        _check(lib().hyperim_server_stats(self._h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().hyperim_server_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

