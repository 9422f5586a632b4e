"""HyperIM CPU oracle -- TEST INFRASTRUCTURE ONLY.

ctypes binding of the plain single-threaded C oracle in ``hyperim_oracle.c``. Only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this package; the
CUDA library never does, and the two share no code.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Optional

import numpy as np

from . import build as _build

MODELS = {"uniform_pair": 0, "wc": 1, "paper_layer": 2}
ROOTS = {"plain": 0, "stratified": 1}
STRATEGIES = {"paper": 0, "binomial_only": 1, "lt": 2}
NSTRATA = 16
P_ONE = 1 << 32

_lib = None


class Stats(C.Structure):
    _fields_ = [(name, C.c_uint64) for name in (
        "rr_sets", "pops", "layers_seen", "draws", "mats", "mat_he", "mat_members", "selected",
        "members_out", "bytes_rr")]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class Plan(C.Structure):
    _fields_ = [("delta", C.c_double), ("ln_binom", C.c_double), ("theta_max", C.c_double),
                ("theta_max_ceil", C.c_uint64), ("theta0", C.c_uint64), ("i_max", C.c_int32)]


class BrrResult(C.Structure):
    _fields_ = [("rounds", C.c_int32), ("theta", C.c_uint64), ("pool_r1", C.c_uint64),
                ("pool_r2", C.c_uint64), ("sigma_r1", C.c_double), ("sigma_r2", C.c_double),
                ("upper", C.c_double), ("lower", C.c_double), ("alpha", C.c_double),
                ("alpha_round", C.c_double * 64), ("lambda_r1", C.c_uint64 * NSTRATA),
                ("lambda_r2", C.c_uint64 * NSTRATA)]


def _p(arr, ctype):
    return arr.ctypes.data_as(C.POINTER(ctype))


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp = C.c_void_p
        u32p, u64p, i32p, i64p = (C.POINTER(C.c_uint32), C.POINTER(C.c_uint64),
                                  C.POINTER(C.c_int32), C.POINTER(C.c_int64))
        sig = {
            "or_philox4x32_10": (None, [u32p, u32p, u32p]),
            "or_exp_neg": (C.c_double, [C.c_double]),
            "or_binomial_h": (C.c_uint32, [C.c_uint32, C.c_uint64, C.c_uint32]),
            "or_poisson_h": (C.c_uint32, [C.c_uint32, C.c_uint64, u32p, C.c_uint32, u32p]),
            "or_poisson_parts": (C.c_uint32, [C.c_uint32, C.c_uint64]),
            "or_graph_build": (C.c_int, [C.c_int32, C.c_int32, i32p, i32p, C.c_int, C.c_uint64,
                                         C.POINTER(vp)]),
            "or_graph_free": (None, [vp]),
            "or_graph_n": (C.c_int32, [vp]),
            "or_graph_nnz": (C.c_int64, [vp]),
            "or_graph_he_size": (C.c_int32, [vp, C.c_int32]),
            "or_graph_dh": (C.c_int32, [vp, C.c_int32]),
            "or_graph_deg": (C.c_int32, [vp, C.c_int32]),
            "or_graph_nlayers": (C.c_int32, [vp, C.c_int32]),
            "or_graph_stratum": (C.c_int32, [vp, C.c_int32]),
            "or_graph_stratum_size": (C.c_int32, [vp, C.c_int32]),
            "or_graph_theta_lstar": (C.c_double, [vp]),
            "or_graph_layer": (C.c_int, [vp, C.c_int32, C.c_int32, u32p, u32p, u64p]),
            "or_graph_layer_members": (C.c_int64, [vp, C.c_int32, C.c_int32, i32p, C.c_int64]),
            "or_allocate": (C.c_int, [vp, C.c_int, C.c_uint64, u64p]),
            "or_root": (C.c_int32, [vp, C.c_uint64, C.c_uint32, C.c_int, C.c_uint32, C.c_uint32]),
            "or_rr_set": (C.c_int64, [vp, C.c_uint64, C.c_uint32, C.c_int, C.c_uint32, C.c_uint32,
                                      C.c_int, i32p, C.c_int64, C.POINTER(Stats)]),
            "or_pool_create": (C.c_int, [vp, C.c_uint64, C.c_uint32, C.c_int, C.c_int,
                                         C.POINTER(vp)]),
            "or_pool_free": (None, [vp]),
            "or_pool_grow": (C.c_int, [vp, u64p]),
            "or_pool_count": (C.c_int64, [vp]),
            "or_pool_total": (C.c_int64, [vp]),
            "or_pool_counts": (None, [vp, u64p]),
            "or_pool_copy": (C.c_int, [vp, i64p, i32p, C.POINTER(C.c_uint8), u32p]),
            "or_pool_stats": (None, [vp, C.POINTER(Stats)]),
            "or_greedy": (C.c_int, [vp, C.c_int32, i32p, u64p, u64p]),
            "or_greedy_upper": (C.c_int, [vp, C.c_int32, i32p, u64p, u64p, u64p]),
            "or_prefix_upper_sigma": (C.c_double, [C.c_uint64, C.c_uint64, C.c_int, C.c_int64,
                                                   C.c_uint64]),
            "or_coverage": (C.c_int, [vp, i32p, C.c_int32, u64p]),
            "or_estimate": (C.c_double, [vp, u64p]),
            "or_forward_spread": (C.c_int, [vp, i32p, C.c_int32, C.c_uint64, C.c_uint64,
                                            C.POINTER(C.c_uint32)]),
            "or_plan_theta": (C.c_int, [C.c_int64, C.c_int32, C.c_double, C.c_double,
                                        C.POINTER(Plan)]),
            "or_upper_bound": (C.c_double, [C.c_double, C.c_int32, C.c_int64, C.c_uint64]),
            "or_lower_bound": (C.c_double, [C.c_double, C.c_double, C.c_int64, C.c_uint64]),
            "or_brr": (C.c_int, [vp, C.c_uint64, C.c_int32, C.c_double, C.c_double, C.c_uint64,
                                 C.c_int, C.c_int, i32p, C.POINTER(BrrResult),
                                 C.POINTER(Stats)]),
            "or_brr_upper": (C.c_int, [vp, C.c_uint64, C.c_int32, C.c_double, C.c_double, C.c_uint64,
                                       C.c_int, C.c_int, C.c_int, i32p, C.POINTER(BrrResult),
                                       C.POINTER(Stats)]),
            "or_graph_worker": (C.c_int, [vp, C.POINTER(vp)]),
            "or_pool_grow_mt": (C.c_int, [vp, u64p, C.POINTER(vp), C.c_int]),
            "or_brr_upper_mt": (C.c_int, [vp, C.c_uint64, C.c_int32, C.c_double, C.c_double, C.c_uint64,
                                          C.c_int, C.c_int, C.c_int, i32p, C.POINTER(BrrResult),
                                          C.POINTER(Stats), C.POINTER(vp), C.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc != 0:
        raise OracleError(f"oracle call failed with status {rc}")


# ---------------------------------------------------------------------------------------------
# primitives
# ---------------------------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def exp_neg(x: float) -> float:
    return lib().or_exp_neg(float(x))


def binomial_h(n: int, thr: int, w0: int) -> int:
    return lib().or_binomial_h(n, thr, w0)


def poisson_h(n: int, thr: int, words) -> tuple:
    w = np.asarray(words, dtype=np.uint32).copy()
    used = C.c_uint32(0)
    h = lib().or_poisson_h(n, thr, _p(w, C.c_uint32), len(w), C.byref(used))
    return h, used.value


def poisson_parts(n: int, thr: int) -> int:
    return lib().or_poisson_parts(n, thr)


# ---------------------------------------------------------------------------------------------
# graph, pools, greedy
# ---------------------------------------------------------------------------------------------
class Graph:
    """Incidence store + layer profile (Sec. 3.1.1) built by the oracle."""

    def __init__(self, n, he_off, he_mem, model="uniform_pair", uniform_threshold=0):
        self.he_off = np.ascontiguousarray(he_off, dtype=np.int32)
        self.he_mem = np.ascontiguousarray(he_mem, dtype=np.int32)
        self.n = int(n)
        self.m = len(self.he_off) - 1
        self.model = model
        h = C.c_void_p()
        mem = self.he_mem if len(self.he_mem) else np.zeros(1, dtype=np.int32)
        _check(lib().or_graph_build(self.n, self.m, _p(self.he_off, C.c_int32),
                                    _p(mem, C.c_int32), MODELS[model], int(uniform_threshold),
                                    C.byref(h)))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and h.value and _lib is not None:
            _lib.or_graph_free(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def dh(self, v): return lib().or_graph_dh(self._h, v)
    def deg(self, v): return lib().or_graph_deg(self._h, v)
    def nlayers(self, v): return lib().or_graph_nlayers(self._h, v)
    def stratum(self, v): return lib().or_graph_stratum(self._h, v)
    def stratum_size(self, s): return lib().or_graph_stratum_size(self._h, s)
    def theta_lstar(self): return lib().or_graph_theta_lstar(self._h)
    def nnz(self): return lib().or_graph_nnz(self._h)

    def layers(self, v):
        """[(w_i, n_i, threshold)] for i = 1..l_v"""
        out = []
        w, n_i, thr = C.c_uint32(), C.c_uint32(), C.c_uint64()
        for i in range(1, self.nlayers(v) + 1):
            _check(lib().or_graph_layer(self._h, v, i, C.byref(w), C.byref(n_i), C.byref(thr)))
            out.append((w.value, n_i.value, thr.value))
        return out

    def layer_members(self, v, i):
        cap = self.n
        buf = np.zeros(cap, dtype=np.int32)
        c = lib().or_graph_layer_members(self._h, v, i, _p(buf, C.c_int32), cap)
        if c < 0:
            raise OracleError(f"layer_members status {c}")
        return buf[:c].copy()

    def forward_spread(self, seeds, sims, seed):
        """Activated-vertex counts of `sims` forward IC cascades from `seeds` (Sec. 2.2)."""
        s = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32))
        out = np.zeros(max(int(sims), 1), dtype=np.uint32)
        _check(lib().or_forward_spread(self._h, _p(s, C.c_int32), len(s), int(sims), int(seed),
                                       _p(out, C.c_uint32)))
        return out[:int(sims)]

    def allocate(self, roots, theta):
        ns = np.zeros(NSTRATA, dtype=np.uint64)
        _check(lib().or_allocate(self._h, ROOTS[roots], int(theta), _p(ns, C.c_uint64)))
        return ns

    def root(self, seed, tag, roots, stratum, j):
        return lib().or_root(self._h, seed, tag, ROOTS[roots], stratum, j)

    def rr_set(self, seed, tag, roots, stratum, j, strategy="paper", stats: Optional[Stats] = None):
        cap = self.n
        buf = np.zeros(cap, dtype=np.int32)
        st = stats if stats is not None else Stats()
        c = lib().or_rr_set(self._h, seed, tag, ROOTS[roots], stratum, j, STRATEGIES[strategy],
                            _p(buf, C.c_int32), cap, C.byref(st))
        if c < 0:
            raise OracleError(f"rr_set status {c}")
        return buf[:c].copy()


@dataclasses.dataclass
class PoolArrays:
    off: np.ndarray
    mem: np.ndarray
    stratum: np.ndarray
    j: np.ndarray


class Pool:
    def __init__(self, graph: Graph, seed=1, tag=0, roots="plain", strategy="paper"):
        self.graph = graph
        self.roots = roots
        h = C.c_void_p()
        _check(lib().or_pool_create(graph.handle, seed, tag, ROOTS[roots], STRATEGIES[strategy],
                                    C.byref(h)))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and h.value and _lib is not None:
            _lib.or_pool_free(h)
            self._h = None

    def grow(self, n_s, workers: Optional["Workers"] = None):
        ns = np.ascontiguousarray(n_s, dtype=np.uint64)
        if workers is not None and len(workers.views) > 1:
            _check(lib().or_pool_grow_mt(self._h, _p(ns, C.c_uint64), workers.array, len(workers.views)))
        else:
            _check(lib().or_pool_grow(self._h, _p(ns, C.c_uint64)))

    def grow_theta(self, theta, workers: Optional["Workers"] = None):
        self.grow(self.graph.allocate(self.roots, theta), workers)

    def count(self): return lib().or_pool_count(self._h)
    def total(self): return lib().or_pool_total(self._h)

    def counts(self):
        ns = np.zeros(NSTRATA, dtype=np.uint64)
        lib().or_pool_counts(self._h, _p(ns, C.c_uint64))
        return ns

    def arrays(self) -> PoolArrays:
        N, T = self.count(), self.total()
        off = np.zeros(N + 1, dtype=np.int64)
        mem = np.zeros(max(T, 1), dtype=np.int32)
        st = np.zeros(max(N, 1), dtype=np.uint8)
        j = np.zeros(max(N, 1), dtype=np.uint32)
        lib().or_pool_copy(self._h, _p(off, C.c_int64), _p(mem, C.c_int32),
                           _p(st, C.c_uint8), _p(j, C.c_uint32))
        return PoolArrays(off, mem[:T], st[:N], j[:N])

    def stats(self) -> dict:
        s = Stats()
        lib().or_pool_stats(self._h, C.byref(s))
        return s.as_dict()

    def greedy(self, k):
        seeds = np.zeros(max(k, 1), dtype=np.int32)
        lam = np.zeros(NSTRATA, dtype=np.uint64)
        gains = np.zeros(max(k, 1), dtype=np.uint64)
        _check(lib().or_greedy(self._h, k, _p(seeds, C.c_int32), _p(lam, C.c_uint64),
                               _p(gains, C.c_uint64)))
        return seeds[:k], lam, gains[:k]

    def greedy_upper(self, k):
        """greedy plus Eq. upper_2 (p_max = 1) as an exact integer in the greedy's weights."""
        seeds = np.zeros(max(k, 1), dtype=np.int32)
        lam = np.zeros(NSTRATA, dtype=np.uint64)
        gains = np.zeros(max(k, 1), dtype=np.uint64)
        pu = np.zeros(2, dtype=np.uint64)
        _check(lib().or_greedy_upper(self._h, k, _p(seeds, C.c_int32), _p(lam, C.c_uint64),
                                     _p(gains, C.c_uint64), _p(pu, C.c_uint64)))
        return seeds[:k], lam, gains[:k], int(pu[0]) | (int(pu[1]) << 64)

    def coverage(self, seeds):
        s = np.ascontiguousarray(seeds, dtype=np.int32)
        lam = np.zeros(NSTRATA, dtype=np.uint64)
        _check(lib().or_coverage(self._h, _p(s, C.c_int32), len(s), _p(lam, C.c_uint64)))
        return lam

    def estimate(self, lam):
        l = np.ascontiguousarray(lam, dtype=np.uint64)
        return lib().or_estimate(self._h, _p(l, C.c_uint64))


def plan_theta(n, k, eps, ell=1.0):
    p = Plan()
    _check(lib().or_plan_theta(int(n), int(k), float(eps), float(ell), C.byref(p)))
    return {"delta": p.delta, "ln_binom": p.ln_binom, "theta_max": p.theta_max,
            "theta_max_ceil": p.theta_max_ceil, "theta0": p.theta0, "i_max": p.i_max}


def upper_bound(lambda1, k, n, theta):
    return lib().or_upper_bound(float(lambda1), int(k), int(n), int(theta))


def lower_bound(lambda2, delta, n, theta):
    return lib().or_lower_bound(float(lambda2), float(delta), int(n), int(theta))


UPPER = {"closed": 0, "prefix": 1}


def prefix_upper_sigma(u, roots, n, N):
    return lib().or_prefix_upper_sigma(u & ((1 << 64) - 1), u >> 64, ROOTS[roots], n, N)


class Workers:
    """Worker views of an oracle graph (one per thread) for the multi-threaded pool growth."""

    def __init__(self, graph: Graph, threads: int):
        self.graph = graph
        self.views = []
        for _ in range(max(int(threads), 1)):
            h = C.c_void_p()
            _check(lib().or_graph_worker(graph.handle, C.byref(h)))
            self.views.append(h)
        self.array = (C.c_void_p * len(self.views))(*[h.value for h in self.views])

    def rr_set(self, t, seed, tag, roots, stratum, j, strategy="paper"):
        """Graph.rr_set on worker view t (call it from one thread per view)."""
        cap = self.graph.n
        buf = np.zeros(cap, dtype=np.int32)
        st = Stats()
        c = lib().or_rr_set(self.views[t], seed, tag, ROOTS[roots], stratum, j, STRATEGIES[strategy],
                            _p(buf, C.c_int32), cap, C.byref(st))
        if c < 0:
            raise OracleError(f"rr_set status {c}")
        return buf[:c].copy()

    def close(self):
        for h in self.views:
            lib().or_graph_free(h)
        self.views = []

    def __del__(self):
        try:
            if _lib is not None:
                self.close()
        except Exception:
            pass


def brr(graph: Graph, seed, k, eps, ell=1.0, cap=0, roots="stratified", strategy="paper", upper="closed",
        threads=1):
    """HyperIM_BRR (Alg. 4) by the oracle; threads > 1 grows the pools with that many threads
    (same pools, same result)."""
    seeds = np.zeros(max(k, 1), dtype=np.int32)
    res = BrrResult()
    st = Stats()
    if threads > 1:
        W = Workers(graph, threads)
        try:
            _check(lib().or_brr_upper_mt(graph.handle, seed, k, eps, ell, cap, ROOTS[roots],
                                         STRATEGIES[strategy], UPPER[upper], _p(seeds, C.c_int32),
                                         C.byref(res), C.byref(st), W.array, len(W.views)))
        finally:
            W.close()
    else:
        _check(lib().or_brr_upper(graph.handle, seed, k, eps, ell, cap, ROOTS[roots], STRATEGIES[strategy],
                                  UPPER[upper], _p(seeds, C.c_int32), C.byref(res), C.byref(st)))
    out = {f: getattr(res, f) for f, _ in BrrResult._fields_
           if f not in ("alpha_round", "lambda_r1", "lambda_r2")}
    out["alpha_round"] = list(res.alpha_round)[:res.rounds]
    out["lambda_r1"] = np.array(res.lambda_r1, dtype=np.uint64)
    out["lambda_r2"] = np.array(res.lambda_r2, dtype=np.uint64)
    out["stats"] = st.as_dict()
    return seeds[:k], out
