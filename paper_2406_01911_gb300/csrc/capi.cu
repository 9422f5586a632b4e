// C ABI of the HyperIM library (declared in include/hyperim.h) and its host-side arithmetic:
// the RR budget of Sec. 4.3, root allocation per stratum, the Eq. 1 estimate, and the
// HyperIM_BRR doubling driver (Algorithm 4). Device work lives in load.cu, rr.cu, greedy.cu.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <shared_mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace hyperim {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

void count_launch(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

hyperim_status set_error(hyperim_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

hyperim_status cuda_fail(cudaError_t e, const char* what) {
    return set_error(e == cudaErrorMemoryAllocation ? HYPERIM_ENOMEM : HYPERIM_ECUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

hyperim_status dev_alloc(hyperim_graph* g, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    hyperim_graph* r = graph_root(g);  // one budget for all handles of a graph
    const size_t before = r->device_bytes.fetch_add(bytes);
    if (r->budget && before + bytes > r->budget) {
        r->device_bytes.fetch_sub(bytes);
        return set_error(HYPERIM_ENOMEM, "device memory budget exceeded (" + std::to_string(before + bytes) +
                                             " > " + std::to_string(r->budget) + " bytes)");
    }
    if (g->alloc_fn) {
        *p = g->alloc_fn(bytes, (void*)g->stream, g->alloc_ctx);
        if (!*p) {
            r->device_bytes.fetch_sub(bytes);
            return set_error(HYPERIM_ENOMEM, "the caller's dev_alloc(" + std::to_string(bytes) + ") returned NULL");
        }
        return HYPERIM_OK;
    }
    cudaError_t e = cudaMallocAsync(p, bytes, g->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        r->device_bytes.fetch_sub(bytes);
        return set_error(HYPERIM_ENOMEM, std::string("cudaMallocAsync(") + std::to_string(bytes) +
                                             "): " + cudaGetErrorString(e));
    }
    return HYPERIM_OK;
}

// releases a device buffer through the allocator the graph was loaded with
static void release(hyperim_graph* g, void* p) {
    if (g->free_fn) g->free_fn(p, (void*)g->stream, g->alloc_ctx);
    else cudaFreeAsync(p, g->stream);
}

void dev_free(hyperim_graph* g, void* p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 16;
    release(g, p);
    graph_root(g)->device_bytes.fetch_sub(bytes);
}

std::mutex& graph_mutex() {
    static std::mutex m;
    return m;
}

hyperim_status check_device_status(hyperim_graph* g, const char* where) {
    DevStatus h;
    HYP_CUDA(cudaMemcpyAsync(&h, g->d_status, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    HYP_CUDA(cudaStreamSynchronize(g->stream));
    if (h.code == kErrNone) return HYPERIM_OK;
    HYP_CUDA(cudaMemsetAsync(g->d_status, 0, sizeof(DevStatus), g->stream));
    HYP_CUDA(cudaStreamSynchronize(g->stream));
    std::string msg = std::string(where) + ": ";
    switch (h.code) {
    case kErrBadMember:
        return set_error(HYPERIM_EINVAL, msg + "member id outside [0, n) in hyperedge " +
                                             std::to_string(h.detail));
    case kErrBadOffsets:
        return set_error(HYPERIM_EINVAL, msg + "hyperedge offsets not monotone from 0 at " +
                                             std::to_string(h.detail));
    case kErrWords:
        return set_error(HYPERIM_EOVERFLOW, msg + "a layer draw at vertex " +
                                                std::to_string(h.detail) +
                                                " needs more than 2^18 Philox words");
    case kErrCapacity:
    case kErrBucket:
        return set_error(HYPERIM_EOVERFLOW, msg + "scratch capacity exceeded at vertex " +
                                                std::to_string(h.detail));
    case kErrSpin:
        return set_error(HYPERIM_ETIMEDOUT, msg + "a bounded work-queue wait gave up in job " +
                                                std::to_string(h.detail));
    default:
        return set_error(HYPERIM_ECUDA, msg + "device error " + std::to_string(h.code));
    }
}

// ---- host arithmetic -----------------------------------------------------------------------
// n_s = ceil(theta |V_s| / n) for every nonempty stratum (stratified roots); theta (plain).
void allocate_strata(const hyperim_graph* g, int32_t root_mode, uint64_t theta,
                     uint64_t n_s[HYPERIM_NSTRATA]) {
    for (int s = 0; s < HYPERIM_NSTRATA; ++s) n_s[s] = 0;
    if (root_mode == HYPERIM_ROOTS_PLAIN) {
        n_s[0] = theta;
        return;
    }
    for (int s = 0; s < HYPERIM_NSTRATA; ++s) {
        if (g->stratum_size[s] == 0 || theta == 0) continue;
        const unsigned __int128 num = (unsigned __int128)theta * (uint64_t)g->stratum_size[s];
        n_s[s] = (uint64_t)((num + (uint64_t)g->n - 1) / (uint64_t)g->n);
    }
}

// Eq. 1 per stratum: sigma = sum_s (|V_s| / n_s) Lambda_s, strata in ascending order.
// Eq. upper_2 (integer greedy weights as {low, high} 64-bit words) in the units of sigma: the
// weights are floor(|V_s| 2^32 / n_s) with stratified roots (scale 2^-32), 1 with plain roots
// (scale n / N)
double prefix_upper_sigma(const uint64_t u[2], int32_t root_mode, int64_t n, uint64_t N) {
    const double x = (double)(((unsigned __int128)u[1] << 64) | u[0]);
    if (root_mode == HYPERIM_ROOTS_STRATIFIED) return x * 0x1p-32;
    return (x * (double)n) / (double)N;
}

double estimate(const hyperim_graph* g, int32_t root_mode, const uint64_t n_s[HYPERIM_NSTRATA],
                const uint64_t lambda_s[HYPERIM_NSTRATA]) {
    double sigma = 0.0;
    for (int s = 0; s < HYPERIM_NSTRATA; ++s) {
        if (n_s[s] == 0) continue;
        const double vs = root_mode == HYPERIM_ROOTS_PLAIN ? (double)g->n : (double)g->stratum_size[s];
        sigma = sigma + (vs / (double)n_s[s]) * (double)lambda_s[s];
    }
    return sigma;
}

uint64_t stratum_weight(const hyperim_graph* g, int32_t root_mode, uint64_t n_s, int s) {
    if (root_mode == HYPERIM_ROOTS_PLAIN) return 1;
    if (n_s == 0) return 0;
    return ((uint64_t)g->stratum_size[s] << 32) / n_s;
}

static hyperim_status plan_theta(int64_t n, int32_t k, double eps, double ell, hyperim_theta_plan* out) {
    if (n < 2 || k < 1 || k > n) return set_error(HYPERIM_EINVAL, "need 1 <= k <= n and n >= 2");
    if (!(eps > 0.0 && eps < 1.0)) return set_error(HYPERIM_EINVAL, "eps must lie in (0, 1)");
    if (!(ell > 0.0)) return set_error(HYPERIM_EINVAL, "ell must be positive");
    const double dn = (double)n, dk = (double)k;
    const double delta = std::pow(dn, -ell);
    // ln C(n, k) = sum_{i=1..k'} ln((n - k' + i) / i) with k' = min(k, n - k)
    const int64_t kk = std::min<int64_t>(k, n - k);
    double lnc = 0.0;
    for (int64_t i = 1; i <= kk; ++i) lnc = lnc + std::log((double)(n - kk + i) / (double)i);
    const double tmax = 2.0 * dn * (std::sqrt(std::log(2.0 / delta)) + std::sqrt(lnc + std::log(6.0 / delta))) /
                        (eps * eps * dk);
    const double t0 = tmax * eps * eps * dk / dn;
    uint64_t t0c = (uint64_t)std::ceil(t0);
    if (t0c < 1) t0c = 1;
    int32_t imax = 0;
    while ((double)t0c * std::ldexp(1.0, imax) < tmax) ++imax;
    out->delta = delta;
    out->ln_binom = lnc;
    out->theta_max = tmax;
    out->theta_max_ceil = (uint64_t)std::ceil(tmax);
    out->theta0 = t0c;
    out->i_max = imax;
    return HYPERIM_OK;
}

// Eq. upper_6 with p_max = 1, scaled to spread units: Lambda1 / (1 - (1 - 1/k)^k) * n / |R1|.
static double upper_bound(double lam1, int32_t k, int64_t n, uint64_t theta) {
    const double base = 1.0 - 1.0 / (double)k;
    double pw = 1.0;
    for (int32_t i = 0; i < k; ++i) pw = pw * base;
    return lam1 / (1.0 - pw) * (double)n / (double)theta;
}

// Sec. 4.2: ((sqrt(Lambda2 + 2 ln(1/delta)/9) - sqrt(ln(1/delta)/2))^2 - ln(1/delta)/18) n/|R2|.
static double lower_bound(double lam2, double delta, int64_t n, uint64_t theta) {
    const double L = std::log(1.0 / delta);
    const double a = std::sqrt(lam2 + 2.0 * L / 9.0) - std::sqrt(L / 2.0);
    return (a * a - L / 18.0) * (double)n / (double)theta;
}

}  // namespace hyperim

using namespace hyperim;

extern "C" {

const char* hyperim_last_error(void) { return g_last_error.c_str(); }

uint64_t hyperim_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

hyperim_status hyperim_load(const hyperim_load_args* a, hyperim_graph_t* out) {
    if (!a || !out) return set_error(HYPERIM_EINVAL, "null argument");
    *out = nullptr;
    if (a->n < 1 || a->n >= 0x7FFFFFFF) return set_error(HYPERIM_EINVAL, "n must lie in [1, 2^31 - 1)");
    if (a->m < 0) return set_error(HYPERIM_EINVAL, "m must be >= 0");
    if (!a->he_off) return set_error(HYPERIM_EINVAL, "he_off is null");
    if (a->model < 0 || a->model > 2) return set_error(HYPERIM_EINVAL, "unknown probability model");
    if (a->uniform_threshold > HYPERIM_P_ONE) return set_error(HYPERIM_EINVAL, "uniform_threshold > 2^32");
    if ((a->dev_alloc == nullptr) != (a->dev_free == nullptr))
        return set_error(HYPERIM_EINVAL, "dev_alloc and dev_free must be given together");
    hyperim_graph* g = new (std::nothrow) hyperim_graph();
    if (!g) return set_error(HYPERIM_ENOMEM, "host allocation failed");
    g->n = a->n;
    g->m = a->m;
    g->model = a->model;
    g->uniform_thr = a->uniform_threshold;
    g->seed = a->seed;
    g->stream = (cudaStream_t)a->cuda_stream;
    g->budget = a->hbm_budget_bytes;
    g->alloc_fn = a->dev_alloc;
    g->free_fn = a->dev_free;
    g->alloc_ctx = a->alloc_ctx;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(e, "device query");
    }
    g->id_bits = 1;
    while (g->id_bits < 31 && (1ll << g->id_bits) < (int64_t)g->n) ++g->id_bits;
    int32_t nnz_in = 0;
    if (a->ptrs_on_device) {
        e = cudaMemcpyAsync(&nnz_in, a->he_off + a->m, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) {
            delete g;
            return cuda_fail(e, "reading he_off[m]");
        }
    } else {
        if (a->he_off[0] != 0) {
            delete g;
            return set_error(HYPERIM_EINVAL, "he_off[0] must be 0");
        }
        nnz_in = a->he_off[a->m];
    }
    if (nnz_in < 0 || (nnz_in > 0 && !a->he_mem)) {
        delete g;
        return set_error(HYPERIM_EINVAL, "bad member array");
    }
    hyperim_status st = dev_alloc(g, (void**)&g->d_status, sizeof(DevStatus));
    if (st == HYPERIM_OK) st = dev_alloc(g, (void**)&g->d_counters, 2 * sizeof(RRCounters));
    if (st == HYPERIM_OK) {
        cudaMemsetAsync(g->d_status, 0, sizeof(DevStatus), g->stream);
        st = build_graph(g, a->he_off, a->he_mem, nnz_in, a->ptrs_on_device != 0);
    }
    if (st != HYPERIM_OK) {
        std::string keep = g_last_error;
        hyperim_graph_free(g);
        g_last_error = keep;
        return st;
    }
    *out = g;
    return HYPERIM_OK;
}

namespace {
// frees what one handle owns: its status word, counters and RR-kernel scratch, and, for the
// loaded graph, the graph data itself when `data` is set
void free_handle(hyperim_graph* g, bool data) {
    cudaStreamSynchronize(g->stream);
    const Scratch& S = g->scratch;
    dev_free(g, g->d_status, sizeof(DevStatus));
    dev_free(g, g->d_counters, 2 * sizeof(RRCounters));
    dev_free(g, S.list, sizeof(int32_t) * S.list_cap * S.blocks);
    dev_free(g, S.bitmap, sizeof(uint32_t) * S.bitmap_words * S.blocks);
    dev_free(g, S.picks, sizeof(uint32_t) * S.pick_cap * S.blocks);
    dev_free(g, S.big, sizeof(uint32_t) * S.big_cap * S.blocks);
    dev_free(g, S.arena, sizeof(int32_t) * S.arena_cap);
    if (data) {
        void* ptrs[] = {g->he_off, g->he_mem, g->v_off, g->v_he, g->tsum, g->v_span, g->vinfo, g->prof_off,
                        g->prof, g->cdf_tab, g->deg, g->stratum, g->vs_off, g->vs_list, g->idx, g->idx_tab,
                        g->mat_sect, g->he_dir, g->v_dir};
        for (void* p : ptrs)
            if (p) release(g, p);
    }
    cudaStreamSynchronize(g->stream);
}

// drops one reference (a share or a pool) on a loaded graph; the last one after the graph's own
// hyperim_graph_free releases it
void release_root(hyperim_graph* r) {
    bool last = false;
    {
        std::lock_guard<std::mutex> lk(graph_mutex());
        last = --r->shares == 0 && r->freed;
    }
    if (last) {
        free_handle(r, true);
        delete r;
    }
}
}  // namespace

void hyperim_graph_free(hyperim_graph_t g) {
    if (!g) return;
    if (g->owner) {
        hyperim_graph* r = g->owner;
        free_handle(g, false);
        delete g;
        release_root(r);
        return;
    }
    bool keep = false;
    {
        std::lock_guard<std::mutex> lk(graph_mutex());
        g->freed = true;
        keep = g->shares > 0;
    }
    if (keep) return;  // the last share releases it
    free_handle(g, true);
    delete g;
}

hyperim_status hyperim_graph_share(hyperim_graph_t g, void* cuda_stream, hyperim_graph_t* out) {
    if (!g || !out) return set_error(HYPERIM_EINVAL, "null argument");
    *out = nullptr;
    hyperim_graph* r = graph_root(g);
    hyperim_graph* h = new (std::nothrow) hyperim_graph();
    if (!h) return set_error(HYPERIM_ENOMEM, "host allocation failed");
    {
        std::lock_guard<std::mutex> lk(graph_mutex());
        ++r->shares;
    }
    h->owner = r;
    h->stream = (cudaStream_t)cuda_stream;
    h->n = r->n;
    h->m = r->m;
    h->nnz = r->nnz;
    h->model = r->model;
    h->uniform_thr = r->uniform_thr;
    h->seed = r->seed;
    h->id_bits = r->id_bits;
    h->he_off = r->he_off;
    h->he_mem = r->he_mem;
    h->v_off = r->v_off;
    h->v_he = r->v_he;
    h->tsum = r->tsum;
    h->v_span = r->v_span;
    h->vinfo = r->vinfo;
    h->prof_off = r->prof_off;
    h->prof = r->prof;
    h->cdf_tab = r->cdf_tab;
    h->table_entries = r->table_entries;
    h->deg = r->deg;
    h->stratum = r->stratum;
    h->vs_off = r->vs_off;
    h->vs_list = r->vs_list;
    h->idx = r->idx;
    h->idx_tab = r->idx_tab;
    h->idx_entries = r->idx_entries;
    h->idx_vertices = r->idx_vertices;
    h->profile_entries = r->profile_entries;
    h->max_layers = r->max_layers;
    h->max_dh = r->max_dh;
    h->max_deg = r->max_deg;
    h->max_tsum = r->max_tsum;
    h->max_layer_n = r->max_layer_n;
    for (int s = 0; s < HYPERIM_NSTRATA; ++s) h->stratum_size[s] = r->stratum_size[s];
    h->theta_lstar = r->theta_lstar;
    h->sm_count = r->sm_count;
    h->schedule = r->schedule;
    h->wait_limit = r->wait_limit;
    h->warp_set_limit = r->warp_set_limit;
    h->early_sets_per_block = r->early_sets_per_block;
    h->arena_entries_per_set = r->arena_entries_per_set;
    h->set_size_hint = r->set_size_hint;
    h->set_cycles_mean = r->set_cycles_mean;
    h->set_cycles_max = r->set_cycles_max;
    h->alloc_fn = r->alloc_fn;
    h->free_fn = r->free_fn;
    h->alloc_ctx = r->alloc_ctx;
    h->mat_sect = r->mat_sect;
    h->he_dir = r->he_dir;
    h->v_dir = r->v_dir;
    h->dir_entries = r->dir_entries;
    hyperim_status st = dev_alloc(h, (void**)&h->d_status, sizeof(DevStatus));
    if (st == HYPERIM_OK) st = dev_alloc(h, (void**)&h->d_counters, 2 * sizeof(RRCounters));
    if (st == HYPERIM_OK) {
        cudaError_t e = cudaMemsetAsync(h->d_status, 0, sizeof(DevStatus), h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "share status word");
    }
    if (st != HYPERIM_OK) {
        std::string keep = g_last_error;
        hyperim_graph_free(h);
        g_last_error = keep;
        return st;
    }
    *out = h;
    return HYPERIM_OK;
}

hyperim_status hyperim_graph_stats(hyperim_graph_t g, hyperim_graph_stats_t* out) {
    if (!g || !out) return set_error(HYPERIM_EINVAL, "null argument");
    out->n = g->n;
    out->m = g->m;
    out->nnz = g->nnz;
    out->profile_entries = g->profile_entries;
    out->max_layers = g->max_layers;
    out->max_dh = g->max_dh;
    out->max_deg = g->max_deg;
    for (int s = 0; s < HYPERIM_NSTRATA; ++s) out->stratum_size[s] = g->stratum_size[s];
    out->theta_lstar = g->theta_lstar;
    out->device_bytes = graph_root(g)->device_bytes.load();
    out->index_vertices = g->idx_vertices;
    out->index_entries = g->idx_entries;
    return HYPERIM_OK;
}

hyperim_status hyperim_forward_spread(hyperim_graph_t g, const int32_t* seeds_host, int32_t k,
                                      uint64_t simulations, uint64_t seed, uint32_t* counts_host,
                                      double* mean, double* std_err) {
    if (!g) return set_error(HYPERIM_EINVAL, "null graph");
    if (k < 0 || (k > 0 && !seeds_host)) return set_error(HYPERIM_EINVAL, "bad seed list");
    if (simulations == 0 || simulations > 0x100000000ull)
        return set_error(HYPERIM_EINVAL, "simulations must be in [1, 2^32]");
    for (int32_t i = 0; i < k; ++i)
        if (seeds_host[i] < 0 || seeds_host[i] >= g->n) return set_error(HYPERIM_EINVAL, "seed outside [0, n)");
    std::vector<uint32_t> counts((size_t)simulations);
    hyperim_status st = forward_spread(g, seeds_host, k, simulations, seed, counts.data());
    if (st != HYPERIM_OK) return st;
    // mean and variance in one pass (Welford), in simulation order
    double m = 0.0, m2 = 0.0;
    for (uint64_t r = 0; r < simulations; ++r) {
        const double x = (double)counts[(size_t)r];
        const double d = x - m;
        m += d / (double)(r + 1);
        m2 += d * (x - m);
    }
    if (mean) *mean = m;
    if (std_err)
        *std_err = simulations > 1 ? std::sqrt(m2 / (double)(simulations - 1) / (double)simulations) : 0.0;
    if (counts_host) std::memcpy(counts_host, counts.data(), sizeof(uint32_t) * (size_t)simulations);
    return HYPERIM_OK;
}

hyperim_status hyperim_graph_chunk_index(hyperim_graph_t g, int32_t v, int32_t* bits, uint32_t* table,
                                         int64_t cap, int64_t* entries) {
    if (!g || !bits || !entries) return set_error(HYPERIM_EINVAL, "null argument");
    if (v < 0 || v >= g->n) return set_error(HYPERIM_EINVAL, "vertex outside [0, n)");
    uint64_t word = 0;
    int4 vi = make_int4(0, 0, 0, 0);
    HYP_CUDA(cudaMemcpyAsync(&word, g->idx + v, sizeof(word), cudaMemcpyDeviceToHost, g->stream));
    HYP_CUDA(cudaMemcpyAsync(&vi, g->vinfo + v, sizeof(vi), cudaMemcpyDeviceToHost, g->stream));
    HYP_CUDA(cudaStreamSynchronize(g->stream));
    const int c = (int)(word >> kIdxBitsShift);
    const int64_t e = word ? (int64_t)vi.y << c : 0;
    *bits = word ? c : 0;
    *entries = e;
    if (!table || e == 0) return HYPERIM_OK;
    if (cap < e) return set_error(HYPERIM_EINVAL, "table buffer smaller than the index");
    const uint64_t off = word & ((1ull << kIdxBitsShift) - 1);
    HYP_CUDA(cudaMemcpyAsync(table, g->idx_tab + off, sizeof(uint32_t) * (size_t)e, cudaMemcpyDeviceToHost,
                             g->stream));
    HYP_CUDA(cudaStreamSynchronize(g->stream));
    return HYPERIM_OK;
}

hyperim_status hyperim_graph_set_schedule(hyperim_graph_t g, int32_t schedule) {
    if (!g) return set_error(HYPERIM_EINVAL, "null graph");
    if (schedule != HYPERIM_SCHED_PERSISTENT && schedule != HYPERIM_SCHED_PLAIN)
        return set_error(HYPERIM_EINVAL, "unknown schedule");
    g->schedule = schedule;
    return HYPERIM_OK;
}

hyperim_status hyperim_graph_set_tuning(hyperim_graph_t g, const hyperim_tuning* t) {
    if (!g || !t) return set_error(HYPERIM_EINVAL, "null argument");
    if (t->warp_set_limit < 0 || t->warp_set_limit > 128) return set_error(HYPERIM_EINVAL, "warp_set_limit outside [0, 128]");
    if (t->early_sets_per_block < 1 || t->early_sets_per_block > 4096)
        return set_error(HYPERIM_EINVAL, "early_sets_per_block outside [1, 4096]");
    if (t->arena_entries_per_set < 0 || t->arena_entries_per_set > (1 << 20))
        return set_error(HYPERIM_EINVAL, "arena_entries_per_set outside [0, 2^20]");
    g->warp_set_limit = t->warp_set_limit;
    g->early_sets_per_block = t->early_sets_per_block;
    g->arena_entries_per_set = t->arena_entries_per_set;
    return HYPERIM_OK;
}

hyperim_status hyperim_graph_get_tuning(hyperim_graph_t g, hyperim_tuning* out) {
    if (!g || !out) return set_error(HYPERIM_EINVAL, "null argument");
    out->warp_set_limit = g->warp_set_limit;
    out->early_sets_per_block = g->early_sets_per_block;
    out->arena_entries_per_set = g->arena_entries_per_set;
    return HYPERIM_OK;
}

static hyperim_status pool_create(hyperim_graph* g, uint32_t tag, int32_t root_mode, int32_t strategy,
                                  hyperim_pool** out);
static hyperim_status pool_grow(hyperim_graph* g, hyperim_pool* p, uint64_t theta);

namespace {
// the autotuner's key: the degree profile of the graph (logarithmic buckets) and the query kind
uint64_t profile_key(const hyperim_graph* g, int32_t root_mode, int32_t strategy) {
    auto lg = [](double x) { return x <= 1.0 ? 0ull : (unsigned long long)std::lround(std::log2(x) * 2.0); };
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the fields
    auto mix = [&h](uint64_t v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (v >> (8 * i)) & 0xFF;
            h *= 1099511628211ull;
        }
    };
    mix((uint64_t)g->model);
    mix(g->uniform_thr);
    mix((uint64_t)root_mode);
    mix((uint64_t)strategy);
    mix(lg((double)g->n));
    mix(lg((double)g->nnz));
    mix(lg((double)g->max_tsum));
    mix(lg((double)g->max_deg));
    for (int s = 0; s < HYPERIM_NSTRATA; ++s) mix(lg(64.0 * (double)g->stratum_size[s] / (double)g->n));
    return h;
}

std::mutex& tune_mutex() {
    static std::mutex m;
    return m;
}

// a cached choice, with the per-set SM cycles (mean, maximum) its candidate measured: a graph of
// the same profile starts with them, so BRR can grow ahead from its first launch
struct TuneEntry {
    hyperim_tuning t;
    double cycles_mean, cycles_max;
};
std::map<uint64_t, TuneEntry>& tune_cache() {
    static std::map<uint64_t, TuneEntry> c;
    return c;
}
}  // namespace

hyperim_status hyperim_graph_autotune(hyperim_graph_t g, int32_t root_mode, int32_t strategy, uint64_t sets,
                                      hyperim_autotune_result* out) {
    if (!g || !out) return set_error(HYPERIM_EINVAL, "null argument");
    if (root_mode != HYPERIM_ROOTS_PLAIN && root_mode != HYPERIM_ROOTS_STRATIFIED)
        return set_error(HYPERIM_EINVAL, "unknown root mode");
    if (strategy < HYPERIM_STRAT_PAPER || strategy > HYPERIM_STRAT_LT) return set_error(HYPERIM_EINVAL, "unknown strategy");
    std::memset(out, 0, sizeof(*out));
    const uint64_t key = profile_key(g, root_mode, strategy);
    out->profile_key = key;
    {
        std::lock_guard<std::mutex> lk(tune_mutex());
        auto it = tune_cache().find(key);
        if (it != tune_cache().end()) {
            hyperim_tuning t = it->second.t;
            t.early_sets_per_block = g->early_sets_per_block;
            t.arena_entries_per_set = g->arena_entries_per_set;
            g->warp_set_limit = t.warp_set_limit;
            if (g->set_cycles_mean <= 0.0) {
                g->set_cycles_mean = it->second.cycles_mean;
                g->set_cycles_max = it->second.cycles_max;
            }
            out->chosen = t;
            out->from_cache = 1;
            return HYPERIM_OK;
        }
    }
    if (sets == 0) sets = 8 * (uint64_t)std::max(g->sm_count, 1);
    const int32_t keep_w = g->warp_set_limit, keep_sched = g->schedule;
    g->schedule = HYPERIM_SCHED_PERSISTENT;
    const int32_t cand[5] = {0, 16, 32, 64, 128};  // warp-phase set limits (0: none)
    double best = -1.0, best_mean = 0.0, best_max = 0.0;
    hyperim_tuning choice{keep_w, g->early_sets_per_block, g->arena_entries_per_set};
    hyperim_status st = HYPERIM_OK;
    int c = 0;
    {
        for (int ci = 0; ci < 5 && st == HYPERIM_OK; ++ci) {
            g->warp_set_limit = cand[ci];
            double secs = -1.0, c_mean = 0.0, c_max = 0.0;
            for (int rep = 0; rep < 2 && st == HYPERIM_OK; ++rep) {
                hyperim_pool* p = nullptr;
                if ((st = pool_create(g, 0xFF, root_mode, strategy, &p))) break;
                {
                    std::unique_lock<std::shared_mutex> lk(p->mu);
                    st = pool_grow(g, p, sets);
                }
                const double t = p->rr_kernel_seconds;
                hyperim_pool_free(p);
                if (st == HYPERIM_OK && (secs < 0.0 || t < secs)) {
                    secs = t;
                    c_mean = g->set_cycles_mean;  // the growth's per-set cycles (block kernel's sets)
                    c_max = g->set_cycles_max;
                }
            }
            if (st != HYPERIM_OK) break;
            out->warp_set_limit[c] = cand[ci];
            out->seconds[c] = secs;
            ++c;
            if (best < 0.0 || secs < best) {
                best = secs;
                choice.warp_set_limit = cand[ci];
            }
            if (cand[ci] == 0) {  // every set on the block kernel: its cycles describe all of them
                best_mean = c_mean;
                best_max = c_max;
            }
        }
    }
    out->candidates = c;
    g->schedule = keep_sched;
    if (st != HYPERIM_OK) {
        g->warp_set_limit = keep_w;
        return st;
    }
    g->warp_set_limit = choice.warp_set_limit;
    if (best_mean > 0.0) {
        g->set_cycles_mean = best_mean;
        g->set_cycles_max = best_max;
    }
    out->chosen = choice;
    std::lock_guard<std::mutex> lk(tune_mutex());
    tune_cache()[key] = TuneEntry{choice, best_mean, best_max};
    return HYPERIM_OK;
}

hyperim_status hyperim_graph_set_wait_limit(hyperim_graph_t g, uint32_t iterations) {
    if (!g) return set_error(HYPERIM_EINVAL, "null graph");
    g->wait_limit = iterations;
    return HYPERIM_OK;
}

hyperim_status hyperim_graph_profile(hyperim_graph_t g, int32_t* deg, int32_t* nlayers, int32_t* stratum,
                                     int64_t* prof_off, uint32_t* layer_w, uint32_t* layer_n,
                                     uint64_t* layer_thr) {
    if (!g) return set_error(HYPERIM_EINVAL, "null graph");
    const size_t n = (size_t)g->n, L = (size_t)g->profile_entries;
    std::vector<int32_t> off(n + 1);
    std::vector<uint8_t> strat(n);
    std::vector<uint4> prof(2 * L);
    HYP_CUDA(cudaMemcpyAsync(off.data(), g->prof_off, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, g->stream));
    HYP_CUDA(cudaMemcpyAsync(strat.data(), g->stratum, n, cudaMemcpyDeviceToHost, g->stream));
    if (L) HYP_CUDA(cudaMemcpyAsync(prof.data(), g->prof, 2 * sizeof(uint4) * L, cudaMemcpyDeviceToHost, g->stream));
    if (deg) HYP_CUDA(cudaMemcpyAsync(deg, g->deg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, g->stream));
    HYP_CUDA(cudaStreamSynchronize(g->stream));
    for (size_t v = 0; v < n; ++v) {
        if (nlayers) nlayers[v] = off[v + 1] - off[v];
        if (stratum) stratum[v] = strat[v];
    }
    if (prof_off)
        for (size_t v = 0; v <= n; ++v) prof_off[v] = off[v];
    for (size_t x = 0; x < L; ++x) {
        const uint4 e = prof[2 * x];
        if (layer_w) layer_w[x] = e.x & ~kPOneFlag;
        if (layer_n) layer_n[x] = e.y;
        if (layer_thr) layer_thr[x] = (e.x & kPOneFlag) ? HYPERIM_P_ONE : (uint64_t)e.z;
    }
    return HYPERIM_OK;
}

hyperim_status hyperim_plan_theta(hyperim_graph_t g, int32_t k, double eps, double ell,
                                  hyperim_theta_plan* out) {
    if (!g || !out) return set_error(HYPERIM_EINVAL, "null argument");
    return plan_theta(g->n, k, eps, ell, out);
}

static hyperim_status pool_create(hyperim_graph* g, uint32_t tag, int32_t root_mode, int32_t strategy,
                                  hyperim_pool** out) {
    if (tag > 0xFF) return set_error(HYPERIM_EINVAL, "pool_tag must be < 256");
    if (root_mode != HYPERIM_ROOTS_PLAIN && root_mode != HYPERIM_ROOTS_STRATIFIED)
        return set_error(HYPERIM_EINVAL, "unknown root mode");
    if (strategy != HYPERIM_STRAT_PAPER && strategy != HYPERIM_STRAT_BINOMIAL_ONLY && strategy != HYPERIM_STRAT_LT)
        return set_error(HYPERIM_EINVAL, "unknown strategy");
    hyperim_pool* p = new (std::nothrow) hyperim_pool();
    if (!p) return set_error(HYPERIM_ENOMEM, "host allocation failed");
    p->g = graph_root(g);
    {
        // a pool keeps the loaded graph alive like a share does (g is a live handle of it)
        std::lock_guard<std::mutex> lk(graph_mutex());
        ++p->g->shares;
    }
    p->tag = tag;
    p->root_mode = root_mode;
    p->strategy = strategy;
    *out = p;
    return HYPERIM_OK;
}

// R1 and R2 of a BRR round grow by the same allocation: one launch generates both.
// theta_last > theta: the growth may go ahead to a later round's theta (doubling, at most
// theta_last) while the new sets' work per block would stay below the longest set of the
// handle's last launch -- such a launch lasts about as long as that set whatever it holds, so
// the later rounds' sets come at little cost, and a query that stops first wastes at most about
// one such tail. Rounds read only their own prefix views, so results never change.
static hyperim_status pool_grow_pair(hyperim_graph* g, hyperim_pool* r1, hyperim_pool* r2, uint64_t theta,
                                     uint64_t theta_last = 0) {
    uint64_t ns[2][HYPERIM_NSTRATA];
    hyperim_pool* pools[2] = {r1, r2};
    // growth is exclusive; the two locks are taken in address order
    std::unique_lock<std::shared_mutex> la(r1 < r2 ? r1->mu : r2->mu), lb(r1 < r2 ? r2->mu : r1->mu);
    auto new_sets = [&](uint64_t t) {
        uint64_t add = 0;
        for (int q = 0; q < 2; ++q) {
            allocate_strata(g, pools[q]->root_mode, t, ns[q]);
            for (int s = 0; s < HYPERIM_NSTRATA; ++s)
                add += ns[q][s] > pools[q]->n_s[s] ? ns[q][s] - pools[q]->n_s[s] : 0;
        }
        return add;
    };
    uint64_t add = new_sets(theta);
    if (add == 0) return HYPERIM_OK;  // an earlier query grew both pools past theta
    if (theta_last > theta && g->schedule == HYPERIM_SCHED_PERSISTENT && g->set_cycles_mean > 0.0) {
        const double blocks = (double)std::max(g->sm_count, 1);  // one RR block per SM
        while (theta < theta_last && (double)add * g->set_cycles_mean / blocks < g->set_cycles_max) {
            theta = std::min(theta_last, theta * 2);
            add = new_sets(theta);
        }
        new_sets(theta);
    }
    for (int q = 0; q < 2; ++q)
        for (int s = 0; s < HYPERIM_NSTRATA; ++s) ns[q][s] = std::max(ns[q][s], pools[q]->n_s[s]);
    return sample_rr_multi(g, pools, 2, ns);
}

static hyperim_status pool_grow(hyperim_graph* g, hyperim_pool* p, uint64_t theta) {
    uint64_t ns[HYPERIM_NSTRATA];
    allocate_strata(g, p->root_mode, theta, ns);
    for (int s = 0; s < HYPERIM_NSTRATA; ++s) ns[s] = std::max(ns[s], p->n_s[s]);
    return sample_rr(g, p, ns);
}

static hyperim_status sample_rr_shard(hyperim_graph_t g, uint32_t pool_tag, uint64_t theta, int32_t root_mode,
                                      int32_t strategy, int32_t rank, int32_t world, hyperim_pool_t* inout) {
    if (!g || !inout) return set_error(HYPERIM_EINVAL, "null argument");
    if (world < 1 || rank < 0 || rank >= world) return set_error(HYPERIM_EINVAL, "need 0 <= rank < world");
    hyperim_status st;
    bool created = false;
    if (!*inout) {
        if ((st = pool_create(g, pool_tag, root_mode, strategy, inout))) return st;
        (*inout)->shard_rank = rank;
        (*inout)->shard_world = world;
        created = true;
    } else {
        hyperim_pool* p = *inout;
        if (graph_root(p->g) != graph_root(g)) return set_error(HYPERIM_ESTATE, "pool belongs to another graph");
        if (p->tag != pool_tag || p->root_mode != root_mode || p->strategy != strategy)
            return set_error(HYPERIM_ESTATE, "pool was created with other tag/root mode/strategy");
        if (p->shard_rank != rank || p->shard_world != world)
            return set_error(HYPERIM_ESTATE, "pool was created as another shard");
    }
    {
        std::unique_lock<std::shared_mutex> lk((*inout)->mu);
        st = pool_grow(g, *inout, theta);
    }
    if (st != HYPERIM_OK && created) {
        std::string keep = g_last_error;
        hyperim_pool_free(*inout);
        *inout = nullptr;
        g_last_error = keep;
    }
    return st;
}

hyperim_status hyperim_sample_rr(hyperim_graph_t g, uint32_t pool_tag, uint64_t theta, int32_t root_mode,
                                 int32_t strategy, hyperim_pool_t* inout) {
    return sample_rr_shard(g, pool_tag, theta, root_mode, strategy, 0, 1, inout);
}

hyperim_status hyperim_sample_rr_shard(hyperim_graph_t g, uint32_t pool_tag, uint64_t theta, int32_t root_mode,
                                       int32_t strategy, int32_t rank, int32_t world, hyperim_pool_t* inout) {
    return sample_rr_shard(g, pool_tag, theta, root_mode, strategy, rank, world, inout);
}

void hyperim_pool_free(hyperim_pool_t p) {
    if (!p) return;
    hyperim_graph* g = p->g;
    dev_free(g, p->rr_off, sizeof(int64_t) * p->cap_off);
    dev_free(g, p->rr_mem, sizeof(int32_t) * p->cap_total);
    dev_free(g, p->rr_stratum, p->cap_stratum);
    dev_free(g, p->rr_j, sizeof(uint32_t) * p->cap_j);
    cudaStreamSynchronize(g->stream);
    delete p;
    release_root(g);
}

hyperim_status hyperim_pool_view(hyperim_pool_t p, hyperim_pool_view_t* out) {
    if (!p || !out) return set_error(HYPERIM_EINVAL, "null argument");
    std::shared_lock<std::shared_mutex> lk(p->mu);
    out->count = p->count;
    out->total = p->total;
    out->rr_off = p->rr_off;
    out->rr_mem = p->rr_mem;
    out->rr_stratum = p->rr_stratum;
    out->rr_j = p->rr_j;
    for (int s = 0; s < HYPERIM_NSTRATA; ++s) out->n_s[s] = p->n_s[s];
    out->pool_tag = p->tag;
    out->root_mode = p->root_mode;
    out->strategy = p->strategy;
    out->pops = p->counters.pops;
    out->layers_seen = p->counters.layers_seen;
    out->draws = p->counters.draws;
    out->mats = p->counters.mats;
    out->mat_he = p->counters.mat_he;
    out->mat_members = p->counters.mat_members;
    out->selected = p->counters.selected;
    out->gathered = p->counters.gathered;
    out->search_words = p->counters.search_words;
    out->rr_launches = p->rr_launches;
    out->rr_kernel_seconds = p->rr_kernel_seconds;
    out->sectors = p->counters.sectors;
    return HYPERIM_OK;
}

hyperim_status hyperim_pool_copy(hyperim_pool_t p, int64_t* rr_off, int32_t* rr_mem, uint8_t* rr_stratum,
                                 uint32_t* rr_j) {
    if (!p) return set_error(HYPERIM_EINVAL, "null pool");
    std::shared_lock<std::shared_mutex> lk(p->mu);
    cudaStream_t s = p->g->stream;
    const size_t N = (size_t)p->count, T = (size_t)p->total;
    if (rr_off) {
        if (N) HYP_CUDA(cudaMemcpyAsync(rr_off, p->rr_off, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToHost, s));
        else rr_off[0] = 0;
    }
    if (rr_mem && T) HYP_CUDA(cudaMemcpyAsync(rr_mem, p->rr_mem, sizeof(int32_t) * T, cudaMemcpyDeviceToHost, s));
    if (rr_stratum && N) HYP_CUDA(cudaMemcpyAsync(rr_stratum, p->rr_stratum, N, cudaMemcpyDeviceToHost, s));
    if (rr_j && N) HYP_CUDA(cudaMemcpyAsync(rr_j, p->rr_j, sizeof(uint32_t) * N, cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    return HYPERIM_OK;
}

hyperim_status hyperim_select_seeds(hyperim_graph_t g, hyperim_pool_t r1, hyperim_pool_t r2, int32_t k,
                                    const hyperim_select_opts* opts, int32_t* seeds_host,
                                    hyperim_select_result* out) {
    if (!g || !r1 || !opts || !seeds_host || !out) return set_error(HYPERIM_EINVAL, "null argument");
    if (k < 1 || k > g->n) return set_error(HYPERIM_EINVAL, "need 1 <= k <= n");
    if (graph_root(r1->g) != graph_root(g) || (r2 && graph_root(r2->g) != graph_root(g)))
        return set_error(HYPERIM_ESTATE, "pool of another graph");
    if (r1 == r2) return set_error(HYPERIM_ESTATE, "r1 and r2 must be distinct pools");
    if (opts->upper_mode != HYPERIM_UPPER_CLOSED && opts->upper_mode != HYPERIM_UPPER_PREFIX)
        return set_error(HYPERIM_EINVAL, "unknown upper bound mode");
    std::memset(out, 0, sizeof(*out));
    hyperim_status st;
    using clk = std::chrono::steady_clock;
    double t_sample = 0.0, t_select = 0.0;
    const bool prefix = opts->upper_mode == HYPERIM_UPPER_PREFIX;
    uint64_t pu[2] = {0, 0};
    if (opts->mode == HYPERIM_SELECT_FIXED) {
        auto t0 = clk::now();
        {
            std::shared_lock<std::shared_mutex> lk(r1->mu);
            if ((st = greedy(g, r1, k, seeds_host, out->lambda_r1, prefix ? pu : nullptr))) return st;
        }
        out->sigma_r1 = estimate(g, r1->root_mode, r1->n_s, out->lambda_r1);
        if (prefix) out->upper = prefix_upper_sigma(pu, r1->root_mode, g->n, (uint64_t)r1->count);
        if (r2) {
            std::shared_lock<std::shared_mutex> lk(r2->mu);
            if ((st = coverage(g, r2, seeds_host, k, out->lambda_r2))) return st;
            out->sigma_r2 = estimate(g, r2->root_mode, r2->n_s, out->lambda_r2);
        }
        t_select = std::chrono::duration<double>(clk::now() - t0).count();
        out->rounds = 1;
        out->pool_r1 = (uint64_t)r1->count;
        out->pool_r2 = r2 ? (uint64_t)r2->count : 0;
        out->seconds_select = t_select;
        return HYPERIM_OK;
    }
    if (opts->mode != HYPERIM_SELECT_BRR) return set_error(HYPERIM_EINVAL, "unknown select mode");
    if (!r2) return set_error(HYPERIM_EINVAL, "BRR needs two pools");
    if (r1->root_mode != r2->root_mode || r1->strategy != r2->strategy)
        return set_error(HYPERIM_ESTATE, "r1 and r2 differ in root mode or strategy");
    hyperim_theta_plan plan;
    if ((st = plan_theta(g->n, k, opts->eps, opts->ell, &plan))) return st;
    const double target = 1.0 - std::exp(-1.0) - opts->eps;
    // Early rounds need few sets, and a launch of few sets lasts as long as its slowest set: the
    // pools are grown to at least theta_early per pool (four sets per resident block of the RR
    // kernel for R1 and R2 together) so that those rounds share one launch. Rounds read only
    // their own prefix, so the result is the same; sets beyond the last round's theta are
    // generated but unused when BRR stops before theta_early.
    uint64_t theta_early = (uint64_t)std::max(g->early_sets_per_block, 1) * (uint64_t)std::max(g->sm_count, 1);
    if (plan.i_max < 40) theta_early = std::min<uint64_t>(theta_early, plan.theta0 << plan.i_max);
    if (opts->theta_cap) theta_early = std::min<uint64_t>(theta_early, opts->theta_cap);
    // the largest theta a round of this query can ask for (growth never goes past it)
    uint64_t theta_last = plan.i_max < 62 ? plan.theta0 << plan.i_max : (uint64_t)1 << 62;
    if (opts->theta_cap) theta_last = std::min<uint64_t>(theta_last, opts->theta_cap);
    for (int32_t i = 0;; ++i) {
        if (i > 62) return set_error(HYPERIM_EOVERFLOW, "theta doubling overflow");
        const uint64_t theta = plan.theta0 << i;
        if (opts->theta_cap && theta > opts->theta_cap)
            return set_error(HYPERIM_EOVERFLOW, "theta_i = " + std::to_string(theta) + " exceeds theta_cap");
        // round i works on the sets a pool grown to theta_i holds (a prefix by (s, j) of pools
        // that an earlier query grew further, so the result does not depend on that history)
        uint64_t v1[HYPERIM_NSTRATA], v2[HYPERIM_NSTRATA];
        allocate_strata(g, r1->root_mode, theta, v1);
        allocate_strata(g, r2->root_mode, theta, v2);
        auto t0 = clk::now();
        if ((st = pool_grow_pair(g, r1, r2, std::max(theta, theta_early), theta_last))) return st;
        auto t1 = clk::now();
        {
            std::shared_lock<std::shared_mutex> lk(r1->mu);
            if ((st = greedy(g, r1, k, seeds_host, out->lambda_r1, prefix ? pu : nullptr, v1))) return st;
        }
        {
            std::shared_lock<std::shared_mutex> lk(r2->mu);
            if ((st = coverage(g, r2, seeds_host, k, out->lambda_r2, v2))) return st;
        }
        auto t2 = clk::now();
        t_sample += std::chrono::duration<double>(t1 - t0).count();
        t_select += std::chrono::duration<double>(t2 - t1).count();
        uint64_t N1 = 0, N2 = 0;
        for (int s = 0; s < HYPERIM_NSTRATA; ++s) {
            N1 += v1[s];
            N2 += v2[s];
        }
        const double s1 = estimate(g, r1->root_mode, v1, out->lambda_r1);
        const double s2 = estimate(g, r2->root_mode, v2, out->lambda_r2);
        const double lam1 = s1 * (double)N1 / (double)g->n;
        const double lam2 = s2 * (double)N2 / (double)g->n;
        const double up = prefix ? prefix_upper_sigma(pu, r1->root_mode, g->n, N1) : upper_bound(lam1, k, g->n, N1);
        const double lo = lower_bound(lam2, plan.delta, g->n, N2);
        const double alpha = lo / up;
        out->rounds = i + 1;
        out->theta = theta;
        out->pool_r1 = N1;
        out->pool_r2 = N2;
        out->sigma_r1 = s1;
        out->sigma_r2 = s2;
        out->upper = up;
        out->lower = lo;
        out->alpha = alpha;
        if (i < 64) out->alpha_round[i] = alpha;
        if (alpha >= target || i >= plan.i_max) break;
    }
    out->seconds_sample = t_sample;
    out->seconds_select = t_select;
    return HYPERIM_OK;
}

hyperim_status hyperim_select_seeds_batch(const hyperim_batch_query* queries, int32_t nq) {
    if (!queries || nq < 1) return set_error(HYPERIM_EINVAL, "need at least one query");
    hyperim_status st;
    struct QS {
        hyperim_theta_plan plan;
        bool running;
        double t_sample, t_select;
    };
    std::vector<QS> qs((size_t)nq);
    std::vector<hyperim_pool*> pools;
    for (int32_t q = 0; q < nq; ++q) {
        const hyperim_batch_query& Q = queries[q];
        if (!Q.graph || !Q.r1 || !Q.r2 || !Q.seeds_host || !Q.result) return set_error(HYPERIM_EINVAL, "null argument");
        if (Q.k < 1 || Q.k > Q.graph->n) return set_error(HYPERIM_EINVAL, "need 1 <= k <= n");
        if (graph_root(Q.r1->g) != graph_root(Q.graph) || graph_root(Q.r2->g) != graph_root(Q.graph))
            return set_error(HYPERIM_ESTATE, "pool of another graph");
        if (Q.r1 == Q.r2) return set_error(HYPERIM_ESTATE, "r1 and r2 must be distinct pools");
        if (Q.r1->root_mode != Q.r2->root_mode || Q.r1->strategy != Q.r2->strategy)
            return set_error(HYPERIM_ESTATE, "r1 and r2 differ in root mode or strategy");
        if ((st = plan_theta(Q.graph->n, Q.k, Q.eps, Q.ell, &qs[q].plan))) return st;
        qs[q].running = true;
        qs[q].t_sample = qs[q].t_select = 0.0;
        std::memset(Q.result, 0, sizeof(*Q.result));
        for (hyperim_pool* p : {Q.r1, Q.r2})
            if (std::find(pools.begin(), pools.end(), p) == pools.end()) pools.push_back(p);
    }
    // every pool held exclusively for the call, locks taken in address order
    std::sort(pools.begin(), pools.end());
    std::vector<std::unique_lock<std::shared_mutex>> locks;
    locks.reserve(pools.size());
    for (hyperim_pool* p : pools) locks.emplace_back(p->mu);
    hyperim_graph* g0 = queries[0].graph;
    {
        std::vector<cudaStream_t> streams;
        for (int32_t q = 0; q < nq; ++q)
            if (std::find(streams.begin(), streams.end(), queries[q].graph->stream) == streams.end())
                streams.push_back(queries[q].graph->stream);
        for (cudaStream_t x : streams) HYP_CUDA(cudaStreamSynchronize(x));
    }
    using clk = std::chrono::steady_clock;
    std::vector<uint64_t> v1((size_t)nq * HYPERIM_NSTRATA), v2((size_t)nq * HYPERIM_NSTRATA);
    std::vector<uint64_t> target(pools.size() * HYPERIM_NSTRATA);
    std::vector<hyperim_graph*> pool_graph(pools.size());
    for (int32_t i = 0;; ++i) {
        std::vector<int32_t> run;
        for (int32_t q = 0; q < nq; ++q)
            if (qs[q].running) run.push_back(q);
        if (run.empty()) break;
        if (i > 62) return set_error(HYPERIM_EOVERFLOW, "theta doubling overflow");
        // growth targets: each pool to the largest allocation a running query reads from it
        for (size_t x = 0; x < pools.size(); ++x)
            for (int s = 0; s < HYPERIM_NSTRATA; ++s) target[x * HYPERIM_NSTRATA + s] = pools[x]->n_s[s];
        for (int32_t q : run) {
            const hyperim_batch_query& Q = queries[q];
            const uint64_t theta = qs[q].plan.theta0 << i;
            uint64_t* a1 = &v1[(size_t)q * HYPERIM_NSTRATA];
            uint64_t* a2 = &v2[(size_t)q * HYPERIM_NSTRATA];
            allocate_strata(Q.graph, Q.r1->root_mode, theta, a1);
            allocate_strata(Q.graph, Q.r2->root_mode, theta, a2);
            const size_t x1 = (size_t)(std::lower_bound(pools.begin(), pools.end(), Q.r1) - pools.begin());
            const size_t x2 = (size_t)(std::lower_bound(pools.begin(), pools.end(), Q.r2) - pools.begin());
            pool_graph[x1] = Q.graph;
            pool_graph[x2] = Q.graph;
            for (int s = 0; s < HYPERIM_NSTRATA; ++s) {
                target[x1 * HYPERIM_NSTRATA + s] = std::max(target[x1 * HYPERIM_NSTRATA + s], a1[s]);
                target[x2 * HYPERIM_NSTRATA + s] = std::max(target[x2 * HYPERIM_NSTRATA + s], a2[s]);
            }
        }
        // one group per graph and pair of pools (same root mode and strategy) that must grow
        std::vector<RRGroup> groups;
        for (size_t x = 0; x < pools.size(); ++x) {
            hyperim_pool* p = pools[x];
            bool grow = false;
            for (int s = 0; s < HYPERIM_NSTRATA; ++s) grow = grow || target[x * HYPERIM_NSTRATA + s] > p->n_s[s];
            if (!grow) continue;
            RRGroup* G = nullptr;
            for (RRGroup& c : groups)
                if (c.npools == 1 && graph_root(c.g) == graph_root(p->g) && c.pools[0]->root_mode == p->root_mode &&
                    c.pools[0]->strategy == p->strategy) {
                    G = &c;
                    break;
                }
            if (!G) {
                groups.push_back(RRGroup{});
                G = &groups.back();
                G->g = pool_graph[x];
                G->npools = 0;
            }
            G->pools[G->npools] = p;
            for (int s = 0; s < HYPERIM_NSTRATA; ++s) G->new_ns[G->npools][s] = target[x * HYPERIM_NSTRATA + s];
            ++G->npools;
        }
        auto t0 = clk::now();
        if (!groups.empty() && (st = sample_rr_batch(g0, groups.data(), (int)groups.size(), nullptr))) return st;
        auto t1 = clk::now();
        std::vector<GreedyBatchItem> items;
        std::vector<int32_t> seeds;
        std::vector<uint64_t> lam((size_t)run.size() * 2 * HYPERIM_NSTRATA);
        size_t seeds_total = 0;
        for (int32_t q : run) seeds_total += (size_t)queries[q].k;
        seeds.resize(seeds_total);
        size_t at = 0;
        for (size_t r = 0; r < run.size(); ++r) {
            const int32_t q = run[r];
            const hyperim_batch_query& Q = queries[q];
            GreedyBatchItem it;
            it.g = Q.graph;
            it.r1 = Q.r1;
            it.r2 = Q.r2;
            it.lim1 = &v1[(size_t)q * HYPERIM_NSTRATA];
            it.lim2 = &v2[(size_t)q * HYPERIM_NSTRATA];
            it.k = Q.k;
            it.seeds_host = seeds.data() + at;
            it.lambda_r1 = &lam[r * 2 * HYPERIM_NSTRATA];
            it.lambda_r2 = &lam[r * 2 * HYPERIM_NSTRATA + HYPERIM_NSTRATA];
            items.push_back(it);
            at += (size_t)Q.k;
        }
        if ((st = greedy_batch(g0, items.data(), (int)items.size()))) return st;
        auto t2 = clk::now();
        const double ds = std::chrono::duration<double>(t1 - t0).count();
        const double dg = std::chrono::duration<double>(t2 - t1).count();
        for (size_t r = 0; r < run.size(); ++r) {
            const int32_t q = run[r];
            const hyperim_batch_query& Q = queries[q];
            const GreedyBatchItem& it = items[r];
            hyperim_select_result* out = Q.result;
            const hyperim_theta_plan& plan = qs[q].plan;
            const hyperim_graph* g = Q.graph;
            const uint64_t* a1 = &v1[(size_t)q * HYPERIM_NSTRATA];
            const uint64_t* a2 = &v2[(size_t)q * HYPERIM_NSTRATA];
            std::memcpy(Q.seeds_host, it.seeds_host, sizeof(int32_t) * (size_t)Q.k);
            uint64_t N1 = 0, N2 = 0;
            for (int s = 0; s < HYPERIM_NSTRATA; ++s) {
                out->lambda_r1[s] = it.lambda_r1[s];
                out->lambda_r2[s] = it.lambda_r2[s];
                N1 += a1[s];
                N2 += a2[s];
            }
            const double s1 = estimate(g, Q.r1->root_mode, a1, out->lambda_r1);
            const double s2 = estimate(g, Q.r2->root_mode, a2, out->lambda_r2);
            const double up = upper_bound(s1 * (double)N1 / (double)g->n, Q.k, g->n, N1);
            const double lo = lower_bound(s2 * (double)N2 / (double)g->n, plan.delta, g->n, N2);
            const double alpha = lo / up;
            out->rounds = i + 1;
            out->theta = plan.theta0 << i;
            out->pool_r1 = N1;
            out->pool_r2 = N2;
            out->sigma_r1 = s1;
            out->sigma_r2 = s2;
            out->upper = up;
            out->lower = lo;
            out->alpha = alpha;
            if (i < 64) out->alpha_round[i] = alpha;
            qs[q].t_sample += ds;
            qs[q].t_select += dg;
            out->seconds_sample = qs[q].t_sample;
            out->seconds_select = qs[q].t_select;
            if (alpha >= 1.0 - std::exp(-1.0) - Q.eps || i >= plan.i_max) qs[q].running = false;
        }
    }
    return HYPERIM_OK;
}

}  // extern "C"

struct hyperim_greedy {
    hyperim::GreedyState* st = nullptr;
};

extern "C" {

hyperim_status hyperim_greedy_begin(hyperim_graph_t g, hyperim_pool_t pool, uint64_t theta, hyperim_greedy_t* out) {
    if (!g || !pool || !out) return set_error(HYPERIM_EINVAL, "null argument");
    *out = nullptr;
    if (graph_root(pool->g) != graph_root(g)) return set_error(HYPERIM_ESTATE, "pool of another graph");
    uint64_t lim[HYPERIM_NSTRATA];
    if (theta) allocate_strata(g, pool->root_mode, theta, lim);
    hyperim_greedy* h = new (std::nothrow) hyperim_greedy();
    if (!h) return set_error(HYPERIM_ENOMEM, "host allocation failed");
    hyperim_status st = greedy_begin(g, pool, theta ? lim : nullptr, &h->st);
    if (st != HYPERIM_OK) {
        delete h;
        return st;
    }
    *out = h;
    return HYPERIM_OK;
}

hyperim_status hyperim_greedy_scores(hyperim_greedy_t s, uint64_t* dev_out) {
    if (!s || !dev_out) return set_error(HYPERIM_EINVAL, "null argument");
    return greedy_scores(s->st, reinterpret_cast<unsigned long long*>(dev_out));
}

hyperim_status hyperim_greedy_pick(hyperim_greedy_t s, const uint64_t* dev_total, int32_t* picked) {
    if (!s || !picked) return set_error(HYPERIM_EINVAL, "null argument");
    return greedy_pick(s->st, reinterpret_cast<const unsigned long long*>(dev_total), picked);
}

hyperim_status hyperim_greedy_end(hyperim_greedy_t s, uint64_t lambda_s[HYPERIM_NSTRATA]) {
    if (!s) return set_error(HYPERIM_EINVAL, "null argument");
    hyperim_status st = greedy_end(s->st, lambda_s);
    delete s;
    return st;
}

hyperim_status hyperim_coverage_view(hyperim_graph_t g, hyperim_pool_t pool, uint64_t theta, const int32_t* seeds_host,
                                     int32_t k, uint64_t lambda_s[HYPERIM_NSTRATA]) {
    if (!g || !pool || !lambda_s || (k > 0 && !seeds_host) || k < 0) return set_error(HYPERIM_EINVAL, "null argument");
    if (graph_root(pool->g) != graph_root(g)) return set_error(HYPERIM_ESTATE, "pool of another graph");
    for (int32_t i = 0; i < k; ++i)
        if (seeds_host[i] < 0 || seeds_host[i] >= g->n) return set_error(HYPERIM_EINVAL, "seed outside [0, n)");
    uint64_t lim[HYPERIM_NSTRATA];
    if (theta) allocate_strata(g, pool->root_mode, theta, lim);
    std::shared_lock<std::shared_mutex> lk(pool->mu);
    return coverage(g, pool, seeds_host, k, lambda_s, theta ? lim : nullptr);
}

hyperim_status hyperim_brr_round(hyperim_graph_t g, int32_t k, double eps, double ell, int32_t root_mode, int32_t round,
                                 const uint64_t lambda_r1[HYPERIM_NSTRATA], const uint64_t lambda_r2[HYPERIM_NSTRATA],
                                 hyperim_brr_round_t* out) {
    if (!g || !lambda_r1 || !lambda_r2 || !out) return set_error(HYPERIM_EINVAL, "null argument");
    if (root_mode != HYPERIM_ROOTS_PLAIN && root_mode != HYPERIM_ROOTS_STRATIFIED)
        return set_error(HYPERIM_EINVAL, "unknown root mode");
    if (round < 0 || round > 62) return set_error(HYPERIM_EINVAL, "round outside [0, 62]");
    hyperim_theta_plan plan;
    hyperim_status st;
    if ((st = plan_theta(g->n, k, eps, ell, &plan))) return st;
    const uint64_t theta = plan.theta0 << round;
    uint64_t ns[HYPERIM_NSTRATA];
    allocate_strata(g, root_mode, theta, ns);
    uint64_t N = 0;
    for (int s = 0; s < HYPERIM_NSTRATA; ++s) N += ns[s];
    const double s1 = estimate(g, root_mode, ns, lambda_r1);
    const double s2 = estimate(g, root_mode, ns, lambda_r2);
    const double lam1 = s1 * (double)N / (double)g->n;
    const double lam2 = s2 * (double)N / (double)g->n;
    out->theta = theta;
    out->sigma_r1 = s1;
    out->sigma_r2 = s2;
    out->upper = upper_bound(lam1, k, g->n, N);
    out->lower = lower_bound(lam2, plan.delta, g->n, N);
    out->alpha = out->lower / out->upper;
    out->stop = (out->alpha >= 1.0 - std::exp(-1.0) - eps || round >= plan.i_max) ? 1 : 0;
    return HYPERIM_OK;
}

hyperim_status hyperim_spread(hyperim_graph_t g, const int32_t* seeds_host, int32_t k, hyperim_pool_t pool,
                              double* sigma_hat, double* std_err) {
    if (!g || !pool || (k > 0 && !seeds_host)) return set_error(HYPERIM_EINVAL, "null argument");
    if (graph_root(pool->g) != graph_root(g)) return set_error(HYPERIM_ESTATE, "pool of another graph");
    if (k < 0) return set_error(HYPERIM_EINVAL, "k must be >= 0");
    for (int32_t i = 0; i < k; ++i)
        if (seeds_host[i] < 0 || seeds_host[i] >= g->n) return set_error(HYPERIM_EINVAL, "seed outside [0, n)");
    uint64_t lam[HYPERIM_NSTRATA];
    std::shared_lock<std::shared_mutex> lk(pool->mu);
    hyperim_status st = coverage(g, pool, seeds_host, k, lam);
    if (st) return st;
    const double sigma = estimate(g, pool->root_mode, pool->n_s, lam);
    double var = 0.0;
    for (int s = 0; s < HYPERIM_NSTRATA; ++s) {
        if (pool->n_s[s] == 0) continue;
        const double vs = pool->root_mode == HYPERIM_ROOTS_PLAIN ? (double)g->n : (double)g->stratum_size[s];
        const double ns = (double)pool->n_s[s];
        const double f = (double)lam[s] / ns;
        const double wgt = vs / ns;
        var += wgt * wgt * ns * f * (1.0 - f);
    }
    if (sigma_hat) *sigma_hat = sigma;
    if (std_err) *std_err = std::sqrt(var);
    return HYPERIM_OK;
}

}  // extern "C"
