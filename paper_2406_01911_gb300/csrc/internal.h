// Internal structures of the HyperIM CUDA library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <shared_mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/hyperim.h"

namespace hyperim {

// Device-side error word: the first kernel to fail stores its code (and a detail value).
enum DevErr : int32_t {
    kErrNone = 0,
    kErrBadMember = 1,     // member id outside [0, n)
    kErrBadOffsets = 2,    // he_off not monotone
    kErrProfile = 3,       // layer sizes inconsistent with the profile
    kErrWords = 4,         // a layer draw needed more than 2^18 Philox words
    kErrCapacity = 5,      // a scratch capacity was exceeded
    kErrBucket = 6,        // id bucket larger than the on-chip buffer
    kErrSpin = 7,          // a bounded wait of the RR kernel's work queue ran out
};

struct DevStatus {
    int32_t code;
    int32_t detail;
    uint64_t arena_need;   // bytes of RR output requested by the last generation launch
};

// Work counters of RR generation (same definitions as the pool view's counters).
struct RRCounters {
    unsigned long long pops, layers_seen, draws, mats, mat_he, mat_members, selected;
    unsigned long long gathered, search_words;
    unsigned long long sectors;  // 32-byte sectors of the method's own data (pool view: sectors)
};

// Chunk index of large neighbourhoods. The ids are split into C = 2^c chunks by their top c of
// id_bits bits, and the index stores, for every layer i of A(mu) and chunk k, the number of
// members of L_i in chunks < k (l_mu x C uint32, layer-major). The position of a pick in L_i
// then names the one chunk that holds it, and only that id range of mu's (sorted) hyperedges is
// read. Which vertices get one, and how large their chunks are, depends on lambda_mu = sum_i
// n_i p_i, the expected number of picks per pop (decided exactly on the integers
// sum_i n_i floor(p_i 2^32) against kIdxFewPicks 2^32):
//   lambda < kIdxFewPicks : indexed when mu's hyperedges hold more than kIdxMinT members besides
//                           mu (repeats counted); chunks of at most kIdxTargetFew members;
//   otherwise             : indexed above kIdxMinTMany members (below that one warp sorts the
//                           whole neighbourhood more cheaply than it visits most of its chunks);
//                           chunks of at most kIdxTargetMany members.
// c is the fewest bits for which no chunk exceeds the target. Vertices with more than kIdxMaxL
// layers, or whose members crowd one id range beyond the target even at 2^kIdxMaxBits chunks,
// are not indexed.
constexpr int kIdxMinT = 1024;
constexpr int kIdxMinTMany = 2048;
constexpr int kIdxTargetFew = 512;
constexpr int kIdxTargetMany = 1024;
constexpr int kIdxTarget = kIdxTargetMany;  // the largest chunk any index holds
constexpr unsigned long long kIdxFewPicks = 4;
constexpr int kIdxMaxBits = 12;
constexpr int kIdxMaxL = 1024;
// idx word of a vertex: 0 = no index, else (c << 56) | offset of its table
constexpr int kIdxBitsShift = 56;

// Id directory of a hyperedge (a lookup structure over its sorted member list): for a hyperedge
// of L members, kDirMinLen < L <= kDirMaxLen, with b = ceil(log2 L) bits (1 <= b <= min(id bits,
// kDirMaxBits)), D[r] (r = 0..2^b) is the number of members whose top b id bits are < r. The
// members whose top c id bits equal k (one chunk of the chunk index) are then positions
// [D[k 2^(b-c)], D[(k+1) 2^(b-c)]) when c <= b, or a sub-range of [D[r], D[r + 1]), r = k >>
// (c - b), when c > b (about one member on average). Entries are uint16 (L < 2^16).
constexpr int kDirMinLen = 16;
constexpr int kDirMaxLen = 65535;
constexpr int kDirMaxBits = 12;

// Profile entry of layer i of A(mu): 32 bytes, two uint4.
//   [0] = {w_i | (p == 1 ? 1u << 31 : 0), n_i, floor(p 2^32) for 0 <= p < 1, T_0}
//   [1] = {offset of the layer's CDF table, table length L, Poisson parts c, kind}
// kind 0: no draw (p = 0 or p = 1); 1: Binomial (n_i <= 20); 2: Poisson with c parts of lambda/c
// (the paper's strategy for n_i > 20). The table holds the inversion's thresholds T_0..T_{L-1}
// (capped at 2^32 - 1), computed at load by the same IEEE sequence as the inversion: a draw below
// some T_k is decided by a table search; only draws beyond the table's last entry (a tail of
// probability < 2^-16) run the double-precision inversion.
constexpr uint32_t kPOneFlag = 0x80000000u;

struct Scratch {
    // per resident block of the RR kernel
    int blocks = 0;
    size_t list_cap = 0;         // entries per block (>= n)
    size_t bitmap_words = 0;     // words per block of the global visited bitmap (0 if on-chip)
    size_t big_cap = 0;          // entries per block for bucketed neighbourhoods
    size_t pick_cap = 0;         // entries per block for picks
    int32_t* list = nullptr;
    uint32_t* bitmap = nullptr;
    uint32_t* big = nullptr;
    uint32_t* picks = nullptr;
    // output arena
    int32_t* arena = nullptr;
    size_t arena_cap = 0;        // entries
};

}  // namespace hyperim

struct hyperim_graph {
    int32_t n = 0, m = 0;
    int64_t nnz = 0;
    int32_t model = 0;
    uint64_t uniform_thr = 0;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0;
    std::atomic<size_t> device_bytes{0};  // on the loaded graph: all handles of it together
    int id_bits = 1;             // ceil(log2 n)
    // incidence store
    int32_t* he_off = nullptr;   // m + 1
    int32_t* he_mem = nullptr;   // nnz, sorted within each hyperedge
    int32_t* v_off = nullptr;    // n + 1
    int32_t* v_he = nullptr;     // nnz, ascending hyperedge ids per vertex
    int32_t* tsum = nullptr;     // n: sum of |he| over he containing v
    int2* v_span = nullptr;      // nnz: {he_off[he], |he|} for each incidence, in v_he order
    int4* vinfo = nullptr;       // n: {profile begin, l, incidence begin, d_H}
    // layer profile
    int32_t* prof_off = nullptr; // n + 1
    uint4* prof = nullptr;       // profile entries (two uint4 per layer)
    uint32_t* cdf_tab = nullptr; // CDF threshold tables of all layers
    int64_t table_entries = 0;
    int32_t* deg = nullptr;      // n
    uint8_t* stratum = nullptr;  // n
    int32_t* vs_off = nullptr;   // 17
    int32_t* vs_list = nullptr;  // n (vertices grouped by stratum, ascending id)
    // chunk index of large neighbourhoods
    uint64_t* idx = nullptr;     // n: 0 or (chunk bits << 56) | table offset
    uint32_t* idx_tab = nullptr; // per indexed vertex: l x 2^bits prefix counts, layer-major
    int64_t idx_entries = 0;
    int32_t idx_vertices = 0;
    // host copies of scalars
    int64_t profile_entries = 0;
    int32_t max_layers = 0, max_dh = 0;
    int64_t max_deg = 0, max_tsum = 0, max_layer_n = 0;
    int64_t stratum_size[HYPERIM_NSTRATA] = {};
    double theta_lstar = 0.0;
    // device status + scratch
    hyperim::DevStatus* d_status = nullptr;
    hyperim::RRCounters* d_counters = nullptr;
    hyperim::Scratch scratch;
    int sm_count = 0;
    int32_t schedule = 0;        // hyperim_schedule of RR generation
    uint32_t wait_limit = 0;     // iterations of a bounded device wait (0: the default)
    int32_t warp_set_limit = 0;  // RR sets up to this size are built by one warp (0: no warp phase)
    int32_t early_sets_per_block = 4;  // BRR's first launch: sets per resident block and pool
    double set_size_hint = 0.0;  // mean RR-set size of this handle's last growth (0: none yet)
    int32_t arena_entries_per_set = 0;  // tuning: initial output arena per new set (0: automatic)
    // per-set SM cycles of this handle's last persistent RR launch (mean, maximum; 0: none yet)
    double set_cycles_mean = 0.0, set_cycles_max = 0.0;
    // caller's device allocator (hyperim_load_args); null: stream-ordered cudaMallocAsync
    void* (*alloc_fn)(size_t, void*, void*) = nullptr;
    void (*free_fn)(void*, void*, void*) = nullptr;
    void* alloc_ctx = nullptr;
    uint32_t* mat_sect = nullptr; // n: sectors of v_he(v) plus those of every mem(he), he in v
    uint16_t* he_dir = nullptr;  // id directories of the hyperedges that have one
    uint2* v_dir = nullptr;      // nnz, in v_he order: {directory offset, b} (b = 0: none)
    int64_t dir_entries = 0;
    // handles made by hyperim_graph_share point at the loaded graph, whose device data they read;
    // it is released once it has been freed and no share is left
    hyperim_graph* owner = nullptr;
    int shares = 0;              // live shares and pools of the loaded graph, under hyperim::graph_mutex()
    bool freed = false;
};

struct hyperim_pool {
    hyperim_graph* g = nullptr;
    uint32_t tag = 0;
    int32_t root_mode = 0, strategy = 0;
    int32_t shard_rank = 0, shard_world = 1;  // a shard holds the sets (s, j) with j = rank (mod world)
    uint64_t n_s[HYPERIM_NSTRATA] = {};       // the allocation it covers (every shard: all of it)
    int64_t count = 0, total = 0;
    size_t cap_off = 0, cap_stratum = 0, cap_j = 0, cap_total = 0;  // allocated entries
    int64_t* rr_off = nullptr;      // count + 1
    int32_t* rr_mem = nullptr;      // total
    uint8_t* rr_stratum = nullptr;  // count
    uint32_t* rr_j = nullptr;       // count
    hyperim::RRCounters counters = {};
    uint64_t rr_launches = 0;
    double rr_kernel_seconds = 0.0;
    double mean_size_hint = 0.0;
    // growth takes it exclusively, readers (greedy, coverage, views) shared: handles of one graph
    // may use a pool from several host threads
    std::shared_mutex mu;
};

namespace hyperim {

// the loaded graph behind a handle (itself, or the graph a share was made from)
inline hyperim_graph* graph_root(hyperim_graph* g) { return g->owner ? g->owner : g; }
inline const hyperim_graph* graph_root(const hyperim_graph* g) { return g->owner ? g->owner : g; }
std::mutex& graph_mutex();

// launch accounting (capi.cu): every kernel launch of the library goes through count_launch()
void count_launch(uint64_t k = 1);

// error handling (capi.cu)
hyperim_status set_error(hyperim_status st, const std::string& msg);
hyperim_status cuda_fail(cudaError_t e, const char* what);
#define HYP_CUDA(call)                                                  \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::hyperim::cuda_fail(e_, #call);  \
    } while (0)

// device memory (capi.cu): stream-ordered allocation accounted against the graph's budget,
// through the caller's allocator when the graph was loaded with one
hyperim_status dev_alloc(hyperim_graph* g, void** p, size_t bytes);
void dev_free(hyperim_graph* g, void* p, size_t bytes);

// Device buffers of one call: every allocation made through it is released (stream-ordered)
// when it goes out of scope, on every return path of the call.
class CallBuffers {
  public:
    explicit CallBuffers(hyperim_graph* g) : g_(g) {}
    CallBuffers(const CallBuffers&) = delete;
    CallBuffers& operator=(const CallBuffers&) = delete;
    ~CallBuffers() {
        for (auto it = bufs_.rbegin(); it != bufs_.rend(); ++it) dev_free(g_, it->first, it->second);
    }
    template <typename T>
    hyperim_status alloc(T** p, size_t bytes) {
        hyperim_status st = dev_alloc(g_, reinterpret_cast<void**>(p), bytes);
        if (st == HYPERIM_OK) bufs_.emplace_back(static_cast<void*>(*p), bytes);
        return st;
    }

  private:
    hyperim_graph* g_;
    std::vector<std::pair<void*, size_t>> bufs_;
};
hyperim_status check_device_status(hyperim_graph* g, const char* where);

// load.cu
hyperim_status build_graph(hyperim_graph* g, const int32_t* he_off, const int32_t* he_mem,
                           int32_t nnz_in, bool on_device);

// load.cu: the listed vertices by descending neighbourhood size (quarter-octave buckets of tsum):
// out[j] = list[i] (or i, emit_index) for the j-th largest; order within a bucket unspecified
hyperim_status size_order(hyperim_graph* g, const int32_t* list, int64_t count, bool emit_index, int32_t* out);

// index.cu: chunk index of the vertices with large neighbourhoods (after the layer profile)
hyperim_status build_chunk_index(hyperim_graph* g);

// scan.cu: exclusive scan of n uint32/int32 counts into int64 (out has n + 1 entries)
hyperim_status exclusive_scan_u32_to_i64(hyperim_graph* g, const uint32_t* in, int64_t* out,
                                         int64_t n);
hyperim_status exclusive_scan_i64(hyperim_graph* g, const int64_t* in, int64_t* out, int64_t n);

// rr.cu: grow one pool, or several pools of the same root mode and strategy in one launch
hyperim_status sample_rr(hyperim_graph* g, hyperim_pool* p, const uint64_t new_ns[HYPERIM_NSTRATA]);
hyperim_status sample_rr_multi(hyperim_graph* g, hyperim_pool* const* pools, int npools,
                               const uint64_t (*new_ns)[HYPERIM_NSTRATA]);

// rr.cu: one launch over the pools of several graphs (the batched form of HyperIM_BRR). Group
// q grows up to two pools of graph g (same root mode and strategy) to new_ns; every group's
// sets are built by one persistent launch on g0's stream (which first waits for the work queued
// on the groups' streams), and one compaction kernel there appends them to their pools (each
// pool's arrays grown beforehand on its graph's stream). seconds: the launch's CUDA-event time.
struct RRGroup {
    hyperim_graph* g;
    hyperim_pool* pools[2];
    int npools;
    uint64_t new_ns[2][HYPERIM_NSTRATA];
};
hyperim_status sample_rr_batch(hyperim_graph* g0, const RRGroup* groups, int ngroups, double* seconds);

// rr.cu: forward Monte-Carlo influence of a seed set (counts_host: nsims entries)
hyperim_status forward_spread(hyperim_graph* g, const int32_t* seeds_host, int32_t k, uint64_t nsims,
                              uint64_t seed, uint32_t* counts_host);

// greedy.cu
// lim (optional): a prefix view, only the RR sets (s, j) with j < lim[s] take part
hyperim_status greedy(hyperim_graph* g, hyperim_pool* p, int32_t k, int32_t* seeds_host,
                      uint64_t lambda_s[HYPERIM_NSTRATA], uint64_t* prefix_upper = nullptr,
                      const uint64_t* lim = nullptr);
hyperim_status coverage(hyperim_graph* g, hyperim_pool* p, const int32_t* seeds_host, int32_t k,
                        uint64_t lambda_s[HYPERIM_NSTRATA], const uint64_t* lim = nullptr);

// greedy.cu: greedy max coverage one round at a time, with the argmax taken over a score vector
// the caller supplies (the sum of every shard's scores); see hyperim_greedy_begin
struct GreedyState;
hyperim_status greedy_begin(hyperim_graph* g, hyperim_pool* p, const uint64_t* lim, GreedyState** out);
hyperim_status greedy_scores(GreedyState* st, unsigned long long* dev_out);
hyperim_status greedy_pick(GreedyState* st, const unsigned long long* dev_total, int32_t* picked);
hyperim_status greedy_end(GreedyState* st, uint64_t lambda_s[HYPERIM_NSTRATA]);

// greedy.cu: the batched form -- greedy max coverage on the R1 view and the coverage of its seeds
// on the R2 view for many queries in one launch (one block per query). lim1 / lim2: prefix views
// (nullptr: the whole pool). Runs on g0's stream; the pools' arrays must be ready there.
struct GreedyBatchItem {
    hyperim_graph* g;
    hyperim_pool* r1;
    hyperim_pool* r2;
    const uint64_t* lim1;
    const uint64_t* lim2;
    int32_t k;
    int32_t* seeds_host;         // k entries
    uint64_t* lambda_r1;         // HYPERIM_NSTRATA entries
    uint64_t* lambda_r2;
};
hyperim_status greedy_batch(hyperim_graph* g0, const GreedyBatchItem* items, int nitems);

// host arithmetic (plan.cpp)
void allocate_strata(const hyperim_graph* g, int32_t root_mode, uint64_t theta,
                     uint64_t n_s[HYPERIM_NSTRATA]);
// Eq. upper_2 bound {lo, hi} (greedy weights) in sigma units
double prefix_upper_sigma(const uint64_t u[2], int32_t root_mode, int64_t n, uint64_t N);
double estimate(const hyperim_graph* g, int32_t root_mode, const uint64_t n_s[HYPERIM_NSTRATA],
                const uint64_t lambda_s[HYPERIM_NSTRATA]);
uint64_t stratum_weight(const hyperim_graph* g, int32_t root_mode, uint64_t n_s, int s);

}  // namespace hyperim
