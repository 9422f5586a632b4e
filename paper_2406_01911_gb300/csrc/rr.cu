// Stratified random RR sets on a hypergraph (Algorithm 3) and their compaction to CSR.
//
// One block builds one RR set at a time (persistent grid over the batch). The reverse BFS runs
// level by level: the warps of the block pop the vertices of the current level in parallel.
// For a popped mu each lane draws h_i for one layer of A(mu) (Binomial if n(L_i) <= 20, else
// Poisson; Sec. 3.1.3) from the keyed Philox stream (RR, mu, layer); if some h_i > 0, the layer
// members at the picked positions are found by materialising A(mu) on chip:
//   - d_H(mu) = 1: A(mu) is the one hyperedge minus mu, already sorted -> direct indexing;
//   - small neighbourhoods: the warp sorts the members of mu's hyperedges in shared memory;
//   - large ones are deferred to the end of the level and processed by the whole block, on chip
//     or, past the on-chip buffer, bucketed by id through a global scratch area.
// Draws are keyed by (RR, vertex, layer), so the set does not depend on the pop order and the
// parallel pops are deterministic. Picks already in R are skipped (visited bitmap).
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <vector>

#include "device_math.cuh"
#include "internal.h"
#include "mat.cuh"

namespace hyperim {
namespace {

constexpr int kThreads = 512;    // a block of the block-per-set kernels: one per SM
constexpr int kWarps = kThreads / 32;
constexpr int kPThreads = 256;   // a block of the warp phase (a set per warp): two per SM
constexpr int kPWarps = kPThreads / 32;
constexpr int kWCap = 2048;      // per-warp on-chip neighbourhood keys (power of two)
constexpr int kWHalf = kWCap / 2;  // raw copy + sorted copy of neighbourhoods up to this size
constexpr int kPCap = 256;       // per-warp picks
constexpr int kLQ = 32;          // per-warp layers with h > 0 handled on the warp path
constexpr int kCG = 64;          // hyperedges per group of the chunk path (two per lane)
constexpr int kBCap = 8192;      // block on-chip keys (power of two)
constexpr int kBLQ = 64;         // layers with h > 0 per block round
constexpr int kDCap = 256;       // deferred pops per level round
constexpr int kBucketBits = 12;
constexpr int kBuckets = 1 << kBucketBits;    // block-path buckets
constexpr int kWBucketBits = 8;
constexpr int kWBuckets = 1 << kWBucketBits;  // warp-path buckets
constexpr int kChunks = 1024;        // first-level id chunks of the largest neighbourhoods
constexpr int kVisSmemBits = 1 << 19;  // visited bitmap on chip when n <= this
constexpr int kMaxPools = 2;           // pools grown by one launch (R1 and R2 of a BRR round)
constexpr int kNStat = 10;             // work counters (stat slots below)
// warp phase: a warp builds a whole RR set alone while it stays within kWQ members
constexpr int kWQ = 128;               // per-warp queue (members of the warp's set)
constexpr int kWHashBits = 8;
constexpr int kWHash = 1 << kWHashBits;  // per-warp open-addressing member set

struct RRJobMap {
    int64_t job_base[HYPERIM_NSTRATA + 1];
    uint32_t j_base[HYPERIM_NSTRATA];
    uint32_t j_step;   // the pool's shard stride: job x of stratum s is j = j_base[s] + x j_step
};

struct RRParams {
    const int4* vinfo;        // per vertex: {profile begin, l, incidence begin, d_H}
    const int2* v_span;       // per incidence: {member begin, |he|}
    const int32_t* he_mem;
    const int32_t* prof_off;
    const uint4* prof;
    const uint32_t* tab;      // CDF threshold tables
    const int32_t* tsum;
    const int32_t* vs_off;
    const int32_t* vs_list;
    const uint64_t* idx;      // per vertex: 0 or (chunk bits << 56) | offset into idx_tab
    const uint32_t* idx_tab;
    const uint32_t* mat_sect; // per vertex: sectors of v_he(v) and of mem(he) for he in v
    const uint16_t* he_dir;   // id directories of the larger hyperedges
    const uint2* v_dir;       // per incidence: {directory offset, bits} (bits 0: none)
    int32_t n;
    int id_bits;
    uint64_t seed;
    int root_mode;
    int strategy;
    int npools;                              // pools grown by this launch (same root mode/strategy)
    int64_t pool_start[kMaxPools + 1];       // jobs of pool q: [pool_start[q], pool_start[q + 1])
    uint32_t tags[kMaxPools];
    RRJobMap jm[kMaxPools];
    int32_t* list;            // per block: list_cap entries
    int64_t list_cap;
    uint32_t* gvis;           // per block: vis_words (when not on chip)
    int vis_smem;             // 1 if the visited bitmap lives in shared memory
    int64_t vis_words;
    uint32_t* picks;          // per block: pick_cap entries
    int64_t pick_cap;
    uint32_t* big;            // per block: big_cap entries
    int64_t big_cap;
    int32_t* arena;
    uint64_t arena_cap;
    unsigned long long* arena_used;
    int64_t* out_pos;
    int32_t* out_size;
    int* next_job;
    int* esc_count;           // jobs the warp phase handed to the block phase
    int32_t* esc_list;        // those jobs
    int block_phase;          // 1: this launch runs the jobs of esc_list (else all jobs)
    int warp_limit;           // warp phase: the largest RR set a warp builds alone (1..kWQ)
    int plain;                // 1: this launch runs jobs [plain_base, plain_base + gridDim.x), one per block
    int64_t plain_base;
    int rewrite;              // 1: a repair launch -- sets go to the arena slots recorded by the first
                              // launch (out_pos), whose arena was too small; no counters are added
    DevStatus* st;
    RRCounters* counters;                    // kMaxPools entries
    int spin_limit;                          // rounds of a bounded wait before it gives up
    unsigned long long* set_cycles;          // optional {sum, max, count} of per-set SM cycles
};

struct Need {                    // a layer with h > 0 at the current pop
    uint32_t w, n, h, ksel, layer;
};

// Buffers of phase 1 (warps pop independently) and of phase 2 / output (the whole block works on
// one deferred pop, or on the finished set) never live at the same time: they share storage.
template <int W>
struct WarpAreaT {
    uint32_t wbuf[W][kWCap];
    int wbkt[W][kWBuckets];
    uint32_t wpick[W][kPCap];
};
using WarpArea = WarpAreaT<kWarps>;
struct BlockArea {
    uint32_t bbuf[kBCap];
    int bucket[kBuckets];
    int chunk_end[kChunks];
    int bpre[2 * kThreads + 1];
};

struct Shared {
    int ctrl[16];
    int tmp[kWarps + 2];
    unsigned long long stat[kMaxPools][kNStat];  // per pool work counters of this block
    unsigned long long wstat[kWarps][kNStat];    // per-warp counters of the current RR set (lane 0)
    unsigned long long out_pos;
    unsigned long long cyc_sum, cyc_max, cyc_count;  // per-set SM cycles of this block's sets
    long long cyc_start;                              // clock of the current set's start
    int32_t deferred[kDCap];
    Need wneed[kWarps][kLQ];
    int wcursor[kWarps];
    int wpre[kWarps][3 * kCG + 1];  // span prefix, starts, holes of a group of hyperedges (chunk path)
    uint32_t wpoff[kWarps][kLQ + 1];
    int wcnt[kWarps][kBLQ];     // per-warp per-layer counts (ranks)
    int lcnt[kBLQ];             // running rank per needed layer (block path)
    Need bneed[kBLQ];
    uint32_t bpick_off[kBLQ + 1];
    union {
        WarpArea w;
        BlockArea b;
    } u;
};
// ctrl slots
enum { C_JOB = 0, C_HEAD, C_TAIL, C_DONE, C_NDEF, C_ROOT, C_NNEED, C_CURSOR, C_STOP, C_BITS, C_OK,
       C_FAIL };
// stat slots
enum { S_POPS = 0, S_LAYERS, S_DRAWS, S_MATS, S_MAT_HE, S_MAT_MEM, S_SEL, S_GATH, S_SRCH, S_SECT };
// the stat slots are the fields of RRCounters, in order
static_assert(sizeof(RRCounters) == kNStat * sizeof(unsigned long long) &&
                  offsetof(RRCounters, sectors) == S_SECT * sizeof(unsigned long long) &&
                  offsetof(RRCounters, gathered) == S_GATH * sizeof(unsigned long long),
              "RRCounters must list the stat slots in order");

// 32-byte sectors spanned by the byte range [a, a + len) (0 when empty)
__device__ __forceinline__ unsigned long long sectors_of(uint64_t a, uint64_t len) {
    return len == 0 ? 0ull : (unsigned long long)(((a + len - 1) >> 5) - (a >> 5) + 1);
}

__device__ __forceinline__ void dev_fail(DevStatus* st, int32_t code, int32_t detail) {
    if (atomicCAS(&st->code, 0, code) == 0) st->detail = detail;
}

// h for one layer (lane-level) from its two profile words and its CDF table. Returns whether a
// draw was made (0 < p < 1). The draw is decided by integer compares against the layer's table
// (T_0 first, which sits in the entry); only words beyond the table's last threshold run the
// double-precision inversion.
__device__ __forceinline__ bool layer_draw(const uint4 e, const uint4 f, const uint32_t* __restrict__ tab,
                                          int strategy, WordStream& ws, uint32_t& h, uint32_t& ksel) {
    const uint32_t n_i = e.y, thr = e.z;
    ksel = 0;
    if (e.x & kPOneFlag) { h = n_i; return false; }
    if (thr == 0) { h = 0; return false; }
    const uint32_t w0 = ws.word(0);
    const uint32_t kind = f.w, L = f.y, c = f.z;
    if (kind == 1) {  // Binomial table: the same draw under both strategies (n_i <= 20)
        ksel = 1;
        if (w0 < e.w) { h = 0; return true; }
        const uint32_t k = table_find(tab + f.x, L, w0);
        h = k < L ? k : (L == n_i ? n_i : binomial_h(n_i, thr, w0));
        return true;
    }
    if (strategy == HYPERIM_STRAT_PAPER) {  // Poisson, c parts (kind 2)
        ksel = c;
        if (c == 1 && w0 < e.w) { h = 0; return true; }
        uint64_t sum = 0;
        for (uint32_t t = 0; t < c; ++t) {
            const uint32_t w = t == 0 ? w0 : ws.word(t);
            const uint32_t k = table_find(tab + f.x, L, w);
            sum += k < L ? k
                 : (L == n_i ? n_i : poisson_part(poisson_part_lambda(poisson_lambda(n_i, thr), c), n_i, w));
        }
        h = sum > n_i ? n_i : (uint32_t)sum;
        return true;
    }
    h = binomial_h(n_i, thr, w0);  // Binomial strategy on a layer the paper draws by Poisson
    ksel = 1;
    return true;
}

// Picks of one layer (warp-cooperative, all lanes pass identical arguments): for r = 0..h-1,
// a = floor(x_r (n - r) / 2^32) from word ksel + r, and the pick is the a-th (0-based) position
// of [0, n) not picked yet (Sec. 3.1.3: one uniform choice from the remainder per step).
// sel[0, h) receives the picked positions in ascending order.
__device__ void gen_picks(WordStream& ws, uint32_t n, uint32_t h, uint32_t ksel, uint32_t* sel) {
    const int lane = threadIdx.x & 31;
    if (h <= 32) {
        // lane r draws a_r from its own word; the picks so far stay sorted across the lanes
        // (lane i holds the i-th smallest), so each step is a few ballots
        uint32_t a = 0, mine = 0xFFFFFFFFu;
        if ((uint32_t)lane < h) {
            const uint32_t x = ws.word(ksel + (uint32_t)lane);
            a = (uint32_t)(((uint64_t)x * (uint64_t)(n - (uint32_t)lane)) >> 32);
        }
        for (uint32_t r = 0; r < h; ++r) {
            const uint32_t ar = __shfl_sync(0xFFFFFFFFu, a, (int)r);
            uint32_t idx = ar;
            for (;;) {  // idx = a_r + #{picks <= idx}
                const uint32_t c = __popc(__ballot_sync(0xFFFFFFFFu, (uint32_t)lane < r && mine <= idx));
                if (ar + c == idx) break;
                idx = ar + c;
            }
            const uint32_t at = __popc(__ballot_sync(0xFFFFFFFFu, (uint32_t)lane < r && mine < idx));
            const uint32_t up = __shfl_up_sync(0xFFFFFFFFu, mine, 1);
            if ((uint32_t)lane > at && (uint32_t)lane <= r) mine = up;
            if ((uint32_t)lane == at) mine = idx;
        }
        if ((uint32_t)lane < h) sel[lane] = mine;
        __syncwarp();
        return;
    }
    for (uint32_t r = 0; r < h; ++r) {
        const uint32_t x = ws.word(ksel + r);
        const uint32_t a = (uint32_t)(((uint64_t)x * (uint64_t)(n - r)) >> 32);
        uint32_t idx = a, c = 0;
        for (;;) {
            uint32_t cnt = 0;
            for (uint32_t t = lane; t < r; t += 32) cnt += sel[t] <= idx ? 1u : 0u;
            cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
            const uint32_t nid = a + cnt;
            c = cnt;
            if (nid == idx) break;
            idx = nid;
        }
        // insert idx at position c (shift sel[c, r) up by one, top chunk first)
        if (r > c) {
            for (int64_t top = (int64_t)r - 1; top >= (int64_t)c; top -= 32) {
                const int64_t t = top - lane;
                uint32_t v = 0;
                const bool act = t >= (int64_t)c;
                if (act) v = sel[t];
                __syncwarp();
                if (act) sel[t + 1] = v;
                __syncwarp();
            }
        }
        if (lane == 0) sel[c] = idx;
        __syncwarp();
    }
}

// LT cascade (Sec. 2.2, LT model) in its live-edge form: the popped mu keeps at most one
// in-neighbour. One thread. With t_i = floor(p_i 2^32) (2^32 for p = 1), masses m_i = n_i t_i
// cumulated as C_i and M = C_l (exact 128-bit integers), one word x of the (RR, mu, layer 0)
// stream gives y = x if M <= 2^32 (no vertex kept when y >= M), else y = floor(x M / 2^32); the
// kept vertex is position floor((y - C_{i-1}) / t_i) of the layer with C_{i-1} <= y < C_i. Returns
// whether a vertex is kept and, through nd, {w_i, n_i, h = 1, kept position, layer i}; *drew
// tells whether a word was used (M > 0).
__device__ bool lt_keep(const RRParams& P, int32_t pb, int32_t l, uint32_t j, uint32_t ybase, int32_t mu,
                        Need& nd, bool* drew) {
    unsigned __int128 M = 0;
    for (int i = 0; i < l; ++i) {
        const uint4 e = P.prof[2 * ((int64_t)pb + i)];
        const uint64_t t = (e.x & kPOneFlag) ? (1ull << 32) : (uint64_t)e.z;
        M += (unsigned __int128)e.y * t;
    }
    *drew = M > 0;
    if (M == 0) return false;
    WordStream ws;
    ws.init(P.seed, j, ybase, (uint32_t)mu, 0u);
    const uint32_t x = ws.word(0);
    unsigned __int128 y = x;
    if (M > ((unsigned __int128)1 << 32)) y = ((unsigned __int128)x * M) >> 32;
    else if (y >= M) return false;
    unsigned __int128 C = 0;
    for (int i = 0; i < l; ++i) {
        const uint4 e = P.prof[2 * ((int64_t)pb + i)];
        const uint64_t t = (e.x & kPOneFlag) ? (1ull << 32) : (uint64_t)e.z;
        const unsigned __int128 m = (unsigned __int128)e.y * t;
        if (y < C + m) {
            nd = Need{e.x & ~kPOneFlag, e.y, 1u, (uint32_t)((uint64_t)(y - C) / t), (uint32_t)(i + 1)};
            return true;
        }
        C += m;
    }
    return false;  // unreachable: y < M
}

__device__ __forceinline__ bool in_sorted(const uint32_t* a, uint32_t len, uint32_t x) {
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint32_t v = a[mid];
        if (v == x) return true;
        if (v < x) lo = mid + 1; else hi = mid;
    }
    return false;
}

// Add nu to R if it is not there yet: reserve a queue slot, then store the id there (a reader
// that claimed the slot waits until the id replaces the empty mark -1).
__device__ __forceinline__ void push(const RRParams& P, Shared& S, uint32_t* vis, int32_t* list,
                                     uint32_t nu) {
    const uint32_t bit = 1u << (nu & 31);
    const uint32_t old = atomicOr(&vis[nu >> 5], bit);
    if (!(old & bit)) {
        const int pos = atomicAdd(&S.ctrl[C_TAIL], 1);
        *(volatile int32_t*)&list[pos] = (int32_t)nu;
    }
}

// Where a pop's activations go: the RR set of a block (its visited bitmap and work queue, the
// queue's tail counter in shared memory), or the RR set a warp builds alone (an open-addressing
// member set and a queue in shared memory).
struct QueueSink {
    uint32_t* vis;
    int32_t* list;
    int* tail;
    __device__ __forceinline__ void push(uint32_t nu) const {
        const uint32_t bit = 1u << (nu & 31);
        const uint32_t old = atomicOr(&vis[nu >> 5], bit);
        if (!(old & bit)) {
            const int pos = atomicAdd(tail, 1);
            *(volatile int32_t*)&list[pos] = (int32_t)nu;
        }
    }
};

struct WarpSink {
    int32_t* hash;   // kWHash slots, -1 empty
    int32_t* queue;  // kWQ slots
    int* tail;       // members so far (may pass limit: the set then leaves the warp phase)
    int limit;       // the largest set a warp builds alone (<= kWQ)
    __device__ __forceinline__ void push(uint32_t nu) const {
        if (*(volatile int*)tail > limit) return;  // already too large: the set is redone by a block
        uint32_t h = (nu * 0x9E3779B1u) >> (32 - kWHashBits);
        for (int probe = 0; probe < kWHash; ++probe) {
            const int32_t old = atomicCAS(&hash[h], -1, (int32_t)nu);
            if (old == -1) {
                const int pos = atomicAdd(tail, 1);
                if (pos < limit) queue[pos] = (int32_t)nu;
                return;
            }
            if (old == (int32_t)nu) return;
            h = (h + 1) & (kWHash - 1);
        }
        atomicMax(tail, limit + 1);  // no free slot (cannot happen below kWQ + 32 members)
    }
};

// Work queue of one RR set (lane 0 of a warp). Slots [0, tail) are reserved, [0, head) claimed,
// done pops are finished (their pushes are in), ndef claimed pops wait for the block path.
// Returns a claimed slot, or -1 when this warp should go to the block barrier: no pop is in
// flight (head - ndef == done) and either the queue is empty or the deferred list is nearly
// full. done is read first and fenced: a pop publishes its pushes (tail, slots) before it counts
// itself done, so the head and tail read afterwards include them, and a warp leaves only when
// the queue is quiescent (a warp that left early would idle at the barrier for the rest of the
// set). The wait is bounded (kErrSpin).
__device__ int claim_slot(const RRParams& P, Shared& S, int64_t job) {
    volatile int* ctrl = S.ctrl;
    for (int it = 0; it < P.spin_limit; ++it) {
        const int d = ctrl[C_DONE];
        __threadfence_block();
        const int h = ctrl[C_HEAD], t = ctrl[C_TAIL], nd = ctrl[C_NDEF];
        if (h < t && nd <= kDCap - kWarps) {
            if (atomicCAS(&S.ctrl[C_HEAD], h, h + 1) == h) return h;
            continue;
        }
        if (h - nd == d) return -1;
        __nanosleep(64);
    }
    dev_fail(P.st, kErrSpin, (int32_t)job);
    return -1;
}

// The id in a claimed slot (its pusher may still be storing it); -1 if the bounded wait ran out.
__device__ int32_t slot_value(const RRParams& P, const int32_t* list, int idx, int64_t job) {
    const volatile int32_t* v = list + idx;
    for (int it = 0; it < P.spin_limit; ++it) {
        const int32_t x = *v;
        if (x >= 0) return x;
        __nanosleep(32);
    }
    dev_fail(P.st, kErrSpin, (int32_t)job);
    return -1;
}

// ------------------------------------------------------------------------------------------
// warp path
// ------------------------------------------------------------------------------------------
// A(mu) with at most kWHalf incidence positions (tsum, mu's own included), by one pass over the
// members: a raw copy goes to buf[kWHalf, kWHalf + tsum) and the members are counted into
// buckets of their top id bits; the raw copy is then scattered into buf[0, T) in bucket order and
// each bucket is sorted (members sorted by id).
template <class SM>
__device__ void small_nbhd(const RRParams& P, SM& S, int32_t mu, int32_t v_begin, int32_t dh, int tsum,
                           int T, uint32_t* buf) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int* bkt = S.u.w.wbkt[wid];
    uint32_t* raw = buf + kWHalf;
    const int nbits = bucket_bits(T, kWBucketBits);
    const int nb = 1 << nbits;
    const int shift = P.id_bits > nbits ? P.id_bits - nbits : 0;
    const uint32_t key_mask = (uint32_t)nb - 1;
    for (int b = lane; b < nb; b += 32) bkt[b] = 0;
    __syncwarp();
    for_each_position<32>(P.v_span, P.he_mem, v_begin, dh, S.wpre[wid], [&](int pos, uint32_t x) {
        raw[pos] = x;
        if (x != (uint32_t)mu) atomicAdd(&bkt[(x >> shift) & key_mask], 1);
    });
    const int maxb = warp_bucket_scan(bkt, nb);  // bucket starts
    warp_scatter_sort(raw, tsum, (uint32_t)mu, buf, T, bkt, nb, 0u, shift, key_mask, maxb);
}

// For every needed layer q < nq (lane q passes its row, k0, pos and whether it searches): the
// last chunk k in [k0, C) whose prefix row[k] is <= pos (row[k0] <= pos is given). The warp
// splits into groups of G = 32 / Q lanes (Q = the power of two >= nq), group q searching for layer
// q G-ary: each round probes G evenly spaced entries of the range at once, so C = 4096 chunks take
// 3 rounds with one or two needed layers instead of 12 dependent probes. Lane q gets its layer's
// answer (-1 for a layer that does not search). With more than 16 needed layers every lane
// searches alone (binary search).
__device__ __forceinline__ int chunk_of(const uint32_t* __restrict__ row, int k0, int C, uint32_t pos,
                                        uint32_t& probes);

__device__ __forceinline__ int warp_chunk_search(const uint32_t* row, int k0, int C, uint32_t pos, bool want,
                                                 uint32_t nq, uint32_t& probes) {
    const int lane = threadIdx.x & 31;
    int Q = 1;
    while (Q < (int)nq) Q <<= 1;
    if (Q > 16) return want ? chunk_of(row, k0, C, pos, probes) : -1;
    const int G = 32 / Q, q = lane / G, gl = lane - q * G;
    const uint32_t* r = reinterpret_cast<const uint32_t*>(
        __shfl_sync(0xFFFFFFFFu, reinterpret_cast<unsigned long long>(row), q));
    int lo = __shfl_sync(0xFFFFFFFFu, k0, q);
    const uint32_t ps = __shfl_sync(0xFFFFFFFFu, pos, q);
    const bool act = __shfl_sync(0xFFFFFFFFu, want ? 1 : 0, q) != 0 && q < (int)nq;
    int hi = act ? C : lo + 1;
    const uint32_t gmask = G == 32 ? 0xFFFFFFFFu : ((1u << G) - 1u);
    while (__any_sync(0xFFFFFFFFu, hi - lo > 1)) {
        const int span = hi - lo;
        const int step = (span + G - 1) / G;
        const int x = lo + gl * step;
        bool pred = gl == 0;  // row[lo] <= pos holds
        if (span > 1 && gl > 0 && x < hi) {
            ++probes;
            pred = r[x] <= ps;
        }
        const uint32_t gb = (__ballot_sync(0xFFFFFFFFu, pred) >> (q * G)) & gmask;
        if (span > 1) {
            const int g = 31 - __clz(gb);
            const int nlo = lo + g * step;
            hi = min(nlo + step, hi);
            lo = nlo;
        }
    }
    const int res = __shfl_sync(0xFFFFFFFFu, lo, lane < Q ? lane * G : 0);
    return want ? res : -1;
}

// Last chunk k in [k0, C) whose prefix row[k] is <= pos (row[k0] <= pos is given).
__device__ __forceinline__ int chunk_of(const uint32_t* __restrict__ row, int k0, int C, uint32_t pos,
                                        uint32_t& probes) {
    int lo = k0, hi = C;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        ++probes;
        if (row[mid] <= pos) lo = mid; else hi = mid;
    }
    return lo;
}

// The slice of one sorted hyperedge (members e[0, len)) whose ids lie in chunk k = lo >> sh of
// the ids' top c = id_bits - sh bits: offsets [l1, l2) and, when mu lies in the range, mu's offset
// l3. Read off the hyperedge's id directory when it has one (two entries when c <= b, else one
// directory range of about one member, scanned), else found by interleaved binary searches.
struct Slice {
    int l1, l2, l3;
};

__device__ __forceinline__ Slice hyperedge_slice(const RRParams& P, int2 sp, uint2 dd, uint32_t lo, uint32_t hi,
                                                 int c, uint32_t k, int32_t mu, bool mu_in, uint32_t& probes) {
    const int32_t* e = P.he_mem + sp.x;
    Slice r{0, 0, 0};
    if (dd.y != 0) {
        const uint16_t* D = P.he_dir + dd.x;
        const int b = (int)dd.y;
        const uint32_t rm = (uint32_t)mu >> (P.id_bits - b);
        int m0 = 0, m1 = 0;
        if (mu_in) {  // mu's directory range (issued with the slice's entries)
            m0 = D[rm];
            m1 = D[rm + 1];
            probes += 2;
        }
        if (c <= b) {
            r.l1 = D[k << (b - c)];
            r.l2 = D[(k + 1) << (b - c)];
            probes += 2;
        } else {
            const uint32_t rr = k >> (c - b);
            const int a0 = D[rr], a1 = D[rr + 1];
            probes += 2;
            r.l1 = a0;
            r.l2 = a0;
            for (int x = a0; x < a1; ++x) {
                const uint32_t v = (uint32_t)e[x];
                ++probes;
                r.l1 += v < lo ? 1 : 0;
                r.l2 += v < hi ? 1 : 0;
            }
        }
        if (mu_in) {
            r.l3 = m0;
            while (r.l3 < m1 && (uint32_t)e[r.l3] < (uint32_t)mu) {
                ++r.l3;
                ++probes;
            }
        }
        return r;
    }
    // three lower bounds (lo, hi, mu) advanced together: their loads overlap
    int l1 = 0, h1 = sp.y, l2 = 0, h2 = sp.y, l3 = 0, h3 = mu_in ? sp.y : 0;
    while (l1 < h1 || l2 < h2 || l3 < h3) {
        const int m1 = (l1 + h1) >> 1, m2 = (l2 + h2) >> 1, m3 = (l3 + h3) >> 1;
        const uint32_t v1 = l1 < h1 ? (uint32_t)e[m1] : 0u;
        const uint32_t v2 = l2 < h2 ? (uint32_t)e[m2] : 0u;
        const uint32_t v3 = l3 < h3 ? (uint32_t)e[m3] : 0u;
        if (l1 < h1) { ++probes; if (v1 < lo) l1 = m1 + 1; else h1 = m1; }
        if (l2 < h2) { ++probes; if (v2 < hi) l2 = m2 + 1; else h2 = m2; }
        if (l3 < h3) { ++probes; if (v3 < (uint32_t)mu) l3 = m3 + 1; else h3 = m3; }
    }
    r.l1 = l1;
    r.l2 = l2;
    r.l3 = l3;
    return r;
}

// The members != mu of mu's hyperedges whose ids lie in [lo, hi), sorted, in buf[0, count);
// returns count, or -1 if they exceed kWHalf. lo is a multiple of 2^sh (the range is chunk
// k = lo >> sh of the ids' top c = id_bits - sh bits). Members of a hyperedge are sorted, so the
// range is one slice of each (hyperedge_slice); when mu lies in the range its own slot in every
// slice is skipped (a hole at mu's offset). The hyperedges are taken kCG at a time, two per lane,
// so that the lookups of both overlap; the slices are gathered with independent loads into the
// raw half of buf and counted into buckets of the id offset within the range, then scattered and
// sorted as in small_nbhd. probes counts the words read to locate the slices.
template <class SM>
__device__ int chunk_nbhd(const RRParams& P, SM& S, int32_t mu, int32_t v_begin, int32_t dh,
                          uint32_t lo, int sh, uint32_t* buf, uint32_t& probes) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int* pre = S.wpre[wid];
    int* start = pre + kCG + 1;
    int* hole = start + kCG;
    uint32_t* raw = buf + kWHalf;
    int* bkt = S.u.w.wbkt[wid];
    constexpr int nb = kWBuckets;
    const int shift = sh > kWBucketBits ? sh - kWBucketBits : 0;
    const uint32_t key_mask = (uint32_t)nb - 1;
    const uint32_t hi = lo + (1u << sh);
    const bool mu_in = (uint32_t)mu >= lo && (uint32_t)mu < hi;
    const int c = P.id_bits - sh;
    const uint32_t k = lo >> sh;
    for (int b = lane; b < nb; b += 32) bkt[b] = 0;
    int base = 0;
    for (int c0 = 0; c0 < dh; c0 += kCG) {
        const int cnt = min(kCG, dh - c0);
        // lane takes hyperedges c0 + lane and c0 + 32 + lane
        int st[2] = {0, 0}, len[2] = {0, 0}, hl[2] = {0x7FFFFFFF, 0x7FFFFFFF};
        int2 sp[2];
        uint2 dd[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int x = u * 32 + lane;
            sp[u] = x < cnt ? P.v_span[v_begin + c0 + x] : make_int2(0, 0);
            dd[u] = x < cnt ? P.v_dir[v_begin + c0 + x] : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int x = u * 32 + lane;
            if (x < cnt) {
                const Slice r = hyperedge_slice(P, sp[u], dd[u], lo, hi, c, k, mu, mu_in, probes);
                st[u] = sp[u].x + r.l1;
                len[u] = r.l2 - r.l1;
                if (mu_in) {
                    hl[u] = r.l3 - r.l1;
                    len[u] -= 1;
                }
            }
        }
        // inclusive prefix of the lengths over the group (first the lanes' first hyperedges)
        int inc0 = len[0], inc1 = len[1];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t0 = __shfl_up_sync(0xFFFFFFFFu, inc0, o);
            const int t1 = __shfl_up_sync(0xFFFFFFFFu, inc1, o);
            if (lane >= o) {
                inc0 += t0;
                inc1 += t1;
            }
        }
        const int tot0 = __shfl_sync(0xFFFFFFFFu, inc0, 31);
        inc1 += tot0;
        __syncwarp();  // the previous group's readers of pre / start / hole are done
        if (lane == 0) pre[0] = 0;
        if (lane < cnt) {
            pre[lane + 1] = inc0;
            start[lane] = st[0];
            hole[lane] = hl[0];
        }
        if (32 + lane < cnt) {
            pre[33 + lane] = inc1;
            start[32 + lane] = st[1];
            hole[32 + lane] = hl[1];
        }
        __syncwarp();
        const int total = pre[cnt];
        if (base + total > kWHalf) return -1;  // uniform
        const bool stepwise = total >= cnt * 8;
        int j = 0;
        constexpr int U = 2;
        for (int p0 = lane; p0 < total; p0 += U * 32) {
            uint32_t xs[U] = {};
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int p = p0 + u * 32;
                if (p < total) {
                    if (stepwise && p != lane) {
                        while (pre[j + 1] <= p) ++j;
                    } else {
                        int l2 = 0, h2 = cnt;
                        while (h2 - l2 > 1) {
                            const int mid = (l2 + h2) >> 1;
                            if (pre[mid] <= p) l2 = mid; else h2 = mid;
                        }
                        j = l2;
                    }
                    int o = p - pre[j];
                    o += o >= hole[j] ? 1 : 0;
                    xs[u] = (uint32_t)P.he_mem[start[j] + o];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int p = p0 + u * 32;
                if (p < total) {
                    raw[base + p] = xs[u];
                    atomicAdd(&bkt[((xs[u] - lo) >> shift) & key_mask], 1);
                }
            }
        }
        base += total;
    }
    __syncwarp();
    const int maxb = warp_bucket_scan(bkt, nb);
    warp_scatter_sort(raw, base, kSentinel, buf, base, bkt, nb, lo, shift, key_mask, maxb);
    return base;
}

// Ranked walk of a sorted warp buffer buf[0, got): a run of multiplicity need[q].w is a member
// of needed layer q, its rank in L_q is cnt[q] (the layer's members before the buffer) plus the
// runs of that layer before it; members whose rank is a pick, or all of them when h = n, enter R.
// The running rank of layer q lives in lane q's register; each 32 positions take one ballot per
// needed layer. Stops once every layer with picks has ranked past its last pick.
template <class SM, class Sink>
__device__ void warp_walk(const RRParams& P, SM& S, const Sink& sink, const uint32_t* buf, int got,
                          uint32_t nneed) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const Need* need = S.wneed[wid];
    const uint32_t* picks = S.u.w.wpick[wid];
    const uint32_t* poff = S.wpoff[wid];
    uint32_t mycnt = (uint32_t)lane < nneed ? (uint32_t)S.wcnt[wid][lane] : 0u;
    // lane q's layer: its last pick (or none when the layer is taken whole)
    uint32_t mylast = 0xFFFFFFFFu;
    bool mypicks = false;
    if ((uint32_t)lane < nneed) {
        const Need nd = need[lane];
        mypicks = nd.h < nd.n;
        if (mypicks) mylast = picks[poff[lane] + nd.h - 1];
    }
    const uint32_t want_mask = nneed >= 32 ? 0xFFFFFFFFu : ((1u << nneed) - 1);
    for (int base = 0; base < got; base += 32) {
        const int p = base + lane;
        bool start = false;
        uint32_t x = kSentinel;
        int mult = 0;
        if (p < got) {
            x = buf[p];
            start = (p == 0) || (buf[p - 1] != x);
            if (start) {
                mult = 1;
                while (p + mult < got && buf[p + mult] == x) ++mult;
            }
        }
        for (uint32_t q = 0; q < nneed; ++q) {
            const bool f = start && (uint32_t)mult == need[q].w;
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, f);
            if (bal == 0) continue;
            const uint32_t before = __shfl_sync(0xFFFFFFFFu, mycnt, (int)q);
            if (f) {
                const Need nd = need[q];
                const uint32_t rank = before + __popc(bal & lanemask_lt());
                if (nd.h >= nd.n || in_sorted(picks + poff[q], nd.h, rank)) sink.push(x);
            }
            if ((uint32_t)lane == q) mycnt = before + __popc(bal);
        }
        const bool done = mypicks && mycnt > mylast;
        if ((__ballot_sync(0xFFFFFFFFu, done) & want_mask) == want_mask) break;
    }
    __syncwarp();
}

// Returns true when the pop must be handed to the block path.
template <class SM, class Sink>
__device__ bool pop_warp(const RRParams& P, SM& S, const Sink& sink, uint32_t j, uint32_t ybase, int32_t mu) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int4 vi = P.vinfo[mu];
    const int32_t pb = vi.x, l = vi.y, v_begin = vi.z, dh = vi.w;
    Need* need = S.wneed[wid];
    uint32_t nneed = 0, ndraw = 0;
    uint32_t hsum = 0;  // sum of h over the layers <= deg(mu) < 2^31
    const bool lt = P.strategy == HYPERIM_STRAT_LT;
    if (lt) {  // one kept in-neighbour at most: one need of h = 1 (ksel holds its position)
        int kept = 0, drew = 0;
        if (lane == 0) {
            Need nd;
            bool dr = false;
            kept = lt_keep(P, pb, l, j, ybase, mu, nd, &dr) ? 1 : 0;
            drew = dr ? 1 : 0;
            if (kept) need[0] = nd;
        }
        kept = __shfl_sync(0xFFFFFFFFu, kept, 0);
        ndraw = (uint32_t)__shfl_sync(0xFFFFFFFFu, drew, 0);
        nneed = (uint32_t)kept;
        hsum = lane == 0 ? (uint32_t)kept : 0u;
    }
    for (int c0 = 0; c0 < (lt ? 0 : l); c0 += 32) {
        const int i = c0 + lane;
        uint32_t h = 0, ksel = 0;
        uint4 e = make_uint4(0, 0, 0, 0);
        bool drew = false;
        if (i < l) {
            e = P.prof[2 * (pb + i)];
            const uint4 f = P.prof[2 * (pb + i) + 1];
            WordStream ws;
            ws.init(P.seed, j, ybase, (uint32_t)mu, (uint32_t)(i + 1));
            drew = layer_draw(e, f, P.tab, P.strategy, ws, h, ksel);
        }
        const bool flag = h > 0;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, flag);
        const uint32_t pos = nneed + __popc(bal & lanemask_lt());
        if (flag && pos < kLQ) need[pos] = Need{e.x & ~kPOneFlag, e.y, h, ksel, (uint32_t)(i + 1)};
        hsum += h;
        nneed += __popc(bal);
        ndraw += __popc(__ballot_sync(0xFFFFFFFFu, drew));
    }
    __syncwarp();
    unsigned long long* wst = S.wstat[wid];
    if (lane == 0) {
        wst[S_POPS] += 1;
        wst[S_LAYERS] += (unsigned long long)l;
        wst[S_DRAWS] += ndraw;
        wst[S_SECT] += sectors_of(12ull * (uint64_t)pb, 12ull * (uint64_t)l);
    }
    if (nneed == 0) return false;
    hsum = __reduce_add_sync(0xFFFFFFFFu, hsum);
    const int32_t tsum = P.tsum[mu];
    if (lane == 0) {
        wst[S_SEL] += hsum;
        wst[S_MATS] += 1;
        wst[S_MAT_HE] += (unsigned long long)dh;
        wst[S_MAT_MEM] += (unsigned long long)tsum;
        wst[S_GATH] += (unsigned long long)tsum;  // one pass over the members (the chunk path corrects it)
        wst[S_SECT] += P.mat_sect[mu];
    }
    if (nneed > kLQ) return true;
    // picks for every needed layer (none when h = n)
    uint32_t total_picks = 0, take_all_n = 0;
    for (uint32_t q = 0; q < nneed; ++q) {
        const Need nd = need[q];
        if (nd.h < nd.n) total_picks += nd.h; else take_all_n += nd.n;
        if (total_picks > kPCap) return true;
    }
    const int T = tsum - dh;
    // a chunk index lets the warp read only the id ranges that hold the picks (and the members
    // of layers taken whole, when there are few of them)
    uint64_t iw = 0;
    if (dh != 1 && T > kIdxMinT && total_picks + take_all_n <= (uint32_t)kPCap) iw = P.idx[mu];
    if (dh != 1 && iw == 0 && T > kWCap) return true;
    uint32_t* picks = S.u.w.wpick[wid];
    uint32_t* poff = S.wpoff[wid];
    uint32_t acc = 0;
    for (uint32_t q = 0; q < nneed; ++q) {
        const Need nd = need[q];
        if (lane == 0) poff[q] = acc;
        if (lt) {
            if (nd.h < nd.n) {
                if (lane == 0) picks[acc] = nd.ksel;
                acc += 1;
            }
            continue;
        }
        if (nd.h < nd.n) {
            if ((uint64_t)nd.ksel + nd.h > (1ull << 18)) {
                if (lane == 0) dev_fail(P.st, kErrWords, mu);
                return false;
            }
            WordStream ws;
            ws.init(P.seed, j, ybase, (uint32_t)mu, nd.layer);
            gen_picks(ws, nd.n, nd.h, nd.ksel, picks + acc);
            acc += nd.h;
        }
    }
    if (lane == 0) poff[nneed] = acc;
    __syncwarp();
    if (dh == 1) {
        // A(mu) = the single hyperedge minus mu, sorted: position x maps to member x or x + 1
        const int2 sp = P.v_span[v_begin];
        const int32_t hb = sp.x, len = sp.y;
        int pmu = 0;
        for (int b = 0; b < len; b += 32) {
            const bool lt = b + lane < len && (uint32_t)P.he_mem[hb + b + lane] < (uint32_t)mu;
            pmu += __popc(__ballot_sync(0xFFFFFFFFu, lt));
        }
        const Need nd = need[0];
        if (nd.h >= nd.n) {
            for (int x = lane; x < len - 1; x += 32)
                sink.push((uint32_t)P.he_mem[hb + x + (x >= pmu ? 1 : 0)]);
        } else {
            for (uint32_t r = lane; r < nd.h; r += 32) {
                const uint32_t x = picks[r];
                sink.push((uint32_t)P.he_mem[hb + x + ((int)x >= pmu ? 1 : 0)]);
            }
        }
        __syncwarp();
        return false;
    }
    uint32_t* buf = S.u.w.wbuf[wid];
    int* cnt = S.wcnt[wid];
    if (iw != 0) {
        // chunk path: lane q follows needed layer q through its row of prefix counts: the next
        // position it needs (its next pick, or for a layer taken whole its next member) and the
        // chunk holding it; the warp visits those chunks in ascending order, each ranked from the
        // row entries at that chunk
        const int c = (int)(iw >> kIdxBitsShift);
        const int C = 1 << c;
        const uint64_t toff = iw & ((1ull << kIdxBitsShift) - 1);
        const int sh = P.id_bits - c;
        uint32_t probes = 0, cur = 0xFFFFFFFFu, cursor = 0;
        unsigned long long gath = 0;
        Need nd{};
        const uint32_t* row = nullptr;
        uint32_t first = 0;
        if ((uint32_t)lane < nneed) {
            nd = need[lane];
            row = P.idx_tab + toff + ((uint64_t)(nd.layer - 1) << c);
            first = nd.h < nd.n ? picks[poff[lane]] : 0u;
        }
        {
            const int r0 = warp_chunk_search(row, 0, C, first, (uint32_t)lane < nneed, nneed, probes);
            if ((uint32_t)lane < nneed) cur = (uint32_t)r0;
        }
        uint32_t k = __reduce_min_sync(0xFFFFFFFFu, cur);
        int chunks = 0;
        while (k != 0xFFFFFFFFu) {
            if ((uint32_t)lane < nneed) {
                cnt[lane] = (int)row[k];
                ++probes;
            }
            __syncwarp();
            const int got = chunk_nbhd(P, S, mu, v_begin, dh, k << sh, sh, buf, probes);
            if (got < 0) {
                if (lane == 0) dev_fail(P.st, kErrBucket, mu);
                return false;
            }
            gath += (unsigned long long)got;
            warp_walk(P, S, sink, buf, got, nneed);
            ++chunks;
            uint32_t nxt = 0xFFFFFFFFu;
            const bool moved = cur == k;  // this lane's layer needs a later chunk (or none)
            if (moved) {
                const uint32_t endk = (int)k + 1 < C ? row[k + 1] : nd.n;  // members of L_q before chunk k + 1
                ++probes;
                if (nd.h < nd.n) {
                    const uint32_t* pk = picks + poff[lane];
                    while (cursor < nd.h && pk[cursor] < endk) ++cursor;
                    if (cursor < nd.h) nxt = pk[cursor];
                } else if (endk < nd.n) {
                    nxt = endk;
                }
            }
            {
                const bool want = moved && nxt != 0xFFFFFFFFu;
                const int r1 = warp_chunk_search(row, (int)k + 1, C, nxt, want, nneed, probes);
                if (moved) cur = want ? (uint32_t)r1 : 0xFFFFFFFFu;
            }
            k = __reduce_min_sync(0xFFFFFFFFu, cur);
        }
        probes = __reduce_add_sync(0xFFFFFFFFu, probes);
        if (lane == 0) {
            wst[S_GATH] += gath;
            wst[S_GATH] -= (unsigned long long)tsum;
            // span entries (2 words) of every chunk after the first are extra reads
            wst[S_SRCH] += (unsigned long long)probes + 2ull * (unsigned long long)dh * (chunks - 1);
        }
        return false;
    }
    // materialise A(mu) in shared memory, sorted by id (bucketed by the top id bits)
    int got;
    if (tsum <= kWHalf) {
        small_nbhd(P, S, mu, v_begin, dh, tsum, T, buf);
        got = T;
    } else {
        got = sorted_nbhd<32>(P.v_span, P.he_mem, mu, v_begin, dh, T, P.id_bits, buf,
                              S.u.w.wbkt[wid], kWBucketBits, S.wpre[wid], nullptr);
    }
    for (uint32_t q = lane; q < nneed; q += 32) cnt[q] = 0;
    __syncwarp();
    warp_walk(P, S, sink, buf, got, nneed);
    return false;
}

// ------------------------------------------------------------------------------------------
// block path (all threads of the block)
// ------------------------------------------------------------------------------------------
// layer index (among the needed layers of this round) of a run of multiplicity mult, or -1
__device__ __forceinline__ int needed_layer(const Shared& S, uint32_t nq, int mult) {
    for (uint32_t t = 0; t < nq; ++t)
        if (S.bneed[t].w == (uint32_t)mult) return (int)t;
    return -1;
}

// true when every needed layer with a strict subset of picks has ranked past its largest pick
__device__ __forceinline__ bool block_done(const Shared& S, uint32_t nq, const uint32_t* picks) {
    for (uint32_t t = 0; t < nq; ++t) {
        const Need nd = S.bneed[t];
        if (nd.h >= nd.n) return false;
        if ((uint32_t)S.lcnt[t] <= picks[S.bpick_off[t] + nd.h - 1]) return false;
    }
    return true;
}

// Ranked walk of a sorted block buffer: warp w owns positions [w L, (w + 1) L) and every run
// that starts there. Pass A counts the runs of each needed layer per warp, the counts are
// prefix-summed across warps (on top of the running layer ranks), pass B re-walks and pushes
// the runs whose rank is a pick. Returns (uniformly) whether all picks have been passed.
template <class Sink>
__device__ bool block_walk(const RRParams& P, Shared& S, const Sink& sink, const uint32_t* buf, int count,
                           uint32_t nq, const uint32_t* picks) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int L = (count + kWarps - 1) / kWarps;
    const int s0 = min(count, wid * L), s1 = min(count, s0 + L);
    for (uint32_t t = lane; t < nq; t += 32) S.wcnt[wid][t] = 0;
    __syncwarp();
    for (int base = s0; base < s1; base += 32) {
        const int p = base + lane;
        if (p < s1) {
            const uint32_t x = buf[p];
            if (p == 0 || buf[p - 1] != x) {
                int mult = 1;
                while (p + mult < count && buf[p + mult] == x) ++mult;
                const int q = needed_layer(S, nq, mult);
                if (q >= 0) atomicAdd(&S.wcnt[wid][q], 1);
            }
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < nq; t += kThreads) {
        int run = S.lcnt[t];
        for (int w = 0; w < kWarps; ++w) {
            const int c = S.wcnt[w][t];
            S.wcnt[w][t] = run;
            run += c;
        }
        S.lcnt[t] = run;
    }
    __syncthreads();
    for (int base = s0; base < s1; base += 32) {
        const int p = base + lane;
        int q = -1;
        uint32_t x = 0;
        if (p < s1) {
            x = buf[p];
            if (p == 0 || buf[p - 1] != x) {
                int mult = 1;
                while (p + mult < count && buf[p + mult] == x) ++mult;
                q = needed_layer(S, nq, mult);
            }
        }
        const uint32_t mask = __match_any_sync(0xFFFFFFFFu, q);
        const int rin = __popc(mask & lanemask_lt());
        if (q >= 0) {
            const Need nd = S.bneed[q];
            const uint32_t rank = (uint32_t)(S.wcnt[wid][q] + rin);
            if (nd.h >= nd.n || in_sorted(picks + S.bpick_off[q], nd.h, rank)) sink.push(x);
        }
        __syncwarp();
        if (q >= 0 && rin == 0) S.wcnt[wid][q] += __popc(mask);
        __syncwarp();
    }
    __syncthreads();
    return block_done(S, nq, picks);
}

template <class Sink>
__device__ __noinline__ void pop_block(const RRParams& P, Shared& S, const Sink& sink, uint32_t j,
                          uint32_t ybase, int32_t mu, uint32_t* picks_g, uint32_t* big) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int4 vi = P.vinfo[mu];
    const int32_t pb = vi.x, l = vi.y, v_begin = vi.z, dh = vi.w;
    // needed layers are processed kBLQ at a time; draws are recomputed per round
    for (uint32_t round_lo = 0;; round_lo += kBLQ) {
        if (wid == 0) {
            uint32_t nneed = 0;
            if (P.strategy == HYPERIM_STRAT_LT) {  // one need of h = 1, ksel = the kept position
                int kept = 0;
                if (lane == 0) {
                    Need nd;
                    bool dr = false;
                    kept = lt_keep(P, pb, l, j, ybase, mu, nd, &dr) ? 1 : 0;
                    if (kept) S.bneed[0] = nd;
                }
                nneed = (uint32_t)__shfl_sync(0xFFFFFFFFu, kept, 0);
            }
            for (int c0 = 0; c0 < (P.strategy == HYPERIM_STRAT_LT ? 0 : l); c0 += 32) {
                const int i = c0 + lane;
                uint32_t h = 0, ksel = 0;
                uint4 e = make_uint4(0, 0, 0, 0);
                if (i < l) {
                    e = P.prof[2 * (pb + i)];
                    const uint4 f = P.prof[2 * (pb + i) + 1];
                    WordStream ws;
                    ws.init(P.seed, j, ybase, (uint32_t)mu, (uint32_t)(i + 1));
                    layer_draw(e, f, P.tab, P.strategy, ws, h, ksel);
                }
                const bool flag = h > 0;
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, flag);
                const uint32_t pos = nneed + __popc(bal & lanemask_lt());
                if (flag && pos >= round_lo && pos < round_lo + kBLQ)
                    S.bneed[pos - round_lo] = Need{e.x & ~kPOneFlag, e.y, h, ksel, (uint32_t)(i + 1)};
                nneed += __popc(bal);
            }
            __syncwarp();
            if (lane == 0) {
                const uint32_t nq = nneed > round_lo ? min(nneed - round_lo, (uint32_t)kBLQ) : 0u;
                S.ctrl[C_NNEED] = (int)nq;
                S.ctrl[C_STOP] = nneed > round_lo + kBLQ ? 0 : 1;
                uint32_t acc = 0;
                for (uint32_t q = 0; q < nq; ++q) {
                    S.bpick_off[q] = acc;
                    if (S.bneed[q].h < S.bneed[q].n) acc += S.bneed[q].h;
                    S.lcnt[q] = 0;
                }
                S.bpick_off[nq] = acc;
                S.ctrl[C_OK] = (int64_t)acc <= P.pick_cap ? 1 : 0;
            }
        }
        __syncthreads();
        const uint32_t nq = (uint32_t)S.ctrl[C_NNEED];
        const bool last_round = S.ctrl[C_STOP] != 0;
        if (!S.ctrl[C_OK]) {
            if (threadIdx.x == 0) dev_fail(P.st, kErrCapacity, mu);
            __syncthreads();
            return;
        }
        if (nq > 0) {
            // picks: warp q % kWarps generates layer q
            for (uint32_t q = wid; q < nq; q += kWarps) {
                const Need nd = S.bneed[q];
                if (P.strategy == HYPERIM_STRAT_LT) {
                    if (nd.h < nd.n && lane == 0) picks_g[S.bpick_off[q]] = nd.ksel;
                    continue;
                }
                if (nd.h < nd.n) {
                    if ((uint64_t)nd.ksel + nd.h > (1ull << 18)) {
                        if (lane == 0) dev_fail(P.st, kErrWords, mu);
                        continue;
                    }
                    WordStream ws;
                    ws.init(P.seed, j, ybase, (uint32_t)mu, nd.layer);
                    gen_picks(ws, nd.n, nd.h, nd.ksel, picks_g + S.bpick_off[q]);
                }
            }
            __threadfence_block();
            __syncthreads();
            if (dh == 1) {
                const int2 sp = P.v_span[v_begin];
                const int32_t hb = sp.x, len = sp.y;
                if (threadIdx.x == 0) S.ctrl[C_CURSOR] = 0;
                __syncthreads();
                for (int b = threadIdx.x; b < len; b += kThreads)
                    if ((uint32_t)P.he_mem[hb + b] < (uint32_t)mu) atomicAdd(&S.ctrl[C_CURSOR], 1);
                __syncthreads();
                const int pmu = S.ctrl[C_CURSOR];
                const Need nd = S.bneed[0];
                if (nd.h >= nd.n) {
                    for (int x = threadIdx.x; x < len - 1; x += kThreads)
                        sink.push((uint32_t)P.he_mem[hb + x + (x >= pmu ? 1 : 0)]);
                } else {
                    for (uint32_t r = threadIdx.x; r < nd.h; r += kThreads) {
                        const uint32_t x = picks_g[r];
                        sink.push((uint32_t)P.he_mem[hb + x + ((int)x >= pmu ? 1 : 0)]);
                    }
                }
                __syncthreads();
            } else {
                const int T = P.tsum[mu] - dh;
                if (T <= kBCap) {
                    const int got = sorted_nbhd<kThreads>(P.v_span, P.he_mem, mu, v_begin, dh, T,
                                                          P.id_bits, S.u.b.bbuf, S.u.b.bucket,
                                                          kBucketBits, S.u.b.bpre, S.tmp);
                    block_walk(P, S, sink, S.u.b.bbuf, got, nq, picks_g);
                } else if ((int64_t)T > P.big_cap) {
                    if (threadIdx.x == 0) dev_fail(P.st, kErrCapacity, mu);
                } else {
                    // first level: chunk by the top b id bits so every chunk fits on chip
                    int b = 0;
                    while (((int64_t)(kBCap / 2) << b) < (int64_t)T && b < P.id_bits &&
                           (2 << b) <= kChunks)
                        ++b;
                    bool ok = false;
                    for (;;) {
                        const int nb = 1 << b, shift = P.id_bits - b;
                        for (int i = threadIdx.x; i < nb; i += kThreads) S.u.b.chunk_end[i] = 0;
                        __syncthreads();
                        for_each_member<kThreads>(P.v_span, P.he_mem, mu, v_begin, dh, S.u.b.bpre,
                                                  [&](uint32_t x) { atomicAdd(&S.u.b.chunk_end[x >> shift], 1); });
                        int mx = 0;
                        for (int i = threadIdx.x; i < nb; i += kThreads) mx = max(mx, S.u.b.chunk_end[i]);
                        mx = __reduce_max_sync(0xFFFFFFFFu, mx);
                        if (lane == 0) S.tmp[wid] = mx;
                        __syncthreads();
                        int allmx = 0;
                        for (int w = 0; w < kWarps; ++w) allmx = max(allmx, S.tmp[w]);
                        __syncthreads();
                        if (allmx <= kBCap) { ok = true; break; }
                        if (b >= P.id_bits || (2 << b) > kChunks) break;
                        ++b;
                    }
                    if (!ok) {
                        if (threadIdx.x == 0) dev_fail(P.st, kErrBucket, mu);
                    } else {
                        const int nb = 1 << b, shift = P.id_bits - b;
                        if (wid == 0) {
                            int carry = 0;
                            for (int base = 0; base < nb; base += 32) {
                                const int i = base + lane;
                                const int v = i < nb ? S.u.b.chunk_end[i] : 0;
                                int inc = v;
                                for (int o = 1; o < 32; o <<= 1) {
                                    const int t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                                    if (lane >= o) inc += t;
                                }
                                if (i < nb) S.u.b.chunk_end[i] = carry + inc - v;
                                carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
                            }
                        }
                        __syncthreads();
                        for_each_member<kThreads>(P.v_span, P.he_mem, mu, v_begin, dh, S.u.b.bpre,
                                                  [&](uint32_t x) { big[atomicAdd(&S.u.b.chunk_end[x >> shift], 1)] = x; });
                        __threadfence_block();
                        __syncthreads();
                        // second level: each chunk bucketed on chip by the next id bits
                        int begin = 0;
                        for (int qb = 0; qb < nb; ++qb) {
                            const int end = S.u.b.chunk_end[qb];
                            const int cnt = end - begin;
                            if (cnt > 0) {
                                sort_chunk<kThreads>(big + begin, cnt, shift, S.u.b.bbuf, S.u.b.bucket,
                                                     kBucketBits, S.tmp);
                                const bool stop = block_walk(P, S, sink, S.u.b.bbuf, cnt, nq, picks_g);
                                if (stop) break;
                            }
                            begin = end;
                        }
                    }
                }
                __syncthreads();
            }
        }
        __syncthreads();
        if (last_round) break;
    }
}

// ------------------------------------------------------------------------------------------
// forward Monte-Carlo influence (the Sec. 2.2 cascade under the IC model)
// ------------------------------------------------------------------------------------------
// One coin per directed pair u -> v and simulation r: word 0 of Philox4x32-10 with the forward
// key and counter (r, u, v, 0xFFFFFFFE) (no RR counter has that last word). The pair is live
// with the probability of u's layer in A(v): the layer of v's profile keyed by w(u, v).
struct FwdParams {
    RRParams P;           // graph arrays, queue scratch, status (RR-only fields unused)
    const int32_t* seeds;
    int32_t k;
    uint64_t nsims;
    uint32_t key0, key1;
    uint32_t* counts;
};

__device__ __forceinline__ bool fwd_live(const RRParams& P, uint32_t key0, uint32_t key1, uint32_t r,
                                         uint32_t u, uint32_t v, uint32_t w) {
    const int4 vv = P.vinfo[v];
    int lo = 0, hi = vv.y;  // v's layers by descending w: the one keyed by w
    uint4 e = make_uint4(0, 0, 0, 0);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        e = P.prof[2 * ((int64_t)vv.x + mid)];
        const uint32_t wm = e.x & ~kPOneFlag;
        if (wm == w) { lo = mid; break; }
        if (wm > w) lo = mid + 1; else hi = mid;
    }
    if ((e.x & ~kPOneFlag) != w) return false;  // unreachable: w(u, v) keys a layer of A(v)
    if (e.x & kPOneFlag) return true;
    if (e.z == 0) return false;
    const uint4 word = philox10(make_uint4(r, u, v, 0xFFFFFFFEu), key0, key1);
    return word.x < e.z;
}

// runs of a sorted buffer of u's neighbours: each distinct v (multiplicity w(u, v)) flips its coin
__device__ void fwd_walk(const FwdParams& F, Shared& S, uint32_t* vis, int32_t* list, const uint32_t* buf,
                         int got, uint32_t r, uint32_t u) {
    const int lane = threadIdx.x & 31;
    for (int base = 0; base < got; base += 32) {
        const int p = base + lane;
        if (p < got) {
            const uint32_t x = buf[p];
            if (p == 0 || buf[p - 1] != x) {
                int mult = 1;
                while (p + mult < got && buf[p + mult] == x) ++mult;
                if (fwd_live(F.P, F.key0, F.key1, r, u, x, (uint32_t)mult)) push(F.P, S, vis, list, x);
            }
        }
    }
    __syncwarp();
}

// One activated vertex u: all of A(u) with multiplicities, in id order, then the coins. Large
// neighbourhoods are taken id range by id range (ranges of expected 256 members; a range that
// still exceeds the warp's buffer is split into 16).
__device__ void fwd_pop_warp(const FwdParams& F, Shared& S, uint32_t* vis, int32_t* list, uint32_t r,
                             int32_t u) {
    const RRParams& P = F.P;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int4 vi = P.vinfo[u];
    const int32_t v_begin = vi.z, dh = vi.w;
    if (dh == 0) return;
    const int32_t tsum = P.tsum[u];
    const int T = tsum - dh;
    if (T == 0) return;
    uint32_t* buf = S.u.w.wbuf[wid];
    if (dh == 1) {
        const int2 sp = P.v_span[v_begin];
        for (int x = lane; x < sp.y; x += 32) {
            const uint32_t v = (uint32_t)P.he_mem[sp.x + x];
            if (v != (uint32_t)u && fwd_live(P, F.key0, F.key1, r, (uint32_t)u, v, 1u)) push(P, S, vis, list, v);
        }
        __syncwarp();
        return;
    }
    if (tsum <= kWHalf) {
        small_nbhd(P, S, u, v_begin, dh, tsum, T, buf);
        fwd_walk(F, S, vis, list, buf, T, r, (uint32_t)u);
        return;
    }
    if (T <= kWCap) {
        const int got = sorted_nbhd<32>(P.v_span, P.he_mem, u, v_begin, dh, T, P.id_bits, buf,
                                        S.u.w.wbkt[wid], kWBucketBits, S.wpre[wid], nullptr);
        fwd_walk(F, S, vis, list, buf, got, r, (uint32_t)u);
        return;
    }
    int b = 0;
    while (b < P.id_bits && (256 << b) < T) ++b;
    const int sh = P.id_bits - b;
    uint32_t probes = 0;
    for (uint32_t k = 0; k < (1u << b); ++k) {
        const int got = chunk_nbhd(P, S, u, v_begin, dh, k << sh, sh, buf, probes);
        if (got >= 0) {
            fwd_walk(F, S, vis, list, buf, got, r, (uint32_t)u);
            continue;
        }
        const int sh2 = sh >= 4 ? sh - 4 : 0;
        for (uint32_t k2 = 0; k2 < (1u << (sh - sh2)); ++k2) {
            const int got2 = chunk_nbhd(P, S, u, v_begin, dh, (k << sh) + (k2 << sh2), sh2, buf, probes);
            if (got2 < 0) {
                if (lane == 0) dev_fail(P.st, kErrBucket, u);
                return;
            }
            fwd_walk(F, S, vis, list, buf, got2, r, (uint32_t)u);
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1) k_forward(FwdParams F) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RRParams& P = F.P;
    Shared& S = *reinterpret_cast<Shared*>(smem_raw);
    uint32_t* vis = P.vis_smem ? reinterpret_cast<uint32_t*>(smem_raw + sizeof(Shared))
                               : P.gvis + (int64_t)blockIdx.x * P.vis_words;
    int32_t* list = P.list + (int64_t)blockIdx.x * P.list_cap;
    const int lane = threadIdx.x & 31;
    for (int64_t w = threadIdx.x; w < P.vis_words; w += kThreads) vis[w] = 0;
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long t = atomicAdd(reinterpret_cast<unsigned long long*>(P.next_job), 1ull);
            S.ctrl[C_JOB] = t < F.nsims ? (int)(t & 0x7FFFFFFF) : -1;
            S.out_pos = t;
            S.ctrl[C_HEAD] = 0;
            S.ctrl[C_TAIL] = 0;
            S.ctrl[C_DONE] = 0;
            S.ctrl[C_NDEF] = 0;
        }
        __syncthreads();
        if (S.ctrl[C_JOB] < 0) break;
        const uint32_t r = (uint32_t)S.out_pos;
        for (int i = threadIdx.x; i < F.k; i += kThreads) push(P, S, vis, list, (uint32_t)F.seeds[i]);
        __syncthreads();
        for (;;) {
            int idx = 0;
            if (lane == 0) idx = claim_slot(P, S, (int64_t)r);
            idx = __shfl_sync(0xFFFFFFFFu, idx, 0);
            if (idx < 0) break;
            int32_t u = 0;
            if (lane == 0) u = slot_value(P, list, idx, (int64_t)r);
            u = __shfl_sync(0xFFFFFFFFu, u, 0);
            if (u >= 0) fwd_pop_warp(F, S, vis, list, r, u);
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();  // this pop's pushes before its completion
                atomicAdd(&S.ctrl[C_DONE], 1);
            }
        }
        __syncthreads();
        const int size = S.ctrl[C_TAIL];
        if (threadIdx.x == 0) F.counts[r] = (uint32_t)size;
        for (int i = threadIdx.x; i < size; i += kThreads) {
            const int32_t v = __ldcg(list + i);
            if (v >= 0) vis[v >> 5] = 0;
            list[i] = -1;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// the kernels
// ------------------------------------------------------------------------------------------
// A job (an RR set of one of the launch's pools): its pool, stratum, index j in the stratum and
// the y word of its Philox counters.
struct Job {
    int pi, s;
    uint32_t j, ybase;
};

__device__ __forceinline__ Job decode_job(const RRParams& P, int64_t job) {
    Job J;
    J.pi = 0;
    while (J.pi + 1 < P.npools && job >= P.pool_start[J.pi + 1]) ++J.pi;
    const RRJobMap& jm = P.jm[J.pi];
    const int64_t local = job - P.pool_start[J.pi];
    J.s = 0;
    while (J.s < HYPERIM_NSTRATA - 1 && local >= jm.job_base[J.s + 1]) ++J.s;
    J.j = jm.j_base[J.s] + (uint32_t)(local - jm.job_base[J.s]) * jm.j_step;
    const uint32_t sfield = P.root_mode == HYPERIM_ROOTS_PLAIN ? 0xFFu : (uint32_t)J.s;
    J.ybase = stream_ybase(P.tags[J.pi], sfield);
    return J;
}

// the root of a job: uniform over its stratum (multiply-shift of one word), or over V
__device__ __forceinline__ int32_t draw_root(const RRParams& P, const Job& J) {
    WordStream ws;
    ws.init(P.seed, J.j, J.ybase, 0xFFFFFFFFu, 0u);
    const uint32_t w0 = ws.word(0);
    if (P.root_mode == HYPERIM_ROOTS_PLAIN) return (int32_t)(((uint64_t)w0 * (uint64_t)(uint32_t)P.n) >> 32);
    const int32_t b = P.vs_off[J.s], size = P.vs_off[J.s + 1] - b;
    return P.vs_list[b + (int32_t)(((uint64_t)w0 * (uint64_t)(uint32_t)size) >> 32)];
}

// Shared memory of the warp phase: the warp-path buffers of every warp, plus each warp's own
// RR set (member set, queue, size).
struct WarpShared {
    unsigned long long stat[kMaxPools][kNStat];  // per pool work counters of this block
    unsigned long long wstat[kPWarps][kNStat];    // per-warp counters of the warp's current set
    Need wneed[kPWarps][kLQ];
    int wpre[kPWarps][3 * kCG + 1];
    uint32_t wpoff[kPWarps][kLQ + 1];
    int wcnt[kPWarps][kBLQ];
    int wtail[kPWarps];
    int32_t whash[kPWarps][kWHash];
    int32_t wqueue[kPWarps][kWQ];
    union {
        WarpAreaT<kPWarps> w;
    } u;
};

// Warp phase of RR generation: every warp takes jobs from the launch's counter and builds each
// RR set alone -- pops in queue order, activations into its own member set -- while the set
// stays within kWQ members and no pop needs the block path. Such sets are written out at once;
// any other job is listed for the block phase (k_rr with block_phase), which builds it again
// from its root (the draws are keyed by (RR, vertex, layer), so the set is the same) and the warp's
// partial counters are dropped. Jobs are taken from the last one down, as in k_rr.
__global__ void __launch_bounds__(kPThreads, 2) k_rr_warp(RRParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpShared& S = *reinterpret_cast<WarpShared*>(smem_raw);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t njobs = P.pool_start[P.npools];
    if (threadIdx.x < kMaxPools * kNStat) (&S.stat[0][0])[threadIdx.x] = 0;
    if (threadIdx.x < kPWarps * kNStat) (&S.wstat[0][0])[threadIdx.x] = 0;
    for (int i = threadIdx.x; i < kPWarps * kWHash; i += kPThreads) (&S.whash[0][0])[i] = -1;
    __syncthreads();
    int32_t* hash = S.whash[wid];
    int32_t* queue = S.wqueue[wid];
    int* tail = &S.wtail[wid];
    const WarpSink sink{hash, queue, tail, P.warp_limit};
    unsigned long long* wst = S.wstat[wid];
    for (;;) {
        int64_t ticket = 0;
        if (lane == 0) ticket = atomicAdd(P.next_job, 1);
        ticket = __shfl_sync(0xFFFFFFFFu, ticket, 0);
        if (ticket >= njobs) break;
        const int64_t job = njobs - 1 - ticket;
        const Job J = decode_job(P, job);
        if (lane == 0) {
            const int32_t root = draw_root(P, J);
            *tail = 0;
            sink.push((uint32_t)root);
        }
        __syncwarp();
        bool escalate = false;
        for (int head = 0;; ++head) {
            const int t = *(volatile int*)tail;
            if (t > P.warp_limit) { escalate = true; break; }
            if (head >= t) break;
            const int32_t mu = queue[head];
            if (pop_warp(P, S, sink, J.j, J.ybase, mu)) { escalate = true; break; }
            __syncwarp();
            if (*(volatile int32_t*)&P.st->code != 0) break;  // a failure elsewhere: stop early
        }
        __syncwarp();
        const int size = min(*(volatile int*)tail, P.warp_limit);
        if (escalate) {
            if (lane == 0) P.esc_list[atomicAdd(P.esc_count, 1)] = (int32_t)job;
        } else {
            // output: the members in ascending order
            uint32_t* buf = S.u.w.wbuf[wid];
            for (int i = lane; i < size; i += 32) buf[i] = (uint32_t)queue[i];
            __syncwarp();
            group_sort<32>(buf, size);
            unsigned long long pos = 0;
            if (lane == 0) {
                pos = atomicAdd(P.arena_used, (unsigned long long)size);
                P.out_pos[job] = (int64_t)pos;
                P.out_size[job] = size;
            }
            pos = __shfl_sync(0xFFFFFFFFu, pos, 0);
            if (pos + (unsigned long long)size <= P.arena_cap)
                for (int i = lane; i < size; i += 32) P.arena[pos + i] = (int32_t)buf[i];
            if (lane < kNStat) atomicAdd(&S.stat[J.pi][lane], wst[lane]);
        }
        __syncwarp();
        if (lane < kNStat) wst[lane] = 0;
        for (int i = lane; i < kWHash; i += 32) hash[i] = -1;
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < P.npools) {
        RRCounters* c = P.counters + threadIdx.x;
        const unsigned long long* st = S.stat[threadIdx.x];
        atomicAdd(&c->pops, st[S_POPS]);
        atomicAdd(&c->layers_seen, st[S_LAYERS]);
        atomicAdd(&c->draws, st[S_DRAWS]);
        atomicAdd(&c->mats, st[S_MATS]);
        atomicAdd(&c->mat_he, st[S_MAT_HE]);
        atomicAdd(&c->mat_members, st[S_MAT_MEM]);
        atomicAdd(&c->selected, st[S_SEL]);
        atomicAdd(&c->gathered, st[S_GATH]);
        atomicAdd(&c->search_words, st[S_SRCH]);
        atomicAdd(&c->sectors, st[S_SECT]);
    }
}

// Output of a finished RR set of `size` members (its queue holds them, its visited bitmap marks
// them): an arena slot for the job, the members in ascending order (sorted on chip up to kBCap,
// else read off the bitmap in id order), and the bitmap cleared again. Whole block. The queue, and
// the bitmap when it is in global memory, were written by other warps through L2 (volatile stores,
// atomics): they are read with L2 loads, never from a possibly stale L1 line.
__device__ void write_set(const RRParams& P, Shared& S, uint32_t* vis, const int32_t* list, int size, int64_t job) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        unsigned long long pos;
        if (P.rewrite) {
            // the slot the first launch reserved for this set (the same set: keyed draws)
            pos = (unsigned long long)P.out_pos[job];
            if (P.out_size[job] != size) dev_fail(P.st, kErrCapacity, (int32_t)job);
        } else {
            pos = atomicAdd(P.arena_used, (unsigned long long)size);
            P.out_pos[job] = (int64_t)pos;
            P.out_size[job] = size;
        }
        S.ctrl[C_ROOT] = pos + (unsigned long long)size <= P.arena_cap ? 1 : 0;
        S.out_pos = pos;
    }
    __syncthreads();
    const bool fits = S.ctrl[C_ROOT] != 0;
    const unsigned long long pos = S.out_pos;
    if (size <= kBCap) {
        for (int i = threadIdx.x; i < size; i += kThreads) S.u.b.bbuf[i] = (uint32_t)__ldcg(list + i);
        __syncthreads();
        group_sort<kThreads>(S.u.b.bbuf, size);
        if (fits)
            for (int i = threadIdx.x; i < size; i += kThreads) P.arena[pos + i] = (int32_t)S.u.b.bbuf[i];
        __syncthreads();
        for (int i = threadIdx.x; i < size; i += kThreads) vis[S.u.b.bbuf[i] >> 5] = 0;
    } else {
        // R is large: read it off the visited bitmap in id order
        const int64_t nwords = ((int64_t)P.n + 31) >> 5;
        int64_t carry = 0;
        for (int64_t b0 = 0; b0 < nwords; b0 += kThreads) {
            const int64_t wi = b0 + threadIdx.x;
            const uint32_t word = wi >= nwords ? 0u : P.vis_smem ? vis[wi] : (uint32_t)__ldcg(vis + wi);
            int total;
            // exclusive sum of popcounts across the block
            const int c = __popc(word);
            int incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane == 31) S.tmp[wid] = incl;
            __syncthreads();
            int woff = 0;
            total = 0;
            for (int w = 0; w < kWarps; ++w) {
                woff += w < wid ? S.tmp[w] : 0;
                total += S.tmp[w];
            }
            __syncthreads();
            int64_t o = carry + woff + incl - c;
            uint32_t bits = word;
            while (bits) {
                const int bpos = __ffs(bits) - 1;
                bits &= bits - 1;
                if (fits) P.arena[pos + o] = (int32_t)(wi * 32 + bpos);
                ++o;
            }
            carry += total;
        }
        __syncthreads();
        for (int64_t w = threadIdx.x; w < nwords; w += kThreads) vis[w] = 0;
    }
}

// One RR set (job `job` of P's pools) built by the whole block: root draw, reverse BFS over the
// block's asynchronous queue, output. Work counters go to the block's per-pool totals (flushed at
// the end of the launch), or straight to the pool's counters when kFlushPerSet (a launch over the
// pools of many graphs, whose blocks change graphs from set to set).
template <bool kFlushPerSet>
__device__ __forceinline__ void run_job(const RRParams& P, Shared& S, uint32_t* vis, int32_t* list,
                                        uint32_t* picks_g, uint32_t* big, int64_t job) {
    const int lane = threadIdx.x & 31;
    const Job J = decode_job(P, job);
    const int pi = J.pi;
    const uint32_t j = J.j, ybase = J.ybase;
    if (threadIdx.x == 0) {
        S.cyc_start = clock64();
        const int32_t root = draw_root(P, J);
        list[0] = root;
        vis[root >> 5] |= 1u << (root & 31);
        S.ctrl[C_HEAD] = 0;
        S.ctrl[C_TAIL] = 1;
        S.ctrl[C_DONE] = 0;
        S.ctrl[C_NDEF] = 0;
    }
    __syncthreads();
    // reverse BFS over an asynchronous queue: a warp pops any vertex already discovered
    // (the draws are keyed by (RR, vertex, layer), so the order of pops does not change R);
    // the block only meets when every pending pop needs the block path
    for (;;) {
        for (;;) {
            int idx = 0;
            if (lane == 0) idx = claim_slot(P, S, job);
            idx = __shfl_sync(0xFFFFFFFFu, idx, 0);
            if (idx < 0) break;
            int32_t mu = 0;
            if (lane == 0) mu = slot_value(P, list, idx, job);
            mu = __shfl_sync(0xFFFFFFFFu, mu, 0);
            const bool defer = mu >= 0 && pop_warp(P, S, QueueSink{vis, list, &S.ctrl[C_TAIL]}, j, ybase, mu);
            __syncwarp();
            if (lane == 0) {
                if (defer) {
                    S.deferred[atomicAdd(&S.ctrl[C_NDEF], 1)] = mu;
                } else {
                    __threadfence_block();  // this pop's pushes before its completion
                    atomicAdd(&S.ctrl[C_DONE], 1);
                }
            }
        }
        if (threadIdx.x == 0) S.ctrl[C_FAIL] = *(volatile int32_t*)&P.st->code != 0;
        __syncthreads();
        if (S.ctrl[C_DONE] == S.ctrl[C_TAIL] || S.ctrl[C_FAIL]) break;  // R is complete (or failed)
        // the block materialises the deferred pops
        const int ndef = S.ctrl[C_NDEF];
        for (int d = 0; d < ndef; ++d)
            pop_block(P, S, QueueSink{vis, list, &S.ctrl[C_TAIL]}, j, ybase, S.deferred[d], picks_g, big);
        __syncthreads();
        if (threadIdx.x == 0) {
            S.ctrl[C_DONE] += ndef;
            S.ctrl[C_NDEF] = 0;
        }
        __syncthreads();
    }
    // work counters of this RR set go to its pool
    if (threadIdx.x < kNStat) {
        unsigned long long sum = 0;
        for (int w = 0; w < kWarps; ++w) {
            sum += S.wstat[w][threadIdx.x];
            S.wstat[w][threadIdx.x] = 0;
        }
        if (kFlushPerSet) {
            if (sum && !P.rewrite) atomicAdd(&P.counters[pi].pops + threadIdx.x, sum);
        } else {
            S.stat[pi][threadIdx.x] += sum;
        }
    }
    // output: members in ascending order
    const int size = S.ctrl[C_TAIL];
    write_set(P, S, vis, list, size, job);
    for (int i = threadIdx.x; i < size; i += kThreads) list[i] = -1;  // queue slots empty again
    if (!kFlushPerSet && threadIdx.x == 0) {
        // the set's duration on this SM (its launch's scheduling uses the mean and the maximum)
        const unsigned long long d = (unsigned long long)(clock64() - S.cyc_start);
        S.cyc_sum += d;
        S.cyc_max = d > S.cyc_max ? d : S.cyc_max;
        S.cyc_count += 1;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 1) k_rr(RRParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shared& S = *reinterpret_cast<Shared*>(smem_raw);
    uint32_t* vis = P.vis_smem ? reinterpret_cast<uint32_t*>(smem_raw + sizeof(Shared))
                               : P.gvis + (int64_t)blockIdx.x * P.vis_words;
    int32_t* list = P.list + (int64_t)blockIdx.x * P.list_cap;
    uint32_t* picks_g = P.picks + (int64_t)blockIdx.x * P.pick_cap;
    uint32_t* big = P.big + (int64_t)blockIdx.x * P.big_cap;
    const int64_t njobs = P.block_phase ? (int64_t)*(volatile int*)P.esc_count : P.pool_start[P.npools];
    if (threadIdx.x < kMaxPools * kNStat) (&S.stat[0][0])[threadIdx.x] = 0;
    if (threadIdx.x < kWarps * kNStat) (&S.wstat[0][0])[threadIdx.x] = 0;
    if (threadIdx.x == 0) S.cyc_sum = S.cyc_max = S.cyc_count = 0;
    for (int64_t w = threadIdx.x; w < P.vis_words; w += kThreads) vis[w] = 0;
    __syncthreads();
    int64_t plain_ticket = P.plain_base + blockIdx.x;  // the plain schedule's one job
    for (;;) {
        // jobs are handed out from the last one down: strata ascend with the job index, and the
        // high strata (roots with many layers, usually the costliest sets) should start first so
        // that cheap sets fill the end of the launch
        if (threadIdx.x == 0) {
            if (P.plain) {
                S.ctrl[C_JOB] = (int)plain_ticket;
                plain_ticket = njobs;
            } else {
                S.ctrl[C_JOB] = atomicAdd(P.next_job + P.block_phase, 1);
            }
        }
        __syncthreads();
        const int64_t ticket = S.ctrl[C_JOB];
        if (ticket >= njobs) break;
        // the block phase takes the jobs the warp phase listed, in listed order
        const int64_t job = P.block_phase ? (int64_t)P.esc_list[ticket] : njobs - 1 - ticket;
        run_job<false>(P, S, vis, list, picks_g, big, job);
    }
    __syncthreads();
    if (threadIdx.x < P.npools && !P.rewrite) {
        RRCounters* c = P.counters + threadIdx.x;
        const unsigned long long* st = S.stat[threadIdx.x];
        for (int i = 0; i < kNStat; ++i)
            if (st[i]) atomicAdd(&c->pops + i, st[i]);
    }
    if (threadIdx.x == 0 && P.set_cycles && !P.rewrite && S.cyc_count) {
        atomicAdd(P.set_cycles, S.cyc_sum);
        atomicMax(P.set_cycles + 1, S.cyc_max);
        atomicAdd(P.set_cycles + 2, S.cyc_count);
    }
}

// The jobs whose sets did not fit in an arena of `cap` entries (slot [pos, pos + size) past it).
__global__ void k_overflow_jobs(const int64_t* __restrict__ pos, const int32_t* __restrict__ size, int64_t njobs,
                                uint64_t cap, int32_t* __restrict__ list, int* __restrict__ count) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < njobs;
         j += (int64_t)gridDim.x * blockDim.x)
        if ((uint64_t)pos[j] + (uint64_t)size[j] > cap) list[atomicAdd(count, 1)] = (int32_t)j;
}

// A launch over the pools of several graphs (the batched form of HyperIM_BRR: every query's
// round grows its graph's pools, all in one launch). Group g -- one graph and up to kMaxPools of
// its pools -- owns the global jobs [group_start[g], group_start[g + 1]) and its own RRParams
// (graph arrays, job maps, outputs, counters); the blocks share one work counter, one output
// arena and one set of scratch buffers sized for the largest graph. A block copies the group of
// its current job into shared memory and builds the set exactly as k_rr does.
struct RRBatchParams {
    const RRParams* groups;
    const int64_t* group_start;  // ngroups + 1
    int ngroups;
    int* next_job;
    const int32_t* rerun;        // a repair launch: the global jobs to build again (else null)
    const int* rerun_count;
    int32_t* list;
    int64_t list_cap;
    uint32_t* gvis;
    int vis_smem;
    int64_t vis_words;
    uint32_t* picks;
    int64_t pick_cap;
    uint32_t* big;
    int64_t big_cap;
};

__global__ void __launch_bounds__(kThreads, 1) k_rr_batch(RRBatchParams B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) RRParams Pc;  // the current job's group
    Shared& S = *reinterpret_cast<Shared*>(smem_raw);
    uint32_t* vis = B.vis_smem ? reinterpret_cast<uint32_t*>(smem_raw + sizeof(Shared))
                               : B.gvis + (int64_t)blockIdx.x * B.vis_words;
    int32_t* list = B.list + (int64_t)blockIdx.x * B.list_cap;
    uint32_t* picks_g = B.picks + (int64_t)blockIdx.x * B.pick_cap;
    uint32_t* big = B.big + (int64_t)blockIdx.x * B.big_cap;
    const int64_t njobs = B.group_start[B.ngroups];
    const int64_t ntickets = B.rerun ? (int64_t)*(volatile const int*)B.rerun_count : njobs;
    if (threadIdx.x < kWarps * kNStat) (&S.wstat[0][0])[threadIdx.x] = 0;
    for (int64_t w = threadIdx.x; w < B.vis_words; w += kThreads) vis[w] = 0;
    __syncthreads();
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) S.ctrl[C_JOB] = atomicAdd(B.next_job, 1);
        __syncthreads();
        const int64_t ticket = S.ctrl[C_JOB];
        if (ticket >= ntickets) break;
        const int64_t gjob = B.rerun ? (int64_t)B.rerun[ticket] : njobs - 1 - ticket;
        int lo = 0, hi = B.ngroups - 1;  // the group holding gjob: last start <= gjob
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B.group_start[mid] <= gjob) lo = mid;
            else hi = mid - 1;
        }
        if (lo != cur) {  // the previous set ended with a barrier: Pc is free
            const uint32_t* src = reinterpret_cast<const uint32_t*>(B.groups + lo);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&Pc);
            for (int i = threadIdx.x; i < (int)(sizeof(RRParams) / 4); i += kThreads) dst[i] = src[i];
            cur = lo;
            __syncthreads();
        }
        run_job<true>(Pc, S, vis, list, picks_g, big, gjob - B.group_start[lo]);
    }
}

}  // namespace
}  // namespace hyperim

namespace hyperim {
namespace {

// Copy each RR set of the batch from the arena to its CSR slot; record stratum and index.
__global__ void k_compact_rr(const int32_t* __restrict__ arena, const int64_t* __restrict__ out_pos,
                             const int64_t* __restrict__ boff, int64_t njobs, int64_t base_count,
                             int64_t base_total, RRJobMap jm, int64_t* __restrict__ rr_off,
                             int32_t* __restrict__ rr_mem, uint8_t* __restrict__ rr_stratum,
                             uint32_t* __restrict__ rr_j) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < njobs; r += nwarps) {
        const int64_t src = out_pos[r], dst = base_total + boff[r], len = boff[r + 1] - boff[r];
        for (int64_t i = lane; i < len; i += 32) rr_mem[dst + i] = arena[src + i];
        if (lane == 0) {
            int s = 0;
            while (s < HYPERIM_NSTRATA - 1 && r >= jm.job_base[s + 1]) ++s;
            rr_off[base_count + r] = dst;
            rr_stratum[base_count + r] = (uint8_t)s;
            rr_j[base_count + r] = jm.j_base[s] + (uint32_t)(r - jm.job_base[s]) * jm.j_step;
            if (r == njobs - 1) rr_off[base_count + njobs] = base_total + boff[njobs];
        }
    }
}

// The batched form's compaction: every pool of a launch in one kernel. Pool d's new sets are the
// global jobs [job_begin, job_begin + jobs); boff is the exclusive scan of all the launch's set
// sizes; the pool's arrays were grown beforehand.
struct CompactDesc {
    int64_t job_begin, jobs, boff_begin, base_count, base_total;
    int64_t* rr_off;
    int32_t* rr_mem;
    uint8_t* rr_stratum;
    uint32_t* rr_j;
    RRJobMap jm;
};

__global__ void k_compact_batch(const int32_t* __restrict__ arena, const int64_t* __restrict__ out_pos,
                                const int64_t* __restrict__ boff, int64_t njobs, const CompactDesc* __restrict__ D,
                                int nd) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < njobs; r += nwarps) {
        int lo = 0, hi = nd - 1;  // the pool holding job r: last job_begin <= r
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (D[mid].job_begin <= r) lo = mid;
            else hi = mid - 1;
        }
        const CompactDesc& d = D[lo];
        const int64_t local = r - d.job_begin;
        if (local < 0 || local >= d.jobs) continue;  // jobs of pools not listed (none by construction)
        const int64_t src = out_pos[r], len = boff[r + 1] - boff[r];
        const int64_t dst = d.base_total + (boff[r] - d.boff_begin);
        for (int64_t i = lane; i < len; i += 32) d.rr_mem[dst + i] = arena[src + i];
        if (lane == 0) {
            int k = 0;
            while (k < HYPERIM_NSTRATA - 1 && local >= d.jm.job_base[k + 1]) ++k;
            d.rr_off[d.base_count + local] = dst;
            d.rr_stratum[d.base_count + local] = (uint8_t)k;
            d.rr_j[d.base_count + local] = d.jm.j_base[k] + (uint32_t)(local - d.jm.job_base[k]) * d.jm.j_step;
            if (local == d.jobs - 1) d.rr_off[d.base_count + d.jobs] = dst + len;
        }
    }
}

__global__ void k_gather_i64(const int64_t* __restrict__ src, const int64_t* __restrict__ idx, int n,
                             int64_t* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = src[idx[i]];
}

template <typename T>
hyperim_status grow_array(hyperim_graph* g, T** arr, size_t used, size_t* cap, size_t need) {
    if (need <= *cap) return HYPERIM_OK;
    size_t nc = *cap ? *cap : 1024;
    while (nc < need) nc *= 2;
    T* na = nullptr;
    hyperim_status st = dev_alloc(g, (void**)&na, sizeof(T) * nc);
    if (st != HYPERIM_OK) return st;
    if (used) HYP_CUDA(cudaMemcpyAsync(na, *arr, sizeof(T) * used, cudaMemcpyDeviceToDevice, g->stream));
    if (*arr) dev_free(g, *arr, sizeof(T) * *cap);
    *arr = na;
    *cap = nc;
    return HYPERIM_OK;
}

// The dynamic shared memory limit of a kernel is one value per function, not per launch: it is
// raised once to the most any launch can ask for (an on-chip visited bitmap of kVisSmemBits), so
// that launches from several host threads with different sizes never race on it.
// the most dynamic shared memory a block of this device may use
size_t smem_optin() {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (size_t)optin;
}

hyperim_status allow_rr_smem() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        const int most = (int)std::min<size_t>(sizeof(Shared) + kVisSmemBits / 8, smem_optin());
        err = cudaFuncSetAttribute(k_rr, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        if (err == cudaSuccess) err = cudaFuncSetAttribute(k_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(k_rr_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(WarpShared));
        if (err == cudaSuccess) {
            cudaFuncAttributes fa;
            err = cudaFuncGetAttributes(&fa, k_rr_batch);
            if (err == cudaSuccess) {
                const size_t room = smem_optin() > fa.sharedSizeBytes ? smem_optin() - fa.sharedSizeBytes : 0;
                const int batch_most = (int)std::min<size_t>(sizeof(Shared) + kVisSmemBits / 8, room);
                err = cudaFuncSetAttribute(k_rr_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, batch_most);
            }
        }
    });
    HYP_CUDA(err);
    return HYPERIM_OK;
}

// rounds of a bounded device wait (hyperim_graph_set_wait_limit; default 2^24)
int wait_rounds(const hyperim_graph* g) {
    const uint32_t w = g->wait_limit ? g->wait_limit : (1u << 24);
    return (int)std::min<uint32_t>(w, 0x7FFFFFFFu);
}

hyperim_status ensure_scratch(hyperim_graph* g, int blocks, bool vis_smem) {
    Scratch& S = g->scratch;
    const size_t list_cap = (size_t)g->n;
    const size_t vis_words = vis_smem ? 0 : ((size_t)g->n + 31) / 32;
    const size_t pick_cap = (size_t)std::max<int64_t>(g->max_deg, 1);  // picks of one pop
    const size_t big_cap = (size_t)std::max<int64_t>(g->max_tsum, 1);
    if (S.blocks >= blocks && S.list_cap >= list_cap && S.bitmap_words >= vis_words &&
        S.pick_cap >= pick_cap && S.big_cap >= big_cap)
        return HYPERIM_OK;
    if (S.list) dev_free(g, S.list, sizeof(int32_t) * S.list_cap * S.blocks);
    if (S.bitmap) dev_free(g, S.bitmap, sizeof(uint32_t) * S.bitmap_words * S.blocks);
    if (S.picks) dev_free(g, S.picks, sizeof(uint32_t) * S.pick_cap * S.blocks);
    if (S.big) dev_free(g, S.big, sizeof(uint32_t) * S.big_cap * S.blocks);
    S = Scratch{0, 0, 0, 0, 0, nullptr, nullptr, nullptr, nullptr, S.arena, S.arena_cap};
    hyperim_status st;
    if ((st = dev_alloc(g, (void**)&S.list, sizeof(int32_t) * list_cap * blocks))) return st;
    HYP_CUDA(cudaMemsetAsync(S.list, 0xFF, sizeof(int32_t) * list_cap * blocks, g->stream));  // empty slots
    if (vis_words) {
        if ((st = dev_alloc(g, (void**)&S.bitmap, sizeof(uint32_t) * vis_words * blocks))) return st;
        HYP_CUDA(cudaMemsetAsync(S.bitmap, 0, sizeof(uint32_t) * vis_words * blocks, g->stream));
    }
    if ((st = dev_alloc(g, (void**)&S.picks, sizeof(uint32_t) * pick_cap * blocks))) return st;
    if ((st = dev_alloc(g, (void**)&S.big, sizeof(uint32_t) * big_cap * blocks))) return st;
    S.blocks = blocks;
    S.list_cap = list_cap;
    S.bitmap_words = vis_words;
    S.pick_cap = pick_cap;
    S.big_cap = big_cap;
    return HYPERIM_OK;
}

// Output arena entries for a growth step: 1.25 x the expected members (each pool's mean set size
// so far, else the graph handle's last growth's). With no size history at all the sets may hold
// anything up to n members: the arena then takes min(jobs x n, 2^27) entries, so that a first
// growth rarely needs the repair launch (which builds again every set that did not fit).
uint64_t arena_want(const hyperim_graph* g, hyperim_pool* const* pools, int npools, const int64_t* pool_start,
                    int64_t n) {
    if (g->arena_entries_per_set > 0)
        return std::max<uint64_t>(1, (uint64_t)(pool_start[npools] - pool_start[0]) * (uint64_t)g->arena_entries_per_set);
    double want = 4096.0;
    bool unknown = false;
    for (int q = 0; q < npools; ++q) {
        const double jobs = (double)(pool_start[q + 1] - pool_start[q]);
        const double hint = pools[q]->mean_size_hint > 0 ? pools[q]->mean_size_hint : g->set_size_hint;
        if (hint > 0) want += jobs * hint * 1.25;
        else unknown = unknown || jobs > 0;
    }
    if (unknown) {
        const double jobs = (double)(pool_start[npools] - pool_start[0]);
        want = std::max(want, std::min(jobs * (double)std::max<int64_t>(n, 1), (double)(1ull << 27)));
    }
    return (uint64_t)want;
}

// after a growth: the handle's set-size hint, and an idle arena far larger than what the growth
// used is released (the next growth allocates what its hint asks for)
void after_growth(hyperim_graph* g, uint64_t used, int64_t njobs, int32_t** arena, uint64_t* cap) {
    if (njobs > 0) g->set_size_hint = std::max(1.0, (double)used / (double)njobs);
    if (*arena && *cap > (1ull << 24) && *cap > 4 * used + 4096) {
        dev_free(g, *arena, sizeof(int32_t) * *cap);
        *arena = nullptr;
        *cap = 0;
    }
}

// Job maps of a growth step: pool q's new sets are jobs [pool_start[q], pool_start[q + 1]),
// stratum by stratum; a shard (rank r of W) holds the sets j = r (mod W) of each stratum's
// allocation.
hyperim_status make_job_maps(hyperim_pool* const* pools, int npools, const uint64_t (*new_ns)[HYPERIM_NSTRATA],
                             RRJobMap* jm, int64_t* pool_start) {
    pool_start[0] = 0;
    for (int q = 0; q < npools; ++q) {
        hyperim_pool* p = pools[q];
        const uint64_t W = (uint64_t)std::max(p->shard_world, 1), R = (uint64_t)std::max(p->shard_rank, 0);
        jm[q].job_base[0] = 0;
        jm[q].j_step = (uint32_t)W;
        for (int s = 0; s < HYPERIM_NSTRATA; ++s) {
            const uint64_t old = p->n_s[s];
            if (new_ns[q][s] > 0xFFFFFFFFull)
                return set_error(HYPERIM_EOVERFLOW, "an RR index within a stratum would reach 2^32");
            const uint64_t j0 = old + (R + W - old % W) % W;  // first j >= old of this shard
            const uint64_t add = new_ns[q][s] > j0 ? (new_ns[q][s] - 1 - j0) / W + 1 : 0;
            jm[q].j_base[s] = (uint32_t)std::min<uint64_t>(j0, 0xFFFFFFFFull);
            jm[q].job_base[s + 1] = jm[q].job_base[s] + (int64_t)add;
        }
        pool_start[q + 1] = pool_start[q] + jm[q].job_base[HYPERIM_NSTRATA];
    }
    return HYPERIM_OK;
}

// the graph's arrays and scalars in P (everything a set's construction reads of the graph)
void fill_graph_params(RRParams& P, const hyperim_graph* g) {
    P.vinfo = g->vinfo;
    P.v_span = g->v_span;
    P.he_mem = g->he_mem;
    P.prof_off = g->prof_off;
    P.prof = g->prof;
    P.tab = g->cdf_tab;
    P.tsum = g->tsum;
    P.vs_off = g->vs_off;
    P.vs_list = g->vs_list;
    P.idx = g->idx;
    P.idx_tab = g->idx_tab;
    P.mat_sect = g->mat_sect;
    P.he_dir = g->he_dir;
    P.v_dir = g->v_dir;
    P.n = g->n;
    P.id_bits = g->id_bits;
    P.seed = g->seed;
}

// a pool's bookkeeping after its new sets were appended (allocation covered, counts, size hint)
void pool_appended(hyperim_pool* p, const uint64_t new_ns[HYPERIM_NSTRATA], int64_t new_count, int64_t new_total) {
    for (int i = 0; i < HYPERIM_NSTRATA; ++i)
        if (new_ns[i] > p->n_s[i]) p->n_s[i] = new_ns[i];
    p->count = new_count;
    p->total = new_total;
    p->mean_size_hint = p->count > 0 ? (double)p->total / (double)p->count : 0.0;
}

// and its work counters, kernel time (its share of the launch's) and launches
void pool_counted(hyperim_pool* p, const RRCounters& c, double seconds, uint64_t launches) {
    unsigned long long* dst = &p->counters.pops;
    const unsigned long long* src = &c.pops;
    for (int i = 0; i < kNStat; ++i) dst[i] += src[i];
    p->rr_kernel_seconds += seconds;
    p->rr_launches += launches;
}

// The launch's sets of pool p (jobs [0, nq) of d_pos / d_size, sizes in the arena) appended to its
// CSR arrays on g's stream (offsets by an exclusive scan of the sizes into d_boff, nq + 1
// entries), and the pool's bookkeeping: allocation, counts, counters, kernel time (its share).
hyperim_status compact_pool(hyperim_graph* g, hyperim_pool* p, const int32_t* arena, const int64_t* d_pos,
                            const int32_t* d_size, int64_t nq, const RRJobMap& jm,
                            const uint64_t new_ns[HYPERIM_NSTRATA], int64_t* d_boff, const RRCounters& c,
                            double seconds, uint64_t launches) {
    cudaStream_t s = g->stream;
    hyperim_status st;
    if (nq > 0) {
        if ((st = exclusive_scan_u32_to_i64(g, reinterpret_cast<const uint32_t*>(d_size), d_boff, nq))) return st;
        int64_t btotal = 0;
        HYP_CUDA(cudaMemcpyAsync(&btotal, d_boff + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HYP_CUDA(cudaStreamSynchronize(s));
        const size_t new_count = (size_t)(p->count + nq), new_total = (size_t)(p->total + btotal);
        if ((st = grow_array(g, &p->rr_off, p->count ? (size_t)p->count + 1 : 0, &p->cap_off, new_count + 1)))
            return st;
        if ((st = grow_array(g, &p->rr_stratum, (size_t)p->count, &p->cap_stratum, new_count))) return st;
        if ((st = grow_array(g, &p->rr_j, (size_t)p->count, &p->cap_j, new_count))) return st;
        if ((st = grow_array(g, &p->rr_mem, (size_t)p->total, &p->cap_total, new_total))) return st;
        const int grid = (int)std::min<int64_t>((nq * 32 + 255) / 256, (int64_t)g->sm_count * 32);
        { k_compact_rr<<<grid, 256, 0, s>>>(arena, d_pos, d_boff, nq, p->count, p->total, jm, p->rr_off,
                                            p->rr_mem, p->rr_stratum, p->rr_j); count_launch(); }
        HYP_CUDA(cudaGetLastError());
        pool_appended(p, new_ns, (int64_t)new_count, (int64_t)new_total);
    }
    pool_counted(p, c, seconds, launches);
    return HYPERIM_OK;
}

}  // namespace

hyperim_status sample_rr_multi(hyperim_graph* g, hyperim_pool* const* pools, int npools,
                               const uint64_t (*new_ns)[HYPERIM_NSTRATA]) {
    if (npools < 1 || npools > kMaxPools) return set_error(HYPERIM_EINVAL, "bad pool count");
    for (int q = 1; q < npools; ++q)
        if (pools[q]->root_mode != pools[0]->root_mode || pools[q]->strategy != pools[0]->strategy)
            return set_error(HYPERIM_ESTATE, "pools grown together must share root mode and strategy");
    RRJobMap jm[kMaxPools];
    int64_t pool_start[kMaxPools + 1];
    hyperim_status st;
    if ((st = make_job_maps(pools, npools, new_ns, jm, pool_start))) return st;
    const int64_t njobs = pool_start[npools];
    if (njobs == 0) return HYPERIM_OK;
    if (njobs >= (int64_t)0x7FFFFFFF) return set_error(HYPERIM_EOVERFLOW, "too many RR sets in one growth step");
    cudaStream_t s = g->stream;

    // the visited bitmap goes on chip while the block still fits on an SM
    if ((st = allow_rr_smem())) return st;
    bool vis_smem = (int64_t)g->n <= kVisSmemBits &&
                    sizeof(Shared) + sizeof(uint32_t) * (((size_t)g->n + 31) / 32) <= smem_optin();
    size_t smem = 0;
    int per_sm = 0;
    for (;;) {
        const size_t vis_bytes = vis_smem ? sizeof(uint32_t) * (((size_t)g->n + 31) / 32) : 0;
        smem = sizeof(Shared) + vis_bytes;
        HYP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rr, kThreads, smem));
        if (per_sm >= 1 || !vis_smem) break;
        vis_smem = false;
    }
    if (per_sm < 1) return set_error(HYPERIM_ECUDA, "RR kernel does not fit on an SM");
    int blocks = g->sm_count * per_sm;
    if ((int64_t)blocks > njobs) blocks = (int)njobs;
    if ((st = ensure_scratch(g, blocks, vis_smem))) return st;

    const uint64_t want = arena_want(g, pools, npools, pool_start, g->n);
    // the warp phase (one RR set per warp) runs first in the persistent schedule, unless the
    // graph's tuning turned it off; its grid
    const bool warp_phase = g->schedule != HYPERIM_SCHED_PLAIN && g->warp_set_limit > 0;
    int wblocks = 0;
    if (warp_phase) {
        int wper_sm = 0;
        HYP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&wper_sm, k_rr_warp, kPThreads, sizeof(WarpShared)));
        if (wper_sm < 1) return set_error(HYPERIM_ECUDA, "RR warp-phase kernel does not fit on an SM");
        wblocks = (int)std::min<int64_t>((int64_t)g->sm_count * wper_sm, (njobs + kPWarps - 1) / kPWarps);
    }
    // control words: two job counters (warp phase, block phase), the listed jobs, the arena fill
    struct Ctrl {
        int next_job[2];
        int esc_count;
        int pad;
        unsigned long long arena_used;
        unsigned long long set_cycles[3];  // sum, max, count over the sets the block kernel built
    };
    int64_t* d_pos = nullptr;
    int32_t* d_size = nullptr;
    int32_t* d_esc = nullptr;
    Ctrl* d_ctrl = nullptr;
    CallBuffers tmp(g);
    if ((st = tmp.alloc(&d_pos, sizeof(int64_t) * (size_t)njobs))) return st;
    if ((st = tmp.alloc(&d_size, sizeof(int32_t) * (size_t)njobs))) return st;
    if ((st = tmp.alloc(&d_esc, sizeof(int32_t) * (size_t)njobs))) return st;
    if ((st = tmp.alloc(&d_ctrl, sizeof(Ctrl)))) return st;
    unsigned long long* d_used = &d_ctrl->arena_used;
    RRParams P;
    std::memset(&P, 0, sizeof(P));
    fill_graph_params(P, g);
    P.root_mode = pools[0]->root_mode;
    P.strategy = pools[0]->strategy;
    P.npools = npools;
    for (int q = 0; q <= npools; ++q) P.pool_start[q] = pool_start[q];
    for (int q = 0; q < npools; ++q) {
        P.tags[q] = pools[q]->tag;
        P.jm[q] = jm[q];
    }
    P.list = g->scratch.list;
    P.list_cap = (int64_t)g->scratch.list_cap;
    P.gvis = g->scratch.bitmap;
    P.vis_smem = vis_smem ? 1 : 0;
    P.vis_words = vis_smem ? (int64_t)(((size_t)g->n + 31) / 32) : (int64_t)g->scratch.bitmap_words;
    P.picks = g->scratch.picks;
    P.pick_cap = (int64_t)g->scratch.pick_cap;
    P.big = g->scratch.big;
    P.big_cap = (int64_t)g->scratch.big_cap;
    P.out_pos = d_pos;
    P.out_size = d_size;
    P.next_job = d_ctrl->next_job;
    P.esc_count = &d_ctrl->esc_count;
    P.esc_list = d_esc;
    P.block_phase = 0;
    P.warp_limit = std::min(std::max(g->warp_set_limit, 1), kWQ);
    P.plain = g->schedule == HYPERIM_SCHED_PLAIN ? 1 : 0;
    P.plain_base = 0;
    P.arena_used = d_used;
    P.st = g->d_status;
    P.counters = g->d_counters;
    P.spin_limit = wait_rounds(g);
    P.set_cycles = d_ctrl->set_cycles;
    unsigned long long used = 0;
    unsigned long long cycles[3] = {0, 0, 0};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    struct Events {
        cudaEvent_t* a;
        cudaEvent_t* b;
        ~Events() {
            if (*a) cudaEventDestroy(*a);
            if (*b) cudaEventDestroy(*b);
        }
    } events{&ev0, &ev1};
    HYP_CUDA(cudaEventCreate(&ev0));
    HYP_CUDA(cudaEventCreate(&ev1));
    double seconds = 0.0;
    int launches = 0;
    if (g->scratch.arena_cap < want) {
        if (g->scratch.arena) dev_free(g, g->scratch.arena, sizeof(int32_t) * g->scratch.arena_cap);
        g->scratch.arena = nullptr;
        g->scratch.arena_cap = 0;
        if ((st = dev_alloc(g, (void**)&g->scratch.arena, sizeof(int32_t) * want))) return st;
        g->scratch.arena_cap = want;
    }
    P.arena = g->scratch.arena;
    P.arena_cap = g->scratch.arena_cap;
    P.rewrite = 0;
    HYP_CUDA(cudaMemsetAsync(d_ctrl, 0, sizeof(Ctrl), s));
    HYP_CUDA(cudaMemsetAsync(g->d_counters, 0, sizeof(RRCounters) * kMaxPools, s));
    HYP_CUDA(cudaEventRecord(ev0, s));
    if (P.plain) {
        // the comparison form: one launch per batch of `blocks` sets, one set per block
        for (int64_t base = 0; base < njobs; base += blocks) {
            P.plain_base = base;
            const int grid = (int)std::min<int64_t>(blocks, njobs - base);
            { k_rr<<<grid, kThreads, smem, s>>>(P); count_launch(); }
            HYP_CUDA(cudaGetLastError());
            ++launches;
        }
    } else if (warp_phase) {
        // warp phase over every job, then the block phase over the jobs it listed
        P.block_phase = 0;
        { k_rr_warp<<<wblocks, kPThreads, sizeof(WarpShared), s>>>(P); count_launch(); }
        HYP_CUDA(cudaGetLastError());
        P.block_phase = 1;
        { k_rr<<<blocks, kThreads, smem, s>>>(P); count_launch(); }
        P.block_phase = 0;
        ++launches;
    } else {
        { k_rr<<<blocks, kThreads, smem, s>>>(P); count_launch(); }
        ++launches;
    }
    HYP_CUDA(cudaGetLastError());
    HYP_CUDA(cudaEventRecord(ev1, s));
    HYP_CUDA(cudaMemcpyAsync(&used, d_used, sizeof(used), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaMemcpyAsync(cycles, d_ctrl->set_cycles, sizeof(cycles), cudaMemcpyDeviceToHost, s));
    auto failed = [&](hyperim_status code) {
        // a failed launch may leave queue slots filled: empty them for the next one
        cudaMemsetAsync(g->scratch.list, 0xFF, sizeof(int32_t) * g->scratch.list_cap * g->scratch.blocks, s);
        return code;
    };
    if ((st = check_device_status(g, "RR generation"))) return failed(st);
    float ms = 0.f;
    HYP_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
    seconds += 1e-3 * (double)ms;
    if (cycles[2] > 0 && !P.plain) {
        g->set_cycles_mean = (double)cycles[0] / (double)cycles[2];
        g->set_cycles_max = (double)cycles[1];
    }
    if (used > g->scratch.arena_cap) {
        // The arena (sized from the pools' mean set size so far) was too small: every set has its
        // slot reserved in [0, used), and the sets that fit are written. The arena grows (its
        // written part copied), and a repair launch builds again only the sets that did not fit
        // and writes them to their reserved slots.
        const uint64_t old_cap = g->scratch.arena_cap;
        const uint64_t new_cap = used + used / 8 + 4096;
        int32_t* na = nullptr;
        if ((st = dev_alloc(g, (void**)&na, sizeof(int32_t) * new_cap))) return st;
        HYP_CUDA(cudaMemcpyAsync(na, g->scratch.arena, sizeof(int32_t) * old_cap, cudaMemcpyDeviceToDevice, s));
        dev_free(g, g->scratch.arena, sizeof(int32_t) * old_cap);
        g->scratch.arena = na;
        g->scratch.arena_cap = new_cap;
        HYP_CUDA(cudaMemsetAsync(&d_ctrl->next_job[1], 0, 2 * sizeof(int), s));  // block-phase counter, list size
        { k_overflow_jobs<<<(int)std::min<int64_t>((njobs + 255) / 256, (int64_t)g->sm_count * 8), 256, 0, s>>>(
              d_pos, d_size, njobs, old_cap, d_esc, &d_ctrl->esc_count); count_launch(); }
        const int plain = P.plain;
        P.arena = na;
        P.arena_cap = new_cap;
        P.plain = 0;
        P.block_phase = 1;
        P.rewrite = 1;
        HYP_CUDA(cudaEventRecord(ev0, s));
        { k_rr<<<blocks, kThreads, smem, s>>>(P); count_launch(); }
        HYP_CUDA(cudaGetLastError());
        HYP_CUDA(cudaEventRecord(ev1, s));
        P.plain = plain;
        P.block_phase = 0;
        P.rewrite = 0;
        ++launches;
        if ((st = check_device_status(g, "RR generation (arena repair)"))) return failed(st);
        HYP_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
        seconds += 1e-3 * (double)ms;
    }
    RRCounters c[kMaxPools];
    HYP_CUDA(cudaMemcpyAsync(c, g->d_counters, sizeof(RRCounters) * kMaxPools, cudaMemcpyDeviceToHost, s));
    // compaction, pool by pool: CSR offsets by an exclusive scan of the sizes
    int64_t* d_boff = nullptr;
    if ((st = tmp.alloc(&d_boff, sizeof(int64_t) * ((size_t)njobs + 1)))) return st;
    for (int q = 0; q < npools; ++q) {
        const int64_t b0 = pool_start[q], nq = pool_start[q + 1] - b0;
        // the launch's time and count are shared by the pools it grew, in proportion to their jobs
        const double share = (double)nq / (double)njobs;
        if ((st = compact_pool(g, pools[q], g->scratch.arena, d_pos + b0, d_size + b0, nq, jm[q], new_ns[q], d_boff,
                               c[q], seconds * share, q == 0 ? (uint64_t)launches : 0)))
            return st;
    }
    after_growth(g, used, njobs, &g->scratch.arena, &g->scratch.arena_cap);
    return check_device_status(g, "RR compaction");
}

hyperim_status sample_rr_batch(hyperim_graph* g0, const RRGroup* groups, int ngroups, double* seconds_out) {
    if (seconds_out) *seconds_out = 0.0;
    if (ngroups < 1) return HYPERIM_OK;
    hyperim_status st;
    std::vector<RRJobMap> jm((size_t)ngroups * kMaxPools);
    std::vector<int64_t> pstart((size_t)ngroups * (kMaxPools + 1));
    std::vector<int64_t> gstart((size_t)ngroups + 1, 0);
    std::vector<cudaStream_t> streams{g0->stream};
    int64_t n_max = 1, deg_max = 1, tsum_max = 1;
    for (int q = 0; q < ngroups; ++q) {
        const RRGroup& G = groups[q];
        if (G.npools < 1 || G.npools > kMaxPools) return set_error(HYPERIM_EINVAL, "bad pool count");
        for (int i = 0; i < G.npools; ++i) {
            if (graph_root(G.pools[i]->g) != graph_root(G.g)) return set_error(HYPERIM_ESTATE, "pool of another graph");
            if (G.pools[i]->root_mode != G.pools[0]->root_mode || G.pools[i]->strategy != G.pools[0]->strategy)
                return set_error(HYPERIM_ESTATE, "pools grown together must share root mode and strategy");
        }
        if ((st = make_job_maps(G.pools, G.npools, G.new_ns, &jm[(size_t)q * kMaxPools],
                                &pstart[(size_t)q * (kMaxPools + 1)])))
            return st;
        gstart[q + 1] = gstart[q] + pstart[(size_t)q * (kMaxPools + 1) + G.npools];
        n_max = std::max<int64_t>(n_max, G.g->n);
        deg_max = std::max<int64_t>(deg_max, G.g->max_deg);
        tsum_max = std::max<int64_t>(tsum_max, G.g->max_tsum);
        if (std::find(streams.begin(), streams.end(), G.g->stream) == streams.end()) streams.push_back(G.g->stream);
    }
    const int64_t njobs = gstart[ngroups];
    if (njobs == 0) return HYPERIM_OK;
    if (njobs >= (int64_t)0x7FFFFFFF) return set_error(HYPERIM_EOVERFLOW, "too many RR sets in one growth step");
    cudaStream_t s = g0->stream;
    // the launch runs on g0's stream after the work already queued on every graph's stream, and
    // each graph's compaction runs on its own stream once the launch is done (host-synchronised)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> waits;
    struct Events {
        cudaEvent_t* a;
        cudaEvent_t* b;
        std::vector<cudaEvent_t>* w;
        ~Events() {
            if (*a) cudaEventDestroy(*a);
            if (*b) cudaEventDestroy(*b);
            for (cudaEvent_t e : *w) cudaEventDestroy(e);
        }
    } events{&ev0, &ev1, &waits};
    for (size_t i = 1; i < streams.size(); ++i) {
        cudaEvent_t e = nullptr;
        HYP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        waits.push_back(e);
        HYP_CUDA(cudaEventRecord(e, streams[i]));
        HYP_CUDA(cudaStreamWaitEvent(s, e, 0));
    }

    if ((st = allow_rr_smem())) return st;
    cudaFuncAttributes fa;
    HYP_CUDA(cudaFuncGetAttributes(&fa, k_rr_batch));
    const size_t words_max = ((size_t)n_max + 31) / 32;
    bool vis_smem = n_max <= kVisSmemBits && sizeof(Shared) + sizeof(uint32_t) * words_max + fa.sharedSizeBytes <= smem_optin();
    size_t smem = 0;
    int per_sm = 0;
    for (;;) {
        smem = sizeof(Shared) + (vis_smem ? sizeof(uint32_t) * words_max : 0);
        HYP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rr_batch, kThreads, smem));
        if (per_sm >= 1 || !vis_smem) break;
        vis_smem = false;
    }
    if (per_sm < 1) return set_error(HYPERIM_ECUDA, "batched RR kernel does not fit on an SM");
    int blocks = g0->sm_count * per_sm;
    if ((int64_t)blocks > njobs) blocks = (int)njobs;

    // scratch of this call, sized for the largest graph: queue (empty slots), visited bitmap,
    // picks and bucketed neighbourhoods per block
    CallBuffers tmp(g0);
    int32_t* list = nullptr;
    uint32_t *gvis = nullptr, *picks = nullptr, *big = nullptr;
    if ((st = tmp.alloc(&list, sizeof(int32_t) * (size_t)n_max * blocks))) return st;
    HYP_CUDA(cudaMemsetAsync(list, 0xFF, sizeof(int32_t) * (size_t)n_max * blocks, s));
    if (!vis_smem) {
        if ((st = tmp.alloc(&gvis, sizeof(uint32_t) * words_max * blocks))) return st;
        HYP_CUDA(cudaMemsetAsync(gvis, 0, sizeof(uint32_t) * words_max * blocks, s));
    }
    if ((st = tmp.alloc(&picks, sizeof(uint32_t) * (size_t)deg_max * blocks))) return st;
    if ((st = tmp.alloc(&big, sizeof(uint32_t) * (size_t)tsum_max * blocks))) return st;
    struct Ctrl {
        int next_job;
        int rerun_count;  // sets listed for an arena repair
        unsigned long long arena_used;
    };
    int64_t* d_pos = nullptr;
    int32_t* d_size = nullptr;
    Ctrl* d_ctrl = nullptr;
    RRParams* d_groups = nullptr;
    int64_t* d_gstart = nullptr;
    RRCounters* d_counters = nullptr;
    if ((st = tmp.alloc(&d_pos, sizeof(int64_t) * (size_t)njobs))) return st;
    if ((st = tmp.alloc(&d_size, sizeof(int32_t) * (size_t)njobs))) return st;
    if ((st = tmp.alloc(&d_ctrl, sizeof(Ctrl)))) return st;
    if ((st = tmp.alloc(&d_groups, sizeof(RRParams) * (size_t)ngroups))) return st;
    if ((st = tmp.alloc(&d_gstart, sizeof(int64_t) * ((size_t)ngroups + 1)))) return st;
    if ((st = tmp.alloc(&d_counters, sizeof(RRCounters) * (size_t)ngroups * kMaxPools))) return st;

    uint64_t want = 0;
    for (int q = 0; q < ngroups; ++q)
        want += arena_want(groups[q].g, groups[q].pools, groups[q].npools, &pstart[(size_t)q * (kMaxPools + 1)],
                           n_max);
    // the arena: reallocated when a launch overflows it
    struct Arena {
        hyperim_graph* g;
        int32_t* p = nullptr;
        uint64_t cap = 0;
        ~Arena() {
            if (p) dev_free(g, p, sizeof(int32_t) * cap);
        }
    } arena{g0};

    std::vector<RRParams> hp((size_t)ngroups);
    for (int q = 0; q < ngroups; ++q) {
        const RRGroup& G = groups[q];
        RRParams& P = hp[q];
        std::memset(&P, 0, sizeof(P));
        fill_graph_params(P, G.g);
        P.root_mode = G.pools[0]->root_mode;
        P.strategy = G.pools[0]->strategy;
        P.npools = G.npools;
        for (int i = 0; i <= G.npools; ++i) P.pool_start[i] = pstart[(size_t)q * (kMaxPools + 1) + i];
        for (int i = 0; i < G.npools; ++i) {
            P.tags[i] = G.pools[i]->tag;
            P.jm[i] = jm[(size_t)q * kMaxPools + i];
        }
        P.list = list;
        P.list_cap = n_max;
        P.gvis = gvis;
        P.vis_smem = vis_smem ? 1 : 0;
        P.vis_words = (int64_t)words_max;
        P.picks = picks;
        P.pick_cap = deg_max;
        P.big = big;
        P.big_cap = tsum_max;
        P.out_pos = d_pos + gstart[q];
        P.out_size = d_size + gstart[q];
        P.arena_used = &d_ctrl->arena_used;
        P.st = g0->d_status;
        P.counters = d_counters + (size_t)q * kMaxPools;
        P.spin_limit = wait_rounds(g0);
    }
    RRBatchParams B;
    B.groups = d_groups;
    B.group_start = d_gstart;
    B.ngroups = ngroups;
    B.next_job = &d_ctrl->next_job;
    B.list = list;
    B.list_cap = n_max;
    B.gvis = gvis;
    B.vis_smem = vis_smem ? 1 : 0;
    B.vis_words = (int64_t)words_max;
    B.picks = picks;
    B.pick_cap = deg_max;
    B.big = big;
    B.big_cap = tsum_max;
    HYP_CUDA(cudaMemcpyAsync(d_gstart, gstart.data(), sizeof(int64_t) * ((size_t)ngroups + 1), cudaMemcpyHostToDevice, s));
    HYP_CUDA(cudaEventCreate(&ev0));
    HYP_CUDA(cudaEventCreate(&ev1));
    unsigned long long used = 0;
    double seconds = 0.0;
    if ((st = dev_alloc(g0, (void**)&arena.p, sizeof(int32_t) * want))) return st;
    arena.cap = want;
    for (RRParams& P : hp) {
        P.arena = arena.p;
        P.arena_cap = arena.cap;
    }
    B.rerun = nullptr;
    B.rerun_count = nullptr;
    HYP_CUDA(cudaMemcpyAsync(d_groups, hp.data(), sizeof(RRParams) * hp.size(), cudaMemcpyHostToDevice, s));
    HYP_CUDA(cudaMemsetAsync(d_ctrl, 0, sizeof(Ctrl), s));
    HYP_CUDA(cudaMemsetAsync(d_counters, 0, sizeof(RRCounters) * (size_t)ngroups * kMaxPools, s));
    HYP_CUDA(cudaEventRecord(ev0, s));
    { k_rr_batch<<<blocks, kThreads, smem, s>>>(B); count_launch(); }
    HYP_CUDA(cudaGetLastError());
    HYP_CUDA(cudaEventRecord(ev1, s));
    HYP_CUDA(cudaMemcpyAsync(&used, &d_ctrl->arena_used, sizeof(used), cudaMemcpyDeviceToHost, s));
    if ((st = check_device_status(g0, "RR generation (batch)"))) return st;  // synchronises s
    float ms = 0.f;
    HYP_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
    seconds += 1e-3 * (double)ms;
    if (used > arena.cap) {
        // as in sample_rr_multi: a larger arena (written part copied) and a repair launch over the
        // sets that did not fit, written to the slots the first launch reserved
        const uint64_t old_cap = arena.cap;
        const uint64_t new_cap = used + used / 8 + 4096;
        int32_t* na = nullptr;
        if ((st = dev_alloc(g0, (void**)&na, sizeof(int32_t) * new_cap))) return st;
        HYP_CUDA(cudaMemcpyAsync(na, arena.p, sizeof(int32_t) * old_cap, cudaMemcpyDeviceToDevice, s));
        dev_free(g0, arena.p, sizeof(int32_t) * old_cap);
        arena.p = na;
        arena.cap = new_cap;
        int32_t* d_list = nullptr;
        if ((st = tmp.alloc(&d_list, sizeof(int32_t) * (size_t)njobs))) return st;
        HYP_CUDA(cudaMemsetAsync(d_ctrl, 0, sizeof(int) * 2, s));  // job counter, list size
        { k_overflow_jobs<<<(int)std::min<int64_t>((njobs + 255) / 256, (int64_t)g0->sm_count * 8), 256, 0, s>>>(
              d_pos, d_size, njobs, old_cap, d_list, &d_ctrl->rerun_count); count_launch(); }
        for (RRParams& P : hp) {
            P.arena = arena.p;
            P.arena_cap = arena.cap;
            P.rewrite = 1;
        }
        HYP_CUDA(cudaMemcpyAsync(d_groups, hp.data(), sizeof(RRParams) * hp.size(), cudaMemcpyHostToDevice, s));
        B.rerun = d_list;
        B.rerun_count = &d_ctrl->rerun_count;
        HYP_CUDA(cudaEventRecord(ev0, s));
        { k_rr_batch<<<blocks, kThreads, smem, s>>>(B); count_launch(); }
        HYP_CUDA(cudaGetLastError());
        HYP_CUDA(cudaEventRecord(ev1, s));
        if ((st = check_device_status(g0, "RR generation (batch, arena repair)"))) return st;
        HYP_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
        seconds += 1e-3 * (double)ms;
    }
    if (seconds_out) *seconds_out = seconds;
    std::vector<RRCounters> c((size_t)ngroups * kMaxPools);
    HYP_CUDA(cudaMemcpyAsync(c.data(), d_counters, sizeof(RRCounters) * c.size(), cudaMemcpyDeviceToHost, s));
    // Compaction of every pool in one kernel on s: one scan of all the sizes, each pool's new total
    // read off the scan at its job range's ends, the pools' arrays grown (on their graphs' streams,
    // then joined), and one copy kernel for all of them.
    HYP_CUDA(cudaStreamSynchronize(s));
    int64_t* d_boff = nullptr;
    if ((st = tmp.alloc(&d_boff, sizeof(int64_t) * ((size_t)njobs + 1)))) return st;
    if ((st = exclusive_scan_u32_to_i64(g0, reinterpret_cast<const uint32_t*>(d_size), d_boff, njobs))) return st;
    struct Slot {
        hyperim_pool* p;
        hyperim_graph* g;
        const uint64_t* new_ns;
        const RRJobMap* jm;
        int64_t b0, nq;
        const RRCounters* c;
    };
    std::vector<Slot> slots;
    std::vector<int64_t> marks;  // job range ends of every pool: boff[b0], boff[b0 + nq]
    for (int q = 0; q < ngroups; ++q) {
        const RRGroup& G = groups[q];
        const int64_t* ps = &pstart[(size_t)q * (kMaxPools + 1)];
        for (int i = 0; i < G.npools; ++i) {
            const int64_t b0 = gstart[q] + ps[i], nq = ps[i + 1] - ps[i];
            slots.push_back(Slot{G.pools[i], G.g, G.new_ns[i], &jm[(size_t)q * kMaxPools + i], b0, nq,
                                 &c[(size_t)q * kMaxPools + i]});
            marks.push_back(b0);
            marks.push_back(b0 + nq);
        }
    }
    int64_t *d_marks = nullptr, *d_vals = nullptr;
    if ((st = tmp.alloc(&d_marks, sizeof(int64_t) * marks.size()))) return st;
    if ((st = tmp.alloc(&d_vals, sizeof(int64_t) * marks.size()))) return st;
    std::vector<int64_t> vals(marks.size());
    HYP_CUDA(cudaMemcpyAsync(d_marks, marks.data(), sizeof(int64_t) * marks.size(), cudaMemcpyHostToDevice, s));
    { k_gather_i64<<<(int)std::min<size_t>((marks.size() + 255) / 256, 1024), 256, 0, s>>>(d_boff, d_marks,
                                                                                       (int)marks.size(), d_vals); count_launch(); }
    HYP_CUDA(cudaMemcpyAsync(vals.data(), d_vals, sizeof(int64_t) * vals.size(), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    std::vector<CompactDesc> desc;
    for (size_t x = 0; x < slots.size(); ++x) {
        const Slot& sl = slots[x];
        hyperim_pool* p = sl.p;
        if (sl.nq == 0) continue;
        const int64_t btotal = vals[2 * x + 1] - vals[2 * x];
        const size_t new_count = (size_t)(p->count + sl.nq), new_total = (size_t)(p->total + btotal);
        if ((st = grow_array(sl.g, &p->rr_off, p->count ? (size_t)p->count + 1 : 0, &p->cap_off, new_count + 1)))
            return st;
        if ((st = grow_array(sl.g, &p->rr_stratum, (size_t)p->count, &p->cap_stratum, new_count))) return st;
        if ((st = grow_array(sl.g, &p->rr_j, (size_t)p->count, &p->cap_j, new_count))) return st;
        if ((st = grow_array(sl.g, &p->rr_mem, (size_t)p->total, &p->cap_total, new_total))) return st;
        desc.push_back(CompactDesc{sl.b0, sl.nq, vals[2 * x], p->count, p->total, p->rr_off, p->rr_mem,
                                   p->rr_stratum, p->rr_j, *sl.jm});
    }
    for (cudaStream_t x : streams) HYP_CUDA(cudaStreamSynchronize(x));  // the grown arrays are ready
    if (!desc.empty()) {
        CompactDesc* d_desc = nullptr;
        if ((st = tmp.alloc(&d_desc, sizeof(CompactDesc) * desc.size()))) return st;
        HYP_CUDA(cudaMemcpyAsync(d_desc, desc.data(), sizeof(CompactDesc) * desc.size(), cudaMemcpyHostToDevice, s));
        const int grid = (int)std::min<int64_t>((njobs * 32 + 255) / 256, (int64_t)g0->sm_count * 32);
        { k_compact_batch<<<grid, 256, 0, s>>>(arena.p, d_pos, d_boff, njobs, d_desc, (int)desc.size()); count_launch(); }
        HYP_CUDA(cudaGetLastError());
        HYP_CUDA(cudaStreamSynchronize(s));
    }
    for (size_t x = 0; x < slots.size(); ++x) {
        const Slot& sl = slots[x];
        if (sl.nq > 0) pool_appended(sl.p, sl.new_ns, sl.p->count + sl.nq, sl.p->total + (vals[2 * x + 1] - vals[2 * x]));
        pool_counted(sl.p, *sl.c, seconds * (double)sl.nq / (double)njobs, 1);
    }
    return check_device_status(g0, "RR compaction (batch)");
}

hyperim_status sample_rr(hyperim_graph* g, hyperim_pool* p, const uint64_t new_ns[HYPERIM_NSTRATA]) {
    hyperim_pool* pools[1] = {p};
    const uint64_t (*ns)[HYPERIM_NSTRATA] = reinterpret_cast<const uint64_t (*)[HYPERIM_NSTRATA]>(new_ns);
    return sample_rr_multi(g, pools, 1, ns);
}


hyperim_status forward_spread(hyperim_graph* g, const int32_t* seeds_host, int32_t k, uint64_t nsims,
                              uint64_t seed, uint32_t* counts_host) {
    if (nsims == 0) return HYPERIM_OK;
    cudaStream_t s = g->stream;
    hyperim_status st;
    if ((st = allow_rr_smem())) return st;
    bool vis_smem = (int64_t)g->n <= kVisSmemBits &&
                    sizeof(Shared) + sizeof(uint32_t) * (((size_t)g->n + 31) / 32) <= smem_optin();
    size_t smem = 0;
    int per_sm = 0;
    for (;;) {
        const size_t vis_bytes = vis_smem ? sizeof(uint32_t) * (((size_t)g->n + 31) / 32) : 0;
        smem = sizeof(Shared) + vis_bytes;
        HYP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_forward, kThreads, smem));
        if (per_sm >= 1 || !vis_smem) break;
        vis_smem = false;
    }
    if (per_sm < 1) return set_error(HYPERIM_ECUDA, "forward kernel does not fit on an SM");
    int blocks = g->sm_count * per_sm;
    if ((uint64_t)blocks > nsims) blocks = (int)nsims;
    if ((st = ensure_scratch(g, blocks, vis_smem))) return st;
    int32_t* d_seeds = nullptr;
    uint32_t* d_counts = nullptr;
    unsigned long long* d_next = nullptr;
    const size_t kk = (size_t)(k > 0 ? k : 1);
    CallBuffers tmp(g);
    if ((st = tmp.alloc(&d_seeds, sizeof(int32_t) * kk))) return st;
    if ((st = tmp.alloc(&d_counts, sizeof(uint32_t) * (size_t)nsims))) return st;
    if ((st = tmp.alloc(&d_next, sizeof(unsigned long long)))) return st;
    if (k > 0) HYP_CUDA(cudaMemcpyAsync(d_seeds, seeds_host, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, s));
    HYP_CUDA(cudaMemsetAsync(d_next, 0, sizeof(unsigned long long), s));
    FwdParams F;
    std::memset(&F, 0, sizeof(F));
    RRParams& P = F.P;
    P.vinfo = g->vinfo;
    P.v_span = g->v_span;
    P.he_mem = g->he_mem;
    P.prof_off = g->prof_off;
    P.prof = g->prof;
    P.tsum = g->tsum;
    P.he_dir = g->he_dir;
    P.v_dir = g->v_dir;
    P.n = g->n;
    P.id_bits = g->id_bits;
    P.list = g->scratch.list;
    P.list_cap = (int64_t)g->scratch.list_cap;
    P.gvis = g->scratch.bitmap;
    P.vis_smem = vis_smem ? 1 : 0;
    P.vis_words = vis_smem ? (int64_t)(((size_t)g->n + 31) / 32) : (int64_t)g->scratch.bitmap_words;
    P.next_job = reinterpret_cast<int*>(d_next);
    P.st = g->d_status;
    P.spin_limit = wait_rounds(g);
    F.seeds = d_seeds;
    F.k = k;
    F.nsims = nsims;
    F.key0 = (uint32_t)seed;
    F.key1 = (uint32_t)(seed >> 32);
    F.counts = d_counts;
    { k_forward<<<blocks, kThreads, smem, s>>>(F); count_launch(); }
    HYP_CUDA(cudaGetLastError());
    if ((st = check_device_status(g, "forward spread"))) {
        cudaMemsetAsync(g->scratch.list, 0xFF, sizeof(int32_t) * g->scratch.list_cap * g->scratch.blocks, s);
        return st;
    }
    HYP_CUDA(cudaMemcpyAsync(counts_host, d_counts, sizeof(uint32_t) * (size_t)nsims, cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    return HYPERIM_OK;
}

}  // namespace hyperim
