// Greedy max coverage over an RR pool (Algorithm 1; marginal coverage of Eq. 2) on the device.
//
// Scores are integers: an RR set of stratum s weighs W_s = floor(|V_s| 2^32 / n_s) (1 with plain
// roots), so sums do not depend on the order of the atomic updates. Each round: argmax over the
// vertices not picked yet (ties to the lowest id), then the RR sets containing the winner that
// are not covered yet are retired: marked covered, counted in Lambda_s, and their weight is
// subtracted from the score of every member. The k rounds run back to back on the stream; the
// winner of a round is read on the device by the next launch.
#include <algorithm>
#include <cstddef>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace hyperim {
namespace {

constexpr int kArgThreads = 256;

struct Weights {
    unsigned long long w[HYPERIM_NSTRATA];
};

// A prefix view of a pool: only the RR sets (stratum s, index j) with j < lim[s] take part (the
// sets a pool grown to a smaller theta would hold). on = 0: every set of the pool.
struct Limits {
    uint32_t lim[HYPERIM_NSTRATA];
    int on;
    __device__ __forceinline__ bool skip(const uint8_t* rr_stratum, const uint32_t* rr_j, int64_t r) const {
        return on && rr_j[r] >= lim[rr_stratum[r]];
    }
};

// occurrences of each vertex over the RR sets of a prefix view; one warp per RR set
__global__ void k_count_occ_view(const int64_t* __restrict__ rr_off, const int32_t* __restrict__ mem,
                                 const uint8_t* __restrict__ rr_stratum, const uint32_t* __restrict__ rr_j,
                                 int64_t N, Limits L, uint32_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < N; r += nwarps) {
        if (L.skip(rr_stratum, rr_j, r)) continue;
        for (int64_t x = rr_off[r] + lane; x < rr_off[r + 1]; x += 32) atomicAdd(&cnt[mem[x]], 1u);
    }
}

__global__ void k_count_occ(const int32_t* __restrict__ mem, int64_t total, uint32_t* __restrict__ cnt) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[mem[x]], 1u);
}

// inverted index (vertex -> RR ids) and initial weighted scores; one warp per RR set
__global__ void k_scatter_inv(const int64_t* __restrict__ rr_off, const int32_t* __restrict__ mem,
                              const uint8_t* __restrict__ rr_stratum, const uint32_t* __restrict__ rr_j,
                              int64_t N, Limits L, const int64_t* __restrict__ inv_off,
                              uint32_t* __restrict__ cur, uint32_t* __restrict__ inv,
                              unsigned long long* __restrict__ score, Weights W) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < N; r += nwarps) {
        if (L.skip(rr_stratum, rr_j, r)) continue;
        const int64_t b = rr_off[r], e = rr_off[r + 1];
        const unsigned long long w = W.w[rr_stratum[r]];
        for (int64_t x = b + lane; x < e; x += 32) {
            const int32_t v = mem[x];
            const uint32_t pos = atomicAdd(&cur[v], 1u);
            inv[inv_off[v] + pos] = (uint32_t)r;
            atomicAdd(&score[v], w);
        }
    }
}

__device__ __forceinline__ bool better(unsigned long long s1, uint32_t i1, unsigned long long s2,
                                       uint32_t i2) {
    return s1 > s2 || (s1 == s2 && i1 < i2);
}

// The best (score, id) among the unpicked vertices of [0, n) visited by one thread (first index
// t, stride T): four consecutive vertices per step, their flags and scores loaded together
// without depending on one another (vectorised: score and picked are 16- and 4-byte aligned).
// `load` reads a score (plain, or through L2 where other threads of the block change scores by
// atomics).
template <bool kL2Scores = false>
__device__ __forceinline__ void scan_unpicked(const unsigned long long* __restrict__ score,
                                              const uint8_t* __restrict__ picked, int64_t n, int64_t t, int64_t T,
                                              unsigned long long& bs, uint32_t& bi) {
    const int64_t n4 = n >> 2;
    for (int64_t q = t; q < n4; q += T) {
        const uchar4 pk = reinterpret_cast<const uchar4*>(picked)[q];
        ulonglong2 a, b;
        if (kL2Scores) {
            a = __ldcg(reinterpret_cast<const ulonglong2*>(score) + 2 * q);
            b = __ldcg(reinterpret_cast<const ulonglong2*>(score) + 2 * q + 1);
        } else {
            a = reinterpret_cast<const ulonglong2*>(score)[2 * q];
            b = reinterpret_cast<const ulonglong2*>(score)[2 * q + 1];
        }
        const uint32_t v = (uint32_t)(4 * q);
        if (!pk.x && better(a.x, v, bs, bi)) { bs = a.x; bi = v; }
        if (!pk.y && better(a.y, v + 1, bs, bi)) { bs = a.y; bi = v + 1; }
        if (!pk.z && better(b.x, v + 2, bs, bi)) { bs = b.x; bi = v + 2; }
        if (!pk.w && better(b.y, v + 3, bs, bi)) { bs = b.y; bi = v + 3; }
    }
    for (int64_t v = 4 * n4 + t; v < n; v += T) {
        if (picked[v]) continue;
        const unsigned long long sc = kL2Scores ? __ldcg(score + v) : score[v];
        if (better(sc, (uint32_t)v, bs, bi)) { bs = sc; bi = (uint32_t)v; }
    }
}

// argmax of score over unpicked vertices, lowest id on ties; the last block to finish reduces
// the per-block winners, records the seed and marks it picked.
// Eq. upper_2 state (see the top-k kernels below)
struct TopK {
    unsigned long long prefix;
    unsigned int kleft, all;  // all: fewer unpicked vertices than k, so all of them count
    unsigned long long cover;
    unsigned long long best_lo, best_hi;
    unsigned int ticket;
    unsigned int first_pass;  // radix passes before it: every unpicked score's digit is 0 there
};

__global__ void __launch_bounds__(kArgThreads)
k_argmax(const unsigned long long* __restrict__ score, uint8_t* __restrict__ picked, int32_t n,
         unsigned long long* __restrict__ bscore, uint32_t* __restrict__ bid,
         unsigned int* __restrict__ ticket, int32_t* __restrict__ best, int32_t* __restrict__ seeds,
         int round, TopK* __restrict__ tk) {
    __shared__ unsigned long long ss[kArgThreads / 32];
    __shared__ uint32_t si[kArgThreads / 32];
    __shared__ bool last;
    unsigned long long bs = 0;
    uint32_t bi = 0xFFFFFFFFu;
    scan_unpicked(score, picked, n, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                  (int64_t)gridDim.x * blockDim.x, bs, bi);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long os = __shfl_xor_sync(0xFFFFFFFFu, bs, o);
        const uint32_t oi = __shfl_xor_sync(0xFFFFFFFFu, bi, o);
        if (better(os, oi, bs, bi)) { bs = os; bi = oi; }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { ss[wid] = bs; si[wid] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kArgThreads / 32; ++w)
            if (better(ss[w], si[w], bs, bi)) { bs = ss[w]; bi = si[w]; }
        bscore[blockIdx.x] = bs;
        bid[blockIdx.x] = bi;
        __threadfence();
        const unsigned int t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    bs = 0;
    bi = 0xFFFFFFFFu;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const unsigned long long s = ((volatile unsigned long long*)bscore)[b];
        const uint32_t i = ((volatile uint32_t*)bid)[b];
        if (better(s, i, bs, bi)) { bs = s; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long os = __shfl_xor_sync(0xFFFFFFFFu, bs, o);
        const uint32_t oi = __shfl_xor_sync(0xFFFFFFFFu, bi, o);
        if (better(os, oi, bs, bi)) { bs = os; bi = oi; }
    }
    if (lane == 0) { ss[wid] = bs; si[wid] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kArgThreads / 32; ++w)
            if (better(ss[w], si[w], bs, bi)) { bs = ss[w]; bi = si[w]; }
        *best = (int32_t)bi;
        seeds[round] = (int32_t)bi;
        picked[bi] = 1;
        // the winner's marginal weight, before its sets are retired; no unpicked score exceeds
        // it, now or later (scores only decrease), so the radix passes above its leading digit
        // can be skipped from here on
        tk->cover += bs;
        const int lead = bs ? (63 - __clzll((long long)bs)) : 0;
        tk->first_pass = (unsigned int)((56 - (lead & ~7)) / 8);
        *ticket = 0;
    }
}

// ---- Eq. upper_2 (p_max = 1): the k largest scores among the vertices not picked yet ---------
// A radix select over 8-bit digits, most significant first, finds the k-th largest score T
// (prefix) and how many of its copies belong to the top k (kleft); the top-k sum is then the sum
// of the scores above T plus kleft T. Every round's bound, cover + top-k sum, enters a running
// minimum; all of it stays on the device between the greedy's launches. 128-bit sums are kept
// as (lo, hi) pairs of 64-bit words.

__device__ __forceinline__ void add128(unsigned long long& lo, unsigned long long& hi, unsigned long long a_lo,
                                       unsigned long long a_hi) {
    const unsigned long long l = lo + a_lo;
    hi += a_hi + (l < lo ? 1ull : 0ull);
    lo = l;
}

__global__ void k_topk_hist(const unsigned long long* __restrict__ score, const uint8_t* __restrict__ picked,
                            int32_t n, const TopK* __restrict__ st, int pass, unsigned int* __restrict__ hist) {
    __shared__ unsigned int h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    // passes above the top bound's leading digit would find every candidate in digit 0: skipped
    if (!st->all && pass >= (int)st->first_pass) {
        const int sh = 56 - 8 * pass;
        const unsigned long long prefix = st->prefix;
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t v0 = blockIdx.x * (int64_t)blockDim.x; v0 < n; v0 += stride) {
            const int64_t v = v0 + threadIdx.x;
            int d = -1;
            if (v < n && !picked[v]) {
                const unsigned long long x = score[v];
                if (pass == 0 || (x >> (sh + 8)) == prefix) d = (int)((x >> sh) & 255u);
            }
            // one shared atomic per distinct digit of the warp
            const unsigned int same = __match_any_sync(0xFFFFFFFFu, d);
            if (d >= 0 && (threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&h[d], (unsigned int)__popc(same));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// one thread: the digit of the k-th largest among the candidates; clears the histogram
__global__ void k_topk_select(TopK* __restrict__ st, unsigned int* __restrict__ hist, int pass) {
    if (!st->all && pass >= (int)st->first_pass) {
        unsigned int cum = 0;
        int d = 255;
        for (; d >= 0; --d) {
            if (cum + hist[d] >= st->kleft) break;
            cum += hist[d];
        }
        if (d < 0) {  // fewer candidates than k (only on the first pass): take every unpicked vertex
            st->all = 1;
            st->prefix = 0;
            st->kleft = 0;
        } else {
            st->prefix = (st->prefix << 8) | (unsigned long long)d;
            st->kleft -= cum;
        }
    }
    for (int i = 0; i < 256; ++i) hist[i] = 0;
}

// sum of the scores above T = prefix over the unpicked vertices (grid reduction, last block
// finishes): K = sum + kleft T; bound = cover + K; running minimum; state reset for next round
__global__ void __launch_bounds__(kArgThreads)
k_topk_sum(const unsigned long long* __restrict__ score, const uint8_t* __restrict__ picked, int32_t n,
           TopK* __restrict__ st, unsigned long long* __restrict__ part, unsigned int k) {
    __shared__ unsigned long long slo[kArgThreads / 32], shi[kArgThreads / 32];
    __shared__ bool last;
    const unsigned long long T = st->prefix;
    unsigned long long lo = 0, hi = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (picked[v]) continue;
        const unsigned long long x = score[v];
        if (x > T) add128(lo, hi, x, 0ull);
    }
    for (int o = 16; o > 0; o >>= 1)
        add128(lo, hi, __shfl_xor_sync(0xFFFFFFFFu, lo, o), __shfl_xor_sync(0xFFFFFFFFu, hi, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { slo[wid] = lo; shi[wid] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kArgThreads / 32; ++w) add128(lo, hi, slo[w], shi[w]);
        part[2 * blockIdx.x] = lo;
        part[2 * blockIdx.x + 1] = hi;
        __threadfence();
        last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    lo = 0;
    hi = 0;
    for (unsigned int b = 0; b < gridDim.x; ++b)
        add128(lo, hi, ((volatile unsigned long long*)part)[2 * b], ((volatile unsigned long long*)part)[2 * b + 1]);
    const unsigned long long kl = st->kleft;
    add128(lo, hi, kl * T, __umul64hi(kl, T));
    add128(lo, hi, st->cover, 0ull);
    if (hi < st->best_hi || (hi == st->best_hi && lo < st->best_lo)) {
        st->best_lo = lo;
        st->best_hi = hi;
    }
    st->prefix = 0;
    st->kleft = k;
    st->all = 0;
    st->ticket = 0;
}

// retire the uncovered RR sets containing the round's winner; one warp per inverted entry
__global__ void k_retire(const int32_t* __restrict__ best, const int64_t* __restrict__ inv_off,
                         const uint32_t* __restrict__ inv, const int64_t* __restrict__ rr_off,
                         const int32_t* __restrict__ mem, const uint8_t* __restrict__ rr_stratum,
                         uint32_t* __restrict__ covered, unsigned long long* __restrict__ score,
                         unsigned long long* __restrict__ lam, Weights W) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t v = *best;
    const int64_t b = inv_off[v], e = inv_off[v + 1];
    for (int64_t t = b + warp; t < e; t += nwarps) {
        const uint32_t r = inv[t];
        uint32_t old = 0;
        if (lane == 0) old = atomicExch(&covered[r], 1u);
        old = __shfl_sync(0xFFFFFFFFu, old, 0);
        if (old) continue;
        const int s = rr_stratum[r];
        const unsigned long long neg = 0ull - W.w[s];
        if (lane == 0) atomicAdd(&lam[s], 1ull);
        for (int64_t x = rr_off[r] + lane; x < rr_off[r + 1]; x += 32) atomicAdd(&score[mem[x]], neg);
    }
}

// coverage of a seed set: RR sets with at least one member in S, per stratum; one warp per set
__global__ void k_coverage(const int64_t* __restrict__ rr_off, const int32_t* __restrict__ mem,
                           const uint8_t* __restrict__ rr_stratum, const uint32_t* __restrict__ rr_j,
                           int64_t N, Limits L, const uint8_t* __restrict__ in_s,
                           unsigned long long* __restrict__ lam) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < N; r += nwarps) {
        if (L.skip(rr_stratum, rr_j, r)) continue;
        const int64_t b = rr_off[r], e = rr_off[r + 1];
        bool hit = false;
        for (int64_t base = b; base < e; base += 32) {
            const int64_t x = base + lane;
            if (__any_sync(0xFFFFFFFFu, x < e && in_s[mem[x]] != 0)) { hit = true; break; }
        }
        if (hit && lane == 0) atomicAdd(&lam[rr_stratum[r]], 1ull);
    }
}

__global__ void k_mark(const int32_t* __restrict__ seeds, int32_t k, uint8_t* __restrict__ in_s) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x)
        in_s[seeds[i]] = 1;
}

// ---- batched form: greedy max coverage and the R2 coverage of many queries, one block each ----
// A query's block builds the inverted index of its R1 view, runs the k greedy rounds (argmax over
// the unpicked vertices, lowest id on ties; retirement of the covered sets) and counts the sets
// of its R2 view that hold a seed: the same integer arithmetic as the grid kernels above, so the
// seeds and coverages are identical. Scratch per block, sized for the batch's largest graph and
// view; queries are taken from a counter, so a block that finishes a small query takes the next.
constexpr int kGBThreads = 1024;
constexpr int kGBWarps = kGBThreads / 32;

struct GreedyBatchQuery {
    const int64_t* off1;
    const int32_t* mem1;
    const uint8_t* str1;
    const uint32_t* j1;
    int64_t count1;
    Limits L1;
    const int64_t* off2;
    const int32_t* mem2;
    const uint8_t* str2;
    const uint32_t* j2;
    int64_t count2;
    Limits L2;
    Weights W;
    int32_t n, k;
    int32_t* seeds;             // k entries
    unsigned long long* lam;    // lambda_r1[16], lambda_r2[16]
};

struct GreedyBatchParams {
    const GreedyBatchQuery* q;
    int nq;
    unsigned int* next;
    unsigned long long* score;  // per block: n_cap
    uint32_t* off;              // per block: n_cap + 1 (counts, then index ends)
    uint8_t* picked;            // per block: n_cap
    uint32_t* inv;              // per block: inv_cap
    uint32_t* covered;          // per block: cov_cap
    int64_t n_cap, inv_cap, cov_cap;
};

__global__ void __launch_bounds__(kGBThreads, 1) k_greedy_batch(GreedyBatchParams B) {
    __shared__ unsigned long long s_lam[2 * HYPERIM_NSTRATA];
    __shared__ unsigned long long ss[kGBWarps];
    __shared__ uint32_t si[kGBWarps];
    __shared__ uint32_t s_part[kGBWarps];
    __shared__ int s_q, s_best;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long* score = B.score + (int64_t)blockIdx.x * B.n_cap;
    uint32_t* off = B.off + (int64_t)blockIdx.x * (B.n_cap + 1);
    uint8_t* picked = B.picked + (int64_t)blockIdx.x * B.n_cap;
    uint32_t* inv = B.inv + (int64_t)blockIdx.x * B.inv_cap;
    uint32_t* covered = B.covered + (int64_t)blockIdx.x * B.cov_cap;
    for (;;) {
        if (threadIdx.x == 0) s_q = (int)atomicAdd(B.next, 1u);
        __syncthreads();
        if (s_q >= B.nq) break;
        const GreedyBatchQuery& Q = B.q[s_q];
        const int32_t n = Q.n;
        for (int64_t v = threadIdx.x; v < n; v += kGBThreads) {
            score[v] = 0;
            off[v] = 0;
            picked[v] = 0;
        }
        for (int64_t r = threadIdx.x; r < Q.count1; r += kGBThreads) covered[r] = 0;
        if (threadIdx.x < 2 * HYPERIM_NSTRATA) s_lam[threadIdx.x] = 0;
        __syncthreads();
        // occurrences of each vertex over the R1 view
        for (int64_t r = wid; r < Q.count1; r += kGBWarps) {
            if (Q.L1.skip(Q.str1, Q.j1, r)) continue;
            for (int64_t x = Q.off1[r] + lane; x < Q.off1[r + 1]; x += 32) atomicAdd(&off[Q.mem1[x]], 1u);
        }
        __syncthreads();
        // exclusive scan of the counts, in place: each thread one contiguous range
        {
            const int64_t per = ((int64_t)n + kGBThreads - 1) / kGBThreads;
            const int64_t b = (int64_t)threadIdx.x * per, e = min((int64_t)n, b + per);
            uint32_t sum = 0;
            for (int64_t v = b; v < e; ++v) sum += __ldcg(off + v);
            uint32_t incl = sum;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane == 31) s_part[wid] = incl;
            __syncthreads();
            uint32_t base = 0;
            for (int w = 0; w < wid; ++w) base += s_part[w];
            uint32_t run = base + incl - sum;
            for (int64_t v = b; v < e; ++v) {
                const uint32_t c = __ldcg(off + v);
                off[v] = run;
                run += c;
            }
        }
        __syncthreads();
        // inverted index and initial scores; afterwards off[v] is the end of v's entries
        for (int64_t r = wid; r < Q.count1; r += kGBWarps) {
            if (Q.L1.skip(Q.str1, Q.j1, r)) continue;
            const unsigned long long w = Q.W.w[Q.str1[r]];
            for (int64_t x = Q.off1[r] + lane; x < Q.off1[r + 1]; x += 32) {
                const int32_t v = Q.mem1[x];
                inv[atomicAdd(&off[v], 1u)] = (uint32_t)r;
                atomicAdd(&score[v], w);
            }
        }
        __syncthreads();
        for (int round = 0; round < Q.k; ++round) {
            unsigned long long bs = 0;
            uint32_t bi = 0xFFFFFFFFu;
            scan_unpicked<true>(score, picked, n, threadIdx.x, kGBThreads, bs, bi);
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long os = __shfl_xor_sync(0xFFFFFFFFu, bs, o);
                const uint32_t oi = __shfl_xor_sync(0xFFFFFFFFu, bi, o);
                if (better(os, oi, bs, bi)) { bs = os; bi = oi; }
            }
            if (lane == 0) { ss[wid] = bs; si[wid] = bi; }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int w = 1; w < kGBWarps; ++w)
                    if (better(ss[w], si[w], bs, bi)) { bs = ss[w]; bi = si[w]; }
                s_best = (int)bi;
                Q.seeds[round] = (int32_t)bi;
                picked[bi] = 1;
            }
            __syncthreads();
            const int32_t v = s_best;
            const int64_t b = v ? (int64_t)__ldcg(off + v - 1) : 0, e = __ldcg(off + v);
            for (int64_t t = b + wid; t < e; t += kGBWarps) {
                const uint32_t r = inv[t];
                uint32_t old = 0;
                if (lane == 0) old = atomicExch(&covered[r], 1u);
                old = __shfl_sync(0xFFFFFFFFu, old, 0);
                if (old) continue;
                const int s = Q.str1[r];
                const unsigned long long neg = 0ull - Q.W.w[s];
                if (lane == 0) atomicAdd(&s_lam[s], 1ull);
                for (int64_t x = Q.off1[r] + lane; x < Q.off1[r + 1]; x += 32) atomicAdd(&score[Q.mem1[x]], neg);
            }
            __syncthreads();
        }
        // coverage of the seed set on the R2 view
        for (int64_t r = wid; r < Q.count2; r += kGBWarps) {
            if (Q.L2.skip(Q.str2, Q.j2, r)) continue;
            const int64_t b = Q.off2[r], e = Q.off2[r + 1];
            bool hit = false;
            for (int64_t base = b; base < e; base += 32) {
                const int64_t x = base + lane;
                if (__any_sync(0xFFFFFFFFu, x < e && picked[Q.mem2[x]] != 0)) { hit = true; break; }
            }
            if (hit && lane == 0) atomicAdd(&s_lam[HYPERIM_NSTRATA + Q.str2[r]], 1ull);
        }
        __syncthreads();
        if (threadIdx.x < 2 * HYPERIM_NSTRATA) Q.lam[threadIdx.x] = s_lam[threadIdx.x];
        __syncthreads();
    }
}

int grid_cap(int64_t items, int threads, int sm, int per_sm) {
    int64_t b = (items + threads - 1) / threads;
    const int64_t cap = (int64_t)sm * per_sm;
    if (b < 1) b = 1;
    return (int)std::min(b, cap);
}

}  // namespace

namespace {
// the view of p that lim names (nullptr: the whole pool); lim[s] <= p->n_s[s]
Limits make_limits(const hyperim_pool* p, const uint64_t* lim, uint64_t view_ns[HYPERIM_NSTRATA]) {
    Limits L{};
    for (int i = 0; i < HYPERIM_NSTRATA; ++i) {
        view_ns[i] = lim ? std::min<uint64_t>(lim[i], p->n_s[i]) : p->n_s[i];
        L.lim[i] = (uint32_t)std::min<uint64_t>(view_ns[i], 0xFFFFFFFFull);
        if (view_ns[i] < p->n_s[i]) L.on = 1;
    }
    return L;
}
}  // namespace

hyperim_status greedy(hyperim_graph* g, hyperim_pool* p, int32_t k, int32_t* seeds_host,
                      uint64_t lambda_s[HYPERIM_NSTRATA], uint64_t* prefix_upper, const uint64_t* lim) {
    cudaStream_t s = g->stream;
    const int32_t n = g->n;
    const int64_t N = p->count, T = p->total;
    const int sm = g->sm_count;
    if (N >= (int64_t)0xFFFFFFFFll) return set_error(HYPERIM_EOVERFLOW, "more than 2^32 - 1 RR sets");
    uint64_t view_ns[HYPERIM_NSTRATA];
    const Limits L = make_limits(p, lim, view_ns);
    Weights W;
    for (int i = 0; i < HYPERIM_NSTRATA; ++i)
        W.w[i] = stratum_weight(g, p->root_mode, view_ns[i], i);
    hyperim_status st;
    CallBuffers tmp(g);
    uint32_t *cnt = nullptr, *inv = nullptr, *covered = nullptr, *bid = nullptr, *ticket = nullptr;
    int64_t* inv_off = nullptr;
    unsigned long long *score = nullptr, *lam = nullptr, *bscore = nullptr;
    uint8_t* picked = nullptr;
    int32_t *best = nullptr, *seeds_d = nullptr;
    const int ablocks = grid_cap(n, kArgThreads, sm, 2);
    const size_t bytes_cnt = sizeof(uint32_t) * ((size_t)n + 1);
    const size_t bytes_inv = sizeof(uint32_t) * (size_t)std::max<int64_t>(T, 1);
    const size_t bytes_cov = sizeof(uint32_t) * (size_t)std::max<int64_t>(N, 1);
    if ((st = tmp.alloc(&cnt, bytes_cnt))) return st;
    if ((st = tmp.alloc(&inv_off, sizeof(int64_t) * ((size_t)n + 1)))) return st;
    if ((st = tmp.alloc(&inv, bytes_inv))) return st;
    if ((st = tmp.alloc(&score, sizeof(unsigned long long) * (size_t)n))) return st;
    if ((st = tmp.alloc(&picked, (size_t)n))) return st;
    if ((st = tmp.alloc(&covered, bytes_cov))) return st;
    if ((st = tmp.alloc(&lam, sizeof(unsigned long long) * HYPERIM_NSTRATA))) return st;
    if ((st = tmp.alloc(&bscore, sizeof(unsigned long long) * ablocks))) return st;
    if ((st = tmp.alloc(&bid, sizeof(uint32_t) * ablocks))) return st;
    if ((st = tmp.alloc(&ticket, sizeof(uint32_t) * 2))) return st;
    if ((st = tmp.alloc(&best, sizeof(int32_t) * 2))) return st;
    if ((st = tmp.alloc(&seeds_d, sizeof(int32_t) * (size_t)k))) return st;
    TopK* tk = nullptr;
    unsigned int* hist = nullptr;
    unsigned long long* part = nullptr;
    const int tblocks = ablocks;
    if ((st = tmp.alloc(&tk, sizeof(TopK)))) return st;
    if ((st = tmp.alloc(&hist, sizeof(unsigned int) * 256))) return st;
    if ((st = tmp.alloc(&part, sizeof(unsigned long long) * 2 * (size_t)tblocks))) return st;
    {
        TopK t0{};
        t0.kleft = (unsigned int)k;
        t0.best_lo = ~0ull;
        t0.best_hi = ~0ull;
        HYP_CUDA(cudaMemcpyAsync(tk, &t0, sizeof(TopK), cudaMemcpyHostToDevice, s));
        HYP_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned int) * 256, s));
    }
    auto topk_round = [&]() -> hyperim_status {
        for (int pass = 0; pass < 8; ++pass) {
            { k_topk_hist<<<tblocks, kArgThreads, 0, s>>>(score, picked, n, tk, pass, hist); count_launch(); }
            { k_topk_select<<<1, 1, 0, s>>>(tk, hist, pass); count_launch(); }
        }
        { k_topk_sum<<<tblocks, kArgThreads, 0, s>>>(score, picked, n, tk, part, (unsigned int)k); count_launch(); }
        return HYPERIM_OK;
    };
    HYP_CUDA(cudaMemsetAsync(cnt, 0, bytes_cnt, s));
    HYP_CUDA(cudaMemsetAsync(score, 0, sizeof(unsigned long long) * (size_t)n, s));
    HYP_CUDA(cudaMemsetAsync(picked, 0, (size_t)n, s));
    HYP_CUDA(cudaMemsetAsync(covered, 0, bytes_cov, s));
    HYP_CUDA(cudaMemsetAsync(lam, 0, sizeof(unsigned long long) * HYPERIM_NSTRATA, s));
    HYP_CUDA(cudaMemsetAsync(ticket, 0, sizeof(uint32_t) * 2, s));
    if (T > 0 && !L.on) { k_count_occ<<<grid_cap(T, 256, sm, 32), 256, 0, s>>>(p->rr_mem, T, cnt); count_launch(); }
    if (T > 0 && L.on)
        { k_count_occ_view<<<grid_cap(N * 32, 256, sm, 32), 256, 0, s>>>(p->rr_off, p->rr_mem, p->rr_stratum,
                                                                        p->rr_j, N, L, cnt); count_launch(); }
    if ((st = exclusive_scan_u32_to_i64(g, cnt, inv_off, n))) return st;
    HYP_CUDA(cudaMemsetAsync(cnt, 0, bytes_cnt, s));
    if (N > 0)
        { k_scatter_inv<<<grid_cap(N * 32, 256, sm, 32), 256, 0, s>>>(p->rr_off, p->rr_mem, p->rr_stratum,
                                                                    p->rr_j, N, L, inv_off, cnt, inv, score,
                                                                    W); count_launch(); }
    const int rblocks = sm * 8;
    for (int32_t round = 0; round < k; ++round) {
        if (prefix_upper) topk_round();
        { k_argmax<<<ablocks, kArgThreads, 0, s>>>(score, picked, n, bscore, bid, ticket, best, seeds_d,
                                                 round, tk); count_launch(); }
        { k_retire<<<rblocks, 256, 0, s>>>(best, inv_off, inv, p->rr_off, p->rr_mem, p->rr_stratum,
                                         covered, score, lam, W); count_launch(); }
    }
    if (prefix_upper) topk_round();  // i = k: the whole seed set
    HYP_CUDA(cudaGetLastError());
    unsigned long long hl[HYPERIM_NSTRATA];
    TopK th{};
    HYP_CUDA(cudaMemcpyAsync(seeds_host, seeds_d, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaMemcpyAsync(hl, lam, sizeof(hl), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaMemcpyAsync(&th, tk, sizeof(TopK), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < HYPERIM_NSTRATA; ++i) lambda_s[i] = hl[i];
    if (prefix_upper) {
        prefix_upper[0] = th.best_lo;
        prefix_upper[1] = th.best_hi;
    }
    return check_device_status(g, "greedy");
}

hyperim_status coverage(hyperim_graph* g, hyperim_pool* p, const int32_t* seeds_host, int32_t k,
                        uint64_t lambda_s[HYPERIM_NSTRATA], const uint64_t* lim) {
    cudaStream_t s = g->stream;
    const int64_t N = p->count;
    uint64_t view_ns[HYPERIM_NSTRATA];
    const Limits L = make_limits(p, lim, view_ns);
    hyperim_status st;
    CallBuffers tmp(g);
    uint8_t* in_s = nullptr;
    unsigned long long* lam = nullptr;
    int32_t* sd = nullptr;
    const size_t kk = (size_t)std::max(k, 1);
    if ((st = tmp.alloc(&in_s, (size_t)g->n))) return st;
    if ((st = tmp.alloc(&lam, sizeof(unsigned long long) * HYPERIM_NSTRATA))) return st;
    if ((st = tmp.alloc(&sd, sizeof(int32_t) * kk))) return st;
    HYP_CUDA(cudaMemsetAsync(in_s, 0, (size_t)g->n, s));
    HYP_CUDA(cudaMemsetAsync(lam, 0, sizeof(unsigned long long) * HYPERIM_NSTRATA, s));
    if (k > 0) {
        HYP_CUDA(cudaMemcpyAsync(sd, seeds_host, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, s));
        { k_mark<<<grid_cap(k, 256, g->sm_count, 4), 256, 0, s>>>(sd, k, in_s); count_launch(); }
    }
    if (N > 0)
        { k_coverage<<<grid_cap(N * 32, 256, g->sm_count, 32), 256, 0, s>>>(p->rr_off, p->rr_mem,
                                                                          p->rr_stratum, p->rr_j, N, L, in_s,
                                                                          lam); count_launch(); }
    HYP_CUDA(cudaGetLastError());
    unsigned long long hl[HYPERIM_NSTRATA];
    HYP_CUDA(cudaMemcpyAsync(hl, lam, sizeof(hl), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < HYPERIM_NSTRATA; ++i) lambda_s[i] = hl[i];
    return check_device_status(g, "coverage");
}

}  // namespace hyperim

// ---- greedy one round at a time (sharded pools) ---------------------------------------------
// The state of Algorithm 1 on one pool (a prefix view of it): the inverted index and the
// weighted marginal scores of its RR sets, which sets are covered, which vertices are picked and
// Lambda per stratum. greedy_pick takes the argmax over a score vector the caller supplies --
// the sum, over every shard of a pool, of their scores (integer sums: the order of the shards'
// additions does not matter) -- then retires the pick's uncovered sets of this shard.
namespace hyperim {

struct GreedyState {
    hyperim_graph* g = nullptr;
    hyperim_pool* p = nullptr;
    std::shared_lock<std::shared_mutex> lock;  // the pool may not grow while the state lives
    Weights W{};
    int ablocks = 0;
    uint32_t *cnt = nullptr, *inv = nullptr, *covered = nullptr, *bid = nullptr, *ticket = nullptr;
    int64_t* inv_off = nullptr;
    unsigned long long *score = nullptr, *lam = nullptr, *bscore = nullptr;
    uint8_t* picked = nullptr;
    int32_t *best = nullptr, *seed_d = nullptr;
    TopK* tk = nullptr;
    size_t bytes_cnt = 0, bytes_inv = 0, bytes_cov = 0;
};

namespace {
void free_state(GreedyState* s) {
    hyperim_graph* g = s->g;
    const size_t n = (size_t)g->n;
    dev_free(g, s->cnt, s->bytes_cnt);
    dev_free(g, s->inv_off, sizeof(int64_t) * (n + 1));
    dev_free(g, s->inv, s->bytes_inv);
    dev_free(g, s->score, sizeof(unsigned long long) * n);
    dev_free(g, s->picked, n);
    dev_free(g, s->covered, s->bytes_cov);
    dev_free(g, s->lam, sizeof(unsigned long long) * HYPERIM_NSTRATA);
    dev_free(g, s->bscore, sizeof(unsigned long long) * s->ablocks);
    dev_free(g, s->bid, sizeof(uint32_t) * s->ablocks);
    dev_free(g, s->ticket, sizeof(uint32_t) * 2);
    dev_free(g, s->best, sizeof(int32_t) * 2);
    dev_free(g, s->seed_d, sizeof(int32_t));
    dev_free(g, s->tk, sizeof(TopK));
    cudaStreamSynchronize(g->stream);
    delete s;
}
}  // namespace

hyperim_status greedy_begin(hyperim_graph* g, hyperim_pool* p, const uint64_t* lim, GreedyState** out) {
    *out = nullptr;
    GreedyState* s = new (std::nothrow) GreedyState();
    if (!s) return set_error(HYPERIM_ENOMEM, "host allocation failed");
    s->g = g;
    s->p = p;
    s->lock = std::shared_lock<std::shared_mutex>(p->mu);
    cudaStream_t st_ = g->stream;
    const int32_t n = g->n;
    const int64_t N = p->count, T = p->total;
    const int sm = g->sm_count;
    if (N >= (int64_t)0xFFFFFFFFll) {
        delete s;
        return set_error(HYPERIM_EOVERFLOW, "more than 2^32 - 1 RR sets");
    }
    uint64_t view_ns[HYPERIM_NSTRATA];
    const Limits L = make_limits(p, lim, view_ns);
    for (int i = 0; i < HYPERIM_NSTRATA; ++i) s->W.w[i] = stratum_weight(g, p->root_mode, view_ns[i], i);
    s->ablocks = grid_cap(n, kArgThreads, sm, 2);
    s->bytes_cnt = sizeof(uint32_t) * ((size_t)n + 1);
    s->bytes_inv = sizeof(uint32_t) * (size_t)std::max<int64_t>(T, 1);
    s->bytes_cov = sizeof(uint32_t) * (size_t)std::max<int64_t>(N, 1);
    hyperim_status st;
    auto fail = [&](hyperim_status e) {
        free_state(s);
        return e;
    };
    if ((st = dev_alloc(g, (void**)&s->cnt, s->bytes_cnt)) || (st = dev_alloc(g, (void**)&s->inv_off, sizeof(int64_t) * ((size_t)n + 1))) ||
        (st = dev_alloc(g, (void**)&s->inv, s->bytes_inv)) || (st = dev_alloc(g, (void**)&s->score, sizeof(unsigned long long) * (size_t)n)) ||
        (st = dev_alloc(g, (void**)&s->picked, (size_t)n)) || (st = dev_alloc(g, (void**)&s->covered, s->bytes_cov)) ||
        (st = dev_alloc(g, (void**)&s->lam, sizeof(unsigned long long) * HYPERIM_NSTRATA)) ||
        (st = dev_alloc(g, (void**)&s->bscore, sizeof(unsigned long long) * s->ablocks)) ||
        (st = dev_alloc(g, (void**)&s->bid, sizeof(uint32_t) * s->ablocks)) || (st = dev_alloc(g, (void**)&s->ticket, sizeof(uint32_t) * 2)) ||
        (st = dev_alloc(g, (void**)&s->best, sizeof(int32_t) * 2)) || (st = dev_alloc(g, (void**)&s->seed_d, sizeof(int32_t))) ||
        (st = dev_alloc(g, (void**)&s->tk, sizeof(TopK))))
        return fail(st);
    cudaError_t e = cudaMemsetAsync(s->cnt, 0, s->bytes_cnt, st_);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->score, 0, sizeof(unsigned long long) * (size_t)n, st_);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->picked, 0, (size_t)n, st_);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->covered, 0, s->bytes_cov, st_);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->lam, 0, sizeof(unsigned long long) * HYPERIM_NSTRATA, st_);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->ticket, 0, sizeof(uint32_t) * 2, st_);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->tk, 0, sizeof(TopK), st_);
    if (e != cudaSuccess) return fail(cuda_fail(e, "greedy state"));
    if (T > 0 && !L.on) { k_count_occ<<<grid_cap(T, 256, sm, 32), 256, 0, st_>>>(p->rr_mem, T, s->cnt); count_launch(); }
    if (T > 0 && L.on)
        { k_count_occ_view<<<grid_cap(N * 32, 256, sm, 32), 256, 0, st_>>>(p->rr_off, p->rr_mem, p->rr_stratum, p->rr_j, N, L,
                                                                          s->cnt); count_launch(); }
    if ((st = exclusive_scan_u32_to_i64(g, s->cnt, s->inv_off, n))) return fail(st);
    e = cudaMemsetAsync(s->cnt, 0, s->bytes_cnt, st_);
    if (e != cudaSuccess) return fail(cuda_fail(e, "greedy state"));
    if (N > 0)
        { k_scatter_inv<<<grid_cap(N * 32, 256, sm, 32), 256, 0, st_>>>(p->rr_off, p->rr_mem, p->rr_stratum, p->rr_j, N, L,
                                                                      s->inv_off, s->cnt, s->inv, s->score, s->W); count_launch(); }
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(cuda_fail(e, "greedy index"));
    *out = s;
    return HYPERIM_OK;
}

hyperim_status greedy_scores(GreedyState* s, unsigned long long* dev_out) {
    HYP_CUDA(cudaMemcpyAsync(dev_out, s->score, sizeof(unsigned long long) * (size_t)s->g->n, cudaMemcpyDeviceToDevice,
                             s->g->stream));
    return HYPERIM_OK;
}

hyperim_status greedy_pick(GreedyState* s, const unsigned long long* dev_total, int32_t* picked) {
    hyperim_graph* g = s->g;
    hyperim_pool* p = s->p;
    cudaStream_t st_ = g->stream;
    { k_argmax<<<s->ablocks, kArgThreads, 0, st_>>>(dev_total ? dev_total : s->score, s->picked, g->n, s->bscore, s->bid,
                                                    s->ticket, s->best, s->seed_d, 0, s->tk); count_launch(); }
    { k_retire<<<g->sm_count * 8, 256, 0, st_>>>(s->best, s->inv_off, s->inv, p->rr_off, p->rr_mem, p->rr_stratum,
                                                 s->covered, s->score, s->lam, s->W); count_launch(); }
    HYP_CUDA(cudaGetLastError());
    HYP_CUDA(cudaMemcpyAsync(picked, s->best, sizeof(int32_t), cudaMemcpyDeviceToHost, st_));
    HYP_CUDA(cudaStreamSynchronize(st_));
    return check_device_status(g, "greedy pick");
}

hyperim_status greedy_end(GreedyState* s, uint64_t lambda_s[HYPERIM_NSTRATA]) {
    unsigned long long hl[HYPERIM_NSTRATA];
    cudaError_t e = cudaMemcpyAsync(hl, s->lam, sizeof(hl), cudaMemcpyDeviceToHost, s->g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->g->stream);
    if (e == cudaSuccess && lambda_s)
        for (int i = 0; i < HYPERIM_NSTRATA; ++i) lambda_s[i] = hl[i];
    free_state(s);
    if (e != cudaSuccess) return cuda_fail(e, "greedy end");
    return HYPERIM_OK;
}

hyperim_status greedy_batch(hyperim_graph* g0, const GreedyBatchItem* items, int nitems) {
    if (nitems < 1) return HYPERIM_OK;
    cudaStream_t s = g0->stream;
    hyperim_status st;
    std::vector<GreedyBatchQuery> hq((size_t)nitems);
    int64_t n_cap = 1, inv_cap = 1, cov_cap = 1, kmax = 1;
    for (int i = 0; i < nitems; ++i) {
        const GreedyBatchItem& it = items[i];
        const hyperim_pool *p1 = it.r1, *p2 = it.r2;
        if (p1->count >= (int64_t)0xFFFFFFFFll || p1->total >= (int64_t)0xFFFFFFFFll)
            return set_error(HYPERIM_EOVERFLOW, "more than 2^32 - 1 RR sets or members in a pool");
        uint64_t v1[HYPERIM_NSTRATA], v2[HYPERIM_NSTRATA];
        GreedyBatchQuery& Q = hq[i];
        Q.off1 = p1->rr_off;
        Q.mem1 = p1->rr_mem;
        Q.str1 = p1->rr_stratum;
        Q.j1 = p1->rr_j;
        Q.count1 = p1->count;
        Q.L1 = make_limits(p1, it.lim1, v1);
        Q.off2 = p2->rr_off;
        Q.mem2 = p2->rr_mem;
        Q.str2 = p2->rr_stratum;
        Q.j2 = p2->rr_j;
        Q.count2 = p2->count;
        Q.L2 = make_limits(p2, it.lim2, v2);
        for (int x = 0; x < HYPERIM_NSTRATA; ++x) Q.W.w[x] = stratum_weight(it.g, p1->root_mode, v1[x], x);
        Q.n = it.g->n;
        Q.k = it.k;
        n_cap = std::max<int64_t>(n_cap, it.g->n);
        inv_cap = std::max<int64_t>(inv_cap, p1->total);
        cov_cap = std::max<int64_t>(cov_cap, p1->count);
        kmax = std::max<int64_t>(kmax, it.k);
    }
    n_cap = (n_cap + 3) & ~(int64_t)3;  // per-block score / flag arrays stay 16- and 4-byte aligned
    // one block per SM at most, and no more blocks than the scratch budget allows
    const size_t per_block = 8 * (size_t)n_cap + 4 * ((size_t)n_cap + 1) + (size_t)n_cap + 4 * (size_t)inv_cap +
                             4 * (size_t)cov_cap;
    const size_t budget = (size_t)2 << 30;
    int blocks = (int)std::min<int64_t>(nitems, std::max(1, g0->sm_count));
    blocks = (int)std::max<size_t>(1, std::min<size_t>((size_t)blocks, budget / std::max<size_t>(per_block, 1)));
    CallBuffers tmp(g0);
    GreedyBatchQuery* d_q = nullptr;
    int32_t* d_seeds = nullptr;
    unsigned long long* d_lam = nullptr;
    unsigned int* d_next = nullptr;
    unsigned long long* score = nullptr;
    uint32_t *off = nullptr, *inv = nullptr, *covered = nullptr;
    uint8_t* picked = nullptr;
    if ((st = tmp.alloc(&d_q, sizeof(GreedyBatchQuery) * (size_t)nitems))) return st;
    if ((st = tmp.alloc(&d_seeds, sizeof(int32_t) * (size_t)nitems * (size_t)kmax))) return st;
    if ((st = tmp.alloc(&d_lam, sizeof(unsigned long long) * 2 * HYPERIM_NSTRATA * (size_t)nitems))) return st;
    if ((st = tmp.alloc(&d_next, sizeof(unsigned int)))) return st;
    if ((st = tmp.alloc(&score, sizeof(unsigned long long) * (size_t)n_cap * blocks))) return st;
    if ((st = tmp.alloc(&off, sizeof(uint32_t) * ((size_t)n_cap + 1) * blocks))) return st;
    if ((st = tmp.alloc(&picked, (size_t)n_cap * blocks))) return st;
    if ((st = tmp.alloc(&inv, sizeof(uint32_t) * (size_t)inv_cap * blocks))) return st;
    if ((st = tmp.alloc(&covered, sizeof(uint32_t) * (size_t)cov_cap * blocks))) return st;
    for (int i = 0; i < nitems; ++i) {
        hq[i].seeds = d_seeds + (size_t)i * (size_t)kmax;
        hq[i].lam = d_lam + (size_t)i * 2 * HYPERIM_NSTRATA;
    }
    HYP_CUDA(cudaMemcpyAsync(d_q, hq.data(), sizeof(GreedyBatchQuery) * hq.size(), cudaMemcpyHostToDevice, s));
    HYP_CUDA(cudaMemsetAsync(d_next, 0, sizeof(unsigned int), s));
    GreedyBatchParams B;
    B.q = d_q;
    B.nq = nitems;
    B.next = d_next;
    B.score = score;
    B.off = off;
    B.picked = picked;
    B.inv = inv;
    B.covered = covered;
    B.n_cap = n_cap;
    B.inv_cap = inv_cap;
    B.cov_cap = cov_cap;
    { k_greedy_batch<<<blocks, kGBThreads, 0, s>>>(B); count_launch(); }
    HYP_CUDA(cudaGetLastError());
    std::vector<int32_t> seeds((size_t)nitems * (size_t)kmax);
    std::vector<unsigned long long> lam((size_t)nitems * 2 * HYPERIM_NSTRATA);
    HYP_CUDA(cudaMemcpyAsync(seeds.data(), d_seeds, sizeof(int32_t) * seeds.size(), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaMemcpyAsync(lam.data(), d_lam, sizeof(unsigned long long) * lam.size(), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < nitems; ++i) {
        const GreedyBatchItem& it = items[i];
        for (int x = 0; x < it.k; ++x) it.seeds_host[x] = seeds[(size_t)i * (size_t)kmax + x];
        for (int x = 0; x < HYPERIM_NSTRATA; ++x) {
            it.lambda_r1[x] = lam[(size_t)i * 2 * HYPERIM_NSTRATA + x];
            it.lambda_r2[x] = lam[(size_t)i * 2 * HYPERIM_NSTRATA + HYPERIM_NSTRATA + x];
        }
    }
    return check_device_status(g0, "greedy (batch)");
}

}  // namespace hyperim
