// Incidence store and layer profile (Sec. 2.1 and Sec. 3.1.1), built on the device.
//
//   he -> members : hyperedges as sorted vertex sets (repeated ids collapsed)
//   v  -> he      : hyperedges containing each vertex, ascending
//   profile       : for every vertex mu, the layers of A(mu) keyed by w(mu,nu), L_1 = largest w,
//                   with n(L_i), the activation threshold floor(p_i 2^32) and the h = 0 shortcut
//   strata        : s(mu) = min(l_mu, 15); V_s lists in ascending id order
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_math.cuh"
#include "internal.h"
#include "mat.cuh"

namespace hyperim {
namespace {

constexpr int kProfThreads = 512;  // two blocks (32 warps) per SM: the sorts are latency-bound
constexpr int kProfBuf = 8192;  // on-chip keys of the profile kernel (power of two)
constexpr int kProfHist = 1024; // on-chip multiplicity histogram bins (d_H >= this: global)
constexpr int kBucketsMax = 4096;
constexpr int kProfWarpT = 1024;  // vertices with at most this many positions: warp profile
constexpr int kPWWarps = 4;
constexpr int kPWThreads = kPWWarps * 32;
constexpr int kProfMidT = 2048;  // vertices with at most this many positions: warp profile, listed
constexpr int kPMWarps = 2;

__device__ __forceinline__ void dev_fail(DevStatus* st, int32_t code, int32_t detail) {
    if (atomicCAS(&st->code, 0, code) == 0) st->detail = detail;
}

// ---- validation -------------------------------------------------------------------------------
__global__ void k_check_offsets(const int32_t* off, int32_t m, DevStatus* st) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        if (off[e + 1] < off[e]) dev_fail(st, kErrBadOffsets, (int32_t)e);
    if (blockIdx.x == 0 && threadIdx.x == 0 && off[0] != 0) dev_fail(st, kErrBadOffsets, 0);
}

// ---- normalisation: sort each hyperedge's members, drop repeats (a hyperedge is a set) -------
// One warp per hyperedge. A member is kept at its first occurrence only; its position in the
// sorted set is the number of distinct values below it.
__global__ void k_normalise(const int32_t* __restrict__ off, const int32_t* __restrict__ mem,
                            int32_t m, int32_t n, int32_t* __restrict__ out,
                            uint8_t* __restrict__ first, uint32_t* __restrict__ newsize,
                            DevStatus* st) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = warp; e < m; e += nwarps) {
        const int32_t b = off[e], len = off[e + 1] - b;
        if (len <= 32) {
            const int32_t x = lane < len ? mem[b + lane] : INT32_MAX;
            if (lane < len && (x < 0 || x >= n)) dev_fail(st, kErrBadMember, (int32_t)e);
            bool dup = false;
            for (int j = 0; j < len; ++j) {
                const int32_t y = __shfl_sync(0xFFFFFFFFu, x, j);
                if (y == x && j < lane) dup = true;
            }
            int below = 0;
            for (int j = 0; j < len; ++j) {
                const int32_t y = __shfl_sync(0xFFFFFFFFu, x, j);
                const int ydup = __shfl_sync(0xFFFFFFFFu, dup ? 1 : 0, j);
                if (!ydup && y < x) ++below;
            }
            const bool keep = lane < len && !dup;
            const uint32_t kb = __ballot_sync(0xFFFFFFFFu, keep);
            if (keep) out[b + below] = x;
            if (lane == 0) newsize[e] = __popc(kb);
        } else {
            // first-occurrence flags, then positions among first occurrences
            for (int i = lane; i < len; i += 32) {
                const int32_t x = mem[b + i];
                if (x < 0 || x >= n) dev_fail(st, kErrBadMember, (int32_t)e);
                bool dup = false;
                for (int j = 0; j < i && !dup; ++j) dup = mem[b + j] == x;
                first[b + i] = dup ? 0 : 1;
            }
            __syncwarp();
            int keep = 0;
            for (int i = lane; i < len; i += 32) {
                if (!first[b + i]) continue;
                const int32_t x = mem[b + i];
                int below = 0;
                for (int j = 0; j < len; ++j) below += (first[b + j] && mem[b + j] < x) ? 1 : 0;
                out[b + below] = x;
                ++keep;
            }
            for (int o = 16; o > 0; o >>= 1) keep += __shfl_xor_sync(0xFFFFFFFFu, keep, o);
            if (lane == 0) newsize[e] = keep;
        }
    }
}

__global__ void k_compact_he(const int32_t* __restrict__ off_in, const int32_t* __restrict__ tmp,
                             const int64_t* __restrict__ off_new, int32_t m,
                             int32_t* __restrict__ he_off, int32_t* __restrict__ he_mem) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = warp; e < m; e += nwarps) {
        const int32_t src = off_in[e];
        const int64_t dst = off_new[e], len = off_new[e + 1] - dst;
        for (int64_t i = lane; i < len; i += 32) he_mem[dst + i] = tmp[src + i];
        if (lane == 0) he_off[e] = (int32_t)dst;
        if (lane == 0 && e == m - 1) he_off[m] = (int32_t)off_new[m];
    }
}

// ---- vertex -> hyperedge lists ------------------------------------------------------------------
__global__ void k_count_dh(const int32_t* __restrict__ he_mem, int64_t nnz, uint32_t* cnt) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < nnz;
         x += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[he_mem[x]], 1u);
}

__global__ void k_scatter_vhe(const int32_t* __restrict__ he_off, const int32_t* __restrict__ he_mem,
                              int32_t m, const int64_t* __restrict__ v_off64, uint32_t* cur,
                              int32_t* __restrict__ v_he, int32_t* __restrict__ tsum) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = warp; e < m; e += nwarps) {
        const int32_t b = he_off[e], len = he_off[e + 1] - b;
        for (int i = lane; i < len; i += 32) {
            const int32_t v = he_mem[b + i];
            const uint32_t pos = atomicAdd(&cur[v], 1u);
            v_he[v_off64[v] + pos] = (int32_t)e;
            atomicAdd(&tsum[v], len);
        }
    }
}

// sort each vertex's hyperedge list (distinct ids): position = number of smaller ids
__global__ void k_sort_vhe(const int64_t* __restrict__ v_off64, int32_t n,
                           const int32_t* __restrict__ in, int32_t* __restrict__ out,
                           int32_t* __restrict__ v_off32) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        const int64_t b = v_off64[v], len = v_off64[v + 1] - b;
        for (int64_t i = lane; i < len; i += 32) {
            const int32_t x = in[b + i];
            int below = 0;
            for (int64_t j = 0; j < len; ++j) below += in[b + j] < x ? 1 : 0;
            out[b + below] = x;
        }
        if (lane == 0) v_off32[v] = (int32_t)b;
        if (lane == 0 && v == n - 1) v_off32[n] = (int32_t)v_off64[n];
    }
}

// ---- layer profile: pass 1 ----------------------------------------------------------------------
// For each vertex mu: the multiplicities w(mu,nu) over its distinct neighbours nu, histogrammed by
// w; the distinct w values in descending order with their counts n_i are written to
// pairs[v_off[mu] ...] (at most d_H(mu) of them). Also l_mu and deg(mu).
struct ProfScratch {
    uint32_t* big;       // per block: bucketed members (big_cap entries)
    uint32_t* hist;      // per block: multiplicity histogram when d_H exceeds kProfHist
    int64_t big_cap;
    int64_t hist_cap;
};

// Distinct multiplicities of hist[1..dh] in descending order -> pairs (w_i, n_i), l, deg and the
// maxima; one warp (lanes 0..31).
__device__ void emit_layers(const uint32_t* hist, int dh, int32_t mu, int32_t e0, uint2* __restrict__ pairs,
                            uint32_t* __restrict__ nlayers, uint32_t* __restrict__ deg,
                            unsigned long long* __restrict__ maxima) {
    const int lane = threadIdx.x & 31;
    int carry = 0;
    uint32_t dsum = 0, nmax = 0;
    for (int top = dh; top >= 1; top -= 32) {
        const int w = top - lane;
        const uint32_t c = w >= 1 ? hist[w] : 0u;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, c > 0);
        const int pos = carry + __popc(bal & lanemask_lt());
        if (c > 0) pairs[e0 + pos] = make_uint2((uint32_t)w, c);
        carry += __popc(bal);
        dsum += c;
        nmax = max(nmax, c);
    }
    dsum = __reduce_add_sync(0xFFFFFFFFu, dsum);
    nmax = __reduce_max_sync(0xFFFFFFFFu, nmax);
    if (lane == 0) {
        nlayers[mu] = (uint32_t)carry;
        deg[mu] = dsum;
        atomicMax(&maxima[0], (unsigned long long)carry);
        atomicMax(&maxima[1], (unsigned long long)dsum);
        atomicMax(&maxima[2], (unsigned long long)nmax);
    }
}

// Layer profile, small vertices: one warp per vertex whose hyperedges hold at most Cap
// positions (mu's own included), and every vertex with d_H <= 1 (list == nullptr: all vertices;
// else the listed ones, all with d_H >= 2 and more than the smaller cap's positions). The
// members are gathered once into a raw copy and counted into buckets of their top id bits,
// scattered into id order and sorted per bucket (the RR kernel's warp sort), then the runs give
// the multiplicity histogram.
template <int Cap, int W>
__global__ void __launch_bounds__(W * 32)
k_profile_warp(int32_t n, const int32_t* __restrict__ list, const int32_t* __restrict__ v_off,
               const int2* __restrict__ v_span, const int32_t* __restrict__ he_mem,
               const int32_t* __restrict__ tsum, int id_bits, uint2* __restrict__ pairs,
               uint32_t* __restrict__ nlayers, uint32_t* __restrict__ deg,
               unsigned long long* __restrict__ maxima) {
    __shared__ uint32_t raw_s[W][Cap + 4];
    __shared__ uint32_t buf_s[W][Cap];
    __shared__ int bkt_s[W][256];
    __shared__ int pre_s[W][2 * 32 + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t* raw = raw_s[wid];
    uint32_t* buf = buf_s[wid];
    int* bkt = bkt_s[wid];
    const int64_t nw = (int64_t)gridDim.x * W;
    for (int64_t v = (int64_t)blockIdx.x * W + wid; v < n; v += nw) {
        const int32_t mu = list ? list[v] : (int32_t)v;
        const int32_t e0 = v_off[mu], dh = v_off[mu + 1] - e0;
        if (dh == 0) {
            if (lane == 0) { nlayers[mu] = 0; deg[mu] = 0; }
            continue;
        }
        if (dh == 1) {
            if (lane == 0) {
                const uint32_t nb = (uint32_t)(v_span[e0].y - 1);
                nlayers[mu] = nb > 0 ? 1 : 0;
                deg[mu] = nb;
                if (nb > 0) {
                    pairs[e0] = make_uint2(1u, nb);
                    atomicMax(&maxima[0], 1ull);
                    atomicMax(&maxima[1], (unsigned long long)nb);
                    atomicMax(&maxima[2], (unsigned long long)nb);
                }
            }
            continue;
        }
        const int ts = tsum[mu];
        if (ts > Cap) continue;  // a vertex of a larger kernel
        const int T = ts - dh;
        const int nbits = bucket_bits(T, 8);
        const int nb = 1 << nbits;
        const int shift = id_bits > nbits ? id_bits - nbits : 0;
        const uint32_t key_mask = (uint32_t)nb - 1;
        for (int b = lane; b < nb; b += 32) bkt[b] = 0;
        __syncwarp();
        for_each_position<32>(v_span, he_mem, e0, dh, pre_s[wid], [&](int pos, uint32_t x) {
            raw[pos] = x;
            if (x != (uint32_t)mu) atomicAdd(&bkt[(x >> shift) & key_mask], 1);
        });
        const int maxb = warp_bucket_scan(bkt, nb);
        warp_scatter_sort(raw, ts, (uint32_t)mu, buf, T, bkt, nb, 0u, shift, key_mask, maxb);
        // multiplicity histogram over w in [1, dh] (the raw copy is free again)
        uint32_t* hist = raw;
        for (int w = lane; w <= dh; w += 32) hist[w] = 0;
        __syncwarp();
        walk_runs<32>(buf, T, [&](bool start, uint32_t, int mult) -> bool {
            if (start) atomicAdd(&hist[mult], 1u);
            return false;
        });
        __syncwarp();
        emit_layers(hist, dh, mu, e0, pairs, nlayers, deg, maxima);
        __syncwarp();
    }
}

// ---- largest first: an order of listed vertices by descending neighbourhood size ----------
// The block-per-vertex kernels take their vertices from a counter; a hub taken last would leave
// one block running while the rest of the grid idles. Listing vertices in descending size (by
// buckets of a quarter octave: exact order within a bucket does not matter) lets the largest start
// first. Each vertex's output does not depend on the order in which vertices are processed.
constexpr int kSizeBuckets = 128;

__device__ __forceinline__ int size_bucket(int32_t t) {
    if (t < 4) return 0;
    const int lg = 31 - __clz(t);
    return min(kSizeBuckets - 1, 4 * lg + (int)(((uint32_t)t >> (lg - 2)) & 3u));
}

__global__ void k_size_hist(const int32_t* __restrict__ list, int64_t count, const int32_t* __restrict__ tsum,
                            unsigned int* __restrict__ hist) {
    __shared__ unsigned int h[kSizeBuckets];
    for (int i = threadIdx.x; i < kSizeBuckets; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[size_bucket(tsum[list[i]])], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < kSizeBuckets; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// one thread: bucket starts in descending bucket order
__global__ void k_size_starts(unsigned int* __restrict__ hist) {
    unsigned int run = 0;
    for (int b = kSizeBuckets - 1; b >= 0; --b) {
        const unsigned int c = hist[b];
        hist[b] = run;
        run += c;
    }
}

__global__ void k_size_scatter(const int32_t* __restrict__ list, int64_t count, const int32_t* __restrict__ tsum,
                               unsigned int* __restrict__ start, int emit_index, int32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = list[i];
        out[atomicAdd(&start[size_bucket(tsum[v])], 1u)] = emit_index ? (int32_t)i : v;
    }
}

// Vertices with d_H >= 2 and lo < positions <= hi (the mid-size warp kernel's, then the block
// kernel's with hi = INT_MAX).
__global__ void k_big_flags(int32_t n, const int32_t* __restrict__ v_off, const int32_t* __restrict__ tsum,
                            int32_t lo, int32_t hi, uint32_t* __restrict__ flag) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        flag[v] = (v_off[v + 1] - v_off[v] >= 2 && tsum[v] > lo && tsum[v] <= hi) ? 1u : 0u;
}

__global__ void k_big_list(int32_t n, const uint32_t* __restrict__ flag, const int64_t* __restrict__ pos,
                           int32_t* __restrict__ list) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        if (flag[v]) list[pos[v]] = (int32_t)v;
}

// Layer profile, large vertices (more than kProfWarpT positions): one block per vertex. Up to
// kProfBuf members are bucket-sorted on chip; larger neighbourhoods are first split into id
// chunks through a global scratch area, and each chunk is bucket-sorted on chip in id order.
__global__ void __launch_bounds__(kProfThreads)
k_profile(Incidence I, const int2* __restrict__ v_span, const int32_t* __restrict__ big_list, int32_t nbig,
          int id_bits, const int32_t* __restrict__ tsum,
          uint2* __restrict__ pairs, uint32_t* __restrict__ nlayers, uint32_t* __restrict__ deg,
          int* __restrict__ next_vertex, ProfScratch S, DevStatus* st,
          unsigned long long* __restrict__ maxima /* [max_l, max_deg, max_layer_n] */) {
    extern __shared__ uint32_t smem[];
    uint32_t* buf = smem;                                  // kProfBuf
    uint32_t* hist_s = buf + kProfBuf;                     // kProfHist
    int* bucket_cnt = (int*)(hist_s + kProfHist);          // kBucketsMax (first-level chunks)
    int* bkt = bucket_cnt + kBucketsMax;                   // kBucketsMax (on-chip sort)
    int* pre = bkt + kBucketsMax;                          // 2 kProfThreads + 1
    int* ctrl = pre + 2 * kProfThreads + 1;                // control block: [0] ticket, [8, 8 + warps)
                                                           // per-warp maxima, [32, 32 + warps) sort scratch
    using Gr = Group<kProfThreads>;
    uint32_t* big = S.big + (int64_t)blockIdx.x * S.big_cap;
    uint32_t* hist_g = S.hist + (int64_t)blockIdx.x * S.hist_cap;

    for (;;) {
        if (threadIdx.x == 0) ctrl[0] = atomicAdd(next_vertex, 1);
        __syncthreads();
        const int bi = ctrl[0];
        __syncthreads();
        if (bi >= nbig) break;
        const int32_t mu = big_list[bi];
        const int32_t e0 = I.v_off[mu], dh = I.v_off[mu + 1] - e0;
        // histogram of multiplicities, indexed by w in [1, dh]
        uint32_t* hist = dh < kProfHist ? hist_s : hist_g;
        if (dh >= kProfHist && (int64_t)dh + 1 > S.hist_cap) {
            if (threadIdx.x == 0) dev_fail(st, kErrCapacity, mu);
            continue;
        }
        for (int w = threadIdx.x; w <= dh; w += kProfThreads) hist[w] = 0;
        __syncthreads();
        auto count_runs = [&](bool start, uint32_t, int mult) -> bool {
            if (start) atomicAdd(&hist[mult], 1u);
            return false;
        };
        const int T = tsum[mu] - dh;  // members other than mu
        if (T <= kProfBuf) {
            const int got = sorted_nbhd<kProfThreads>(v_span, I.he_mem, mu, e0, dh, T, id_bits, buf, bkt, 12,
                                                      pre, ctrl + 32);
            walk_runs<kProfThreads>(buf, got, count_runs);
        } else {
            // bucket the members by their top id bits so each bucket fits on chip
            if ((int64_t)T > S.big_cap) {
                if (threadIdx.x == 0) dev_fail(st, kErrCapacity, mu);
                continue;
            }
            int b = 0;
            while ((int64_t)(kProfBuf / 4) << b < (int64_t)T && b < id_bits && (1 << (b + 1)) <= kBucketsMax) ++b;
            bool ok = false;
            for (;;) {
                const int nb = 1 << b;
                const int shift = id_bits - b;
                for (int i = threadIdx.x; i < nb; i += kProfThreads) bucket_cnt[i] = 0;
                __syncthreads();
                for_each_member<kProfThreads>(v_span, I.he_mem, mu, e0, dh, pre,
                                              [&](uint32_t x) { atomicAdd(&bucket_cnt[x >> shift], 1); });
                int mx = 0;
                for (int i = threadIdx.x; i < nb; i += kProfThreads) mx = max(mx, bucket_cnt[i]);
                const int bmax = __reduce_max_sync(0xFFFFFFFFu, mx);
                if ((threadIdx.x & 31) == 0) ctrl[8 + (threadIdx.x >> 5)] = bmax;
                __syncthreads();
                int all_max = 0;
                for (int w = 0; w < kProfThreads / 32; ++w) all_max = max(all_max, ctrl[8 + w]);
                __syncthreads();
                if (all_max <= kProfBuf) { ok = true; break; }
                if (b >= id_bits || (1 << (b + 1)) > kBucketsMax) break;
                ++b;
            }
            if (!ok) {
                if (threadIdx.x == 0) dev_fail(st, kErrBucket, mu);
                __syncthreads();
                continue;
            }
            const int nb = 1 << b;
            const int shift = id_bits - b;
            // exclusive scan of bucket counts (single warp, nb <= 4096)
            if (threadIdx.x < 32) {
                int carry = 0;
                for (int base = 0; base < nb; base += 32) {
                    const int i = base + threadIdx.x;
                    const int v = i < nb ? bucket_cnt[i] : 0;
                    int inc = v;
                    for (int o = 1; o < 32; o <<= 1) {
                        const int t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                        if ((int)threadIdx.x >= o) inc += t;
                    }
                    if (i < nb) bucket_cnt[i] = carry + inc - v;
                    carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
                }
            }
            __syncthreads();
            // scatter into the global bucket area; bucket_cnt becomes the running end
            for_each_member<kProfThreads>(v_span, I.he_mem, mu, e0, dh, pre,
                                          [&](uint32_t x) { big[atomicAdd(&bucket_cnt[x >> shift], 1)] = x; });
            __threadfence_block();
            __syncthreads();
            int begin = 0;
            for (int q = 0; q < nb; ++q) {
                const int end = bucket_cnt[q];
                const int cnt = end - begin;
                if (cnt > 0) {
                    sort_chunk<kProfThreads>(big + begin, cnt, shift, buf, bkt, 12, ctrl + 32);
                    walk_runs<kProfThreads>(buf, cnt, count_runs);
                    __syncthreads();
                }
                begin = end;
            }
        }
        __syncthreads();
        if (threadIdx.x < 32) emit_layers(hist, dh, mu, e0, pairs, nlayers, deg, maxima);
        __syncthreads();
    }
}

// ---- layer profile: pass 2 (thresholds, inversion kind, CDF table lengths) ------------------
// Entry [0] = {w_i | p = 1 flag, n_i, floor(p 2^32), T_0}; entry [1] = {table offset, table
// length, Poisson parts c, kind}; kind 0: no draw (p = 0 or 1), 1: Binomial (n_i <= 20), 2:
// Poisson with c parts of lambda / c each (Sec. 3.1.3). The table and T_0 are filled by pass 3.
__global__ void k_profile_write(int32_t n, const int32_t* __restrict__ v_off,
                                const uint2* __restrict__ pairs, const int64_t* __restrict__ poff64,
                                const uint32_t* __restrict__ deg, int32_t model, uint64_t uthr,
                                const double* __restrict__ ln_l1, uint4* __restrict__ prof,
                                uint32_t* __restrict__ tab_len, int32_t* __restrict__ prof_off,
                                uint8_t* __restrict__ stratum) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pb = poff64[v];
        const int l = (int)(poff64[v + 1] - pb);
        prof_off[v] = (int32_t)pb;
        if (v == n - 1) prof_off[n] = (int32_t)poff64[n];
        stratum[v] = (uint8_t)(l < HYPERIM_NSTRATA - 1 ? l : HYPERIM_NSTRATA - 1);
        const uint32_t dg = deg[v];
        for (int i = 0; i < l; ++i) {
            const uint2 wn = pairs[v_off[v] + i];
            const uint32_t n_i = wn.y;
            uint64_t thr;
            if (model == HYPERIM_P_UNIFORM_PAIR) {
                thr = uthr;
            } else if (model == HYPERIM_P_WC) {
                thr = dg <= 1 ? kPOne : (kPOne / (uint64_t)dg);
            } else {
                // P(L_i) = 1/(i ln(l+1)) (Sec. 3.1.1); per member P(L_i)/n_i, clamped to 1
                const double PL = __ddiv_rn(1.0, __dmul_rn((double)(i + 1), ln_l1[l]));
                const double pd = __ddiv_rn(PL, (double)n_i);
                thr = pd >= 1.0 ? kPOne : __double2ull_rz(__dmul_rn(pd, 4294967296.0));
            }
            uint32_t flags = 0, kind = 0, c = 0, L = 0;
            if (thr >= kPOne) {
                flags = kPOneFlag;
            } else if (thr > 0) {
                if (n_i <= 20) {
                    kind = 1;
                    c = 1;
                    L = cdf_table(n_i, thr, false, 0.0, kTableCap, nullptr);
                } else {
                    kind = 2;
                    const double lam = poisson_lambda(n_i, thr);
                    c = poisson_parts(lam);
                    L = cdf_table(n_i, thr, true, poisson_part_lambda(lam, c), kTableCap, nullptr);
                }
            }
            prof[2 * (pb + i)] = make_uint4(wn.x | flags, n_i, thr >= kPOne ? 0u : (uint32_t)thr, 0u);
            prof[2 * (pb + i) + 1] = make_uint4(0u, L, c, kind);
            tab_len[pb + i] = L;
        }
    }
}

// ---- layer profile: pass 3 (CDF threshold tables) -----------------------------------------------
__global__ void k_table_fill(int64_t layers, const int64_t* __restrict__ tab_off, uint4* __restrict__ prof,
                             uint32_t* __restrict__ tab) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < layers;
         x += (int64_t)gridDim.x * blockDim.x) {
        uint4 a = prof[2 * x], b = prof[2 * x + 1];
        const uint32_t n_i = a.y, kind = b.w;
        const uint32_t off = (uint32_t)tab_off[x];
        b.x = off;
        if (kind == 1) {
            cdf_table(n_i, a.z, false, 0.0, kTableCap, tab + off);
        } else if (kind == 2) {
            const double lam = poisson_lambda(n_i, a.z);
            cdf_table(n_i, a.z, true, poisson_part_lambda(lam, b.z), kTableCap, tab + off);
        }
        a.w = b.y > 0 ? tab[off] : 0u;  // T_0 beside the entry: the common h = 0 needs no table read
        prof[2 * x] = a;
        prof[2 * x + 1] = b;
    }
}

__global__ void k_stratum_flags(const uint8_t* __restrict__ stratum, int32_t n, int s,
                                uint32_t* __restrict__ flags) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        flags[v] = stratum[v] == s ? 1u : 0u;
}

__global__ void k_stratum_scatter(const uint32_t* __restrict__ flags, const int64_t* __restrict__ pos,
                                  int32_t n, int32_t base, int32_t* __restrict__ vs_list) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        if (flags[v]) vs_list[base + pos[v]] = (int32_t)v;
}

__global__ void k_hist_layers(const int64_t* __restrict__ poff64, int32_t n,
                              unsigned long long* __restrict__ hist, int hmax) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = poff64[v + 1] - poff64[v];
        atomicAdd(&hist[l < hmax ? l : hmax], 1ull);
    }
}

__global__ void k_max_i32(const int32_t* __restrict__ a, int64_t n, unsigned long long* out) {
    unsigned long long mx = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        mx = max(mx, (unsigned long long)a[i]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

__global__ void k_vhe_len(const int64_t* __restrict__ v_off64, int32_t n, int32_t* __restrict__ dh) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        dh[v] = (int32_t)(v_off64[v + 1] - v_off64[v]);
}

// per-incidence spans and per-vertex records read by the RR kernel (fewer dependent loads)
__global__ void k_build_spans(const int32_t* __restrict__ v_he, int64_t nnz,
                              const int32_t* __restrict__ he_off, int2* __restrict__ v_span) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < nnz;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t he = v_he[x];
        v_span[x] = make_int2(he_off[he], he_off[he + 1] - he_off[he]);
    }
}

// 32-byte sectors of the method's data that a materialising pop of v touches (the work counter
// behind the pool view's `sectors`): the ids of v_he(v) and of mem(he) for every hyperedge he
// containing v, 4-byte ids at their offsets in the normalised incidence store. One warp per vertex.
__device__ __forceinline__ uint32_t span_sectors(uint64_t a, uint64_t len) {
    return len == 0 ? 0u : (uint32_t)(((a + len - 1) >> 5) - (a >> 5) + 1);
}

__global__ void k_mat_sect(int32_t n, const int32_t* __restrict__ v_off, const int2* __restrict__ v_span,
                           uint32_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < n;
         v += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t b = v_off[v], e = v_off[v + 1];
        uint32_t acc = 0;
        for (int32_t x = b + lane; x < e; x += 32) {
            const int2 sp = v_span[x];
            acc += span_sectors(4ull * (uint64_t)sp.x, 4ull * (uint64_t)sp.y);
        }
        acc = __reduce_add_sync(0xFFFFFFFFu, acc);
        if (lane == 0) out[v] = acc + span_sectors(4ull * (uint64_t)b, 4ull * (uint64_t)(e - b));
    }
}

// directory bits of a hyperedge of L members (0: no directory)
__device__ __forceinline__ uint32_t dir_bits(int32_t L, int id_bits) {
    if (L <= kDirMinLen || L > kDirMaxLen) return 0;
    uint32_t b = 1;
    while ((1 << b) < L) ++b;
    const uint32_t cap = (uint32_t)min(id_bits, kDirMaxBits);
    return b < cap ? b : cap;
}

__global__ void k_dir_size(const int32_t* __restrict__ he_off, int32_t m, int id_bits, uint32_t* __restrict__ size) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = dir_bits(he_off[e + 1] - he_off[e], id_bits);
        size[e] = b ? (1u << b) + 1u : 0u;
    }
}

// one warp per hyperedge: member x (top b bits t_x) sets D[r] = x for t_{x-1} < r <= t_x; the
// entries above the last member's bits hold L
__global__ void k_dir_fill(const int32_t* __restrict__ he_off, const int32_t* __restrict__ he_mem, int32_t m,
                           int id_bits, const int64_t* __restrict__ dir_off, uint16_t* __restrict__ dir) {
    const int lane = threadIdx.x & 31;
    for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < m;
         e += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t b0 = he_off[e], L = he_off[e + 1] - b0;
        const uint32_t b = dir_bits(L, id_bits);
        if (!b) continue;
        const int sh = id_bits - (int)b;
        uint16_t* D = dir + dir_off[e];
        for (int32_t x = lane; x <= L; x += 32) {
            const int64_t t = x < L ? (int64_t)((uint32_t)he_mem[b0 + x] >> sh) : (int64_t)(1u << b);
            const int64_t tp = x > 0 ? (int64_t)((uint32_t)he_mem[b0 + x - 1] >> sh) : -1;
            for (int64_t r = tp + 1; r <= t; ++r) D[r] = (uint16_t)x;
        }
    }
}

// per incidence (v_he order): {offset of its hyperedge's directory, bits} or {0, 0}
__global__ void k_dir_incidence(const int32_t* __restrict__ v_he, int64_t nnz, const int32_t* __restrict__ he_off,
                                int id_bits, const int64_t* __restrict__ dir_off, uint2* __restrict__ v_dir) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < nnz; x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = v_he[x];
        const uint32_t b = dir_bits(he_off[e + 1] - he_off[e], id_bits);
        v_dir[x] = b ? make_uint2((uint32_t)dir_off[e], b) : make_uint2(0u, 0u);
    }
}

__global__ void k_build_vinfo(int32_t n, const int32_t* __restrict__ prof_off,
                              const int32_t* __restrict__ v_off, int4* __restrict__ vinfo) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        vinfo[v] = make_int4(prof_off[v], prof_off[v + 1] - prof_off[v], v_off[v], v_off[v + 1] - v_off[v]);
}

int grid_for(int64_t items, int threads, int sm) {
    int64_t b = (items + threads - 1) / threads;
    int64_t cap = (int64_t)sm * 32;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

}  // namespace

hyperim_status size_order(hyperim_graph* g, const int32_t* list, int64_t count, bool emit_index, int32_t* out) {
    if (count <= 0) return HYPERIM_OK;
    cudaStream_t s = g->stream;
    hyperim_status st;
    CallBuffers tmp(g);
    unsigned int* hist = nullptr;
    if ((st = tmp.alloc(&hist, sizeof(unsigned int) * kSizeBuckets))) return st;
    HYP_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned int) * kSizeBuckets, s));
    const int grid = grid_for(count, 256, g->sm_count);
    { k_size_hist<<<grid, 256, 0, s>>>(list, count, g->tsum, hist); count_launch(); }
    { k_size_starts<<<1, 1, 0, s>>>(hist); count_launch(); }
    { k_size_scatter<<<grid, 256, 0, s>>>(list, count, g->tsum, hist, emit_index ? 1 : 0, out); count_launch(); }
    HYP_CUDA(cudaGetLastError());
    return HYPERIM_OK;
}

hyperim_status build_graph(hyperim_graph* g, const int32_t* he_off_in, const int32_t* he_mem_in,
                           int32_t nnz_in, bool on_device) {
    cudaStream_t s = g->stream;
    const int32_t n = g->n, m = g->m;
    const int sm = g->sm_count;
    hyperim_status st;
    CallBuffers tmp(g);
    // --- upload
    int32_t *d_off_in = nullptr, *d_mem_in = nullptr, *d_tmp = nullptr;
    const size_t nnz_alloc = (size_t)(nnz_in > 0 ? nnz_in : 1);
    if ((st = tmp.alloc(&d_off_in, sizeof(int32_t) * ((size_t)m + 1)))) return st;
    if ((st = tmp.alloc(&d_mem_in, sizeof(int32_t) * nnz_alloc))) return st;
    if ((st = tmp.alloc(&d_tmp, sizeof(int32_t) * nnz_alloc))) return st;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    HYP_CUDA(cudaMemcpyAsync(d_off_in, he_off_in, sizeof(int32_t) * ((size_t)m + 1), kind, s));
    if (nnz_in > 0)
        HYP_CUDA(cudaMemcpyAsync(d_mem_in, he_mem_in, sizeof(int32_t) * (size_t)nnz_in, kind, s));
    if (m > 0) { k_check_offsets<<<grid_for(m, 256, sm), 256, 0, s>>>(d_off_in, m, g->d_status); count_launch(); }
    if ((st = check_device_status(g, "hyperedge offsets"))) return st;

    // --- normalise hyperedges
    uint32_t* d_newsize = nullptr;
    int64_t* d_off_new = nullptr;
    if ((st = tmp.alloc(&d_newsize, sizeof(uint32_t) * ((size_t)m + 1)))) return st;
    if ((st = tmp.alloc(&d_off_new, sizeof(int64_t) * ((size_t)m + 1)))) return st;
    uint8_t* d_first = nullptr;
    if ((st = tmp.alloc(&d_first, nnz_alloc))) return st;
    if (m > 0)
        { k_normalise<<<grid_for((int64_t)m * 32, 256, sm), 256, 0, s>>>(d_off_in, d_mem_in, m, n,
                                                                       d_tmp, d_first, d_newsize,
                                                                       g->d_status); count_launch(); }
    if ((st = check_device_status(g, "hyperedge members"))) return st;
    if ((st = exclusive_scan_u32_to_i64(g, d_newsize, d_off_new, m))) return st;
    int64_t nnz = 0;
    HYP_CUDA(cudaMemcpyAsync(&nnz, d_off_new + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    g->nnz = nnz;
    const size_t nnz_a = (size_t)(nnz > 0 ? nnz : 1);
    if ((st = dev_alloc(g, (void**)&g->he_off, sizeof(int32_t) * ((size_t)m + 1)))) return st;
    if ((st = dev_alloc(g, (void**)&g->he_mem, sizeof(int32_t) * nnz_a))) return st;
    if (m > 0)
        { k_compact_he<<<grid_for((int64_t)m * 32, 256, sm), 256, 0, s>>>(d_off_in, d_tmp, d_off_new,
                                                                        m, g->he_off, g->he_mem); count_launch(); }
    else
        HYP_CUDA(cudaMemsetAsync(g->he_off, 0, sizeof(int32_t), s));

    // --- vertex -> hyperedge lists
    uint32_t* d_cnt = nullptr;
    int64_t* d_voff64 = nullptr;
    if ((st = tmp.alloc(&d_cnt, sizeof(uint32_t) * ((size_t)n + 1)))) return st;
    if ((st = tmp.alloc(&d_voff64, sizeof(int64_t) * ((size_t)n + 1)))) return st;
    if ((st = dev_alloc(g, (void**)&g->v_off, sizeof(int32_t) * ((size_t)n + 1)))) return st;
    if ((st = dev_alloc(g, (void**)&g->v_he, sizeof(int32_t) * nnz_a))) return st;
    if ((st = dev_alloc(g, (void**)&g->tsum, sizeof(int32_t) * (size_t)n))) return st;
    HYP_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(uint32_t) * ((size_t)n + 1), s));
    HYP_CUDA(cudaMemsetAsync(g->tsum, 0, sizeof(int32_t) * (size_t)n, s));
    if (nnz > 0) { k_count_dh<<<grid_for(nnz, 256, sm), 256, 0, s>>>(g->he_mem, nnz, d_cnt); count_launch(); }
    if ((st = exclusive_scan_u32_to_i64(g, d_cnt, d_voff64, n))) return st;
    HYP_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(uint32_t) * ((size_t)n + 1), s));
    if (m > 0)
        { k_scatter_vhe<<<grid_for((int64_t)m * 32, 256, sm), 256, 0, s>>>(
            g->he_off, g->he_mem, m, d_voff64, d_cnt, d_tmp, g->tsum); count_launch(); }
    { k_sort_vhe<<<grid_for((int64_t)n * 32, 256, sm), 256, 0, s>>>(d_voff64, n, d_tmp, g->v_he,
                                                                   g->v_off); count_launch(); }

    // --- maxima of d_H and T
    unsigned long long* d_max = nullptr;
    if ((st = tmp.alloc(&d_max, sizeof(unsigned long long) * 8))) return st;
    HYP_CUDA(cudaMemsetAsync(d_max, 0, sizeof(unsigned long long) * 8, s));
    int32_t* d_dh = (int32_t*)d_cnt;  // reuse
    { k_vhe_len<<<grid_for(n, 256, sm), 256, 0, s>>>(d_voff64, n, d_dh); count_launch(); }
    { k_max_i32<<<grid_for(n, 256, sm), 256, 0, s>>>(d_dh, n, d_max + 3); count_launch(); }
    { k_max_i32<<<grid_for(n, 256, sm), 256, 0, s>>>(g->tsum, n, d_max + 4); count_launch(); }
    unsigned long long hmax[8];
    HYP_CUDA(cudaMemcpyAsync(hmax, d_max, sizeof(hmax), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    g->max_dh = (int32_t)hmax[3];
    g->max_tsum = (int64_t)hmax[4];

    // --- layer profile pass 1
    uint2* d_pairs = nullptr;
    uint32_t *d_nl = nullptr, *d_deg = nullptr;
    int* d_next = nullptr;
    if ((st = tmp.alloc(&d_pairs, sizeof(uint2) * nnz_a))) return st;
    if ((st = tmp.alloc(&d_nl, sizeof(uint32_t) * ((size_t)n + 1)))) return st;
    if ((st = dev_alloc(g, (void**)&g->deg, sizeof(int32_t) * (size_t)n))) return st;
    d_deg = (uint32_t*)g->deg;
    if ((st = tmp.alloc(&d_next, sizeof(int)))) return st;
    HYP_CUDA(cudaMemsetAsync(d_next, 0, sizeof(int), s));
    // per-incidence spans first: both profile kernels gather through them
    if ((st = dev_alloc(g, (void**)&g->v_span, sizeof(int2) * nnz_a))) return st;
    if (nnz > 0)
        { k_build_spans<<<grid_for(nnz, 256, sm), 256, 0, s>>>(g->v_he, nnz, g->he_off, g->v_span); count_launch(); }
    { k_profile_warp<kProfWarpT, kPWWarps><<<grid_for((int64_t)n * 32, kPWThreads, sm), kPWThreads, 0, s>>>(
        n, nullptr, g->v_off, g->v_span, g->he_mem, g->tsum, g->id_bits, d_pairs, d_nl, d_deg, d_max); count_launch(); }
    const size_t prof_smem = sizeof(uint32_t) * (kProfBuf + kProfHist) +
                             sizeof(int) * (2 * kBucketsMax + 2 * kProfThreads + 1 + 64);
    HYP_CUDA(cudaFuncSetAttribute(k_profile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)prof_smem));
    int per_sm = 0;
    HYP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_profile, kProfThreads,
                                                           prof_smem));
    if (per_sm < 1) per_sm = 1;
    ProfScratch PS;
    PS.big_cap = g->max_tsum > kProfBuf ? g->max_tsum : 1;
    int pblocks = sm * per_sm;
    // keep the bucketing scratch area within 2 GiB
    while (pblocks > sm && (int64_t)pblocks * PS.big_cap * 4 > ((int64_t)2 << 30)) pblocks -= sm;
    PS.hist_cap = g->max_dh >= kProfHist ? (int64_t)g->max_dh + 1 : 1;
    if ((st = tmp.alloc(&PS.big, sizeof(uint32_t) * (size_t)PS.big_cap * pblocks)))
        return st;
    if ((st = tmp.alloc(&PS.hist, sizeof(uint32_t) * (size_t)PS.hist_cap * pblocks)))
        return st;
    Incidence I{g->he_off, g->he_mem, g->v_off, g->v_he};
    // the large vertices, listed
    uint32_t* d_bflag = nullptr;
    int64_t* d_bpos = nullptr;
    int32_t* d_blist = nullptr;
    if ((st = tmp.alloc(&d_bflag, sizeof(uint32_t) * (size_t)(n > 0 ? n : 1)))) return st;
    if ((st = tmp.alloc(&d_bpos, sizeof(int64_t) * ((size_t)n + 1)))) return st;
    // mid-size vertices (kProfWarpT < positions <= kProfMidT): one warp each, listed
    if (n > 0 && g->max_tsum > kProfWarpT) {
        { k_big_flags<<<grid_for(n, 256, sm), 256, 0, s>>>(n, g->v_off, g->tsum, kProfWarpT, kProfMidT, d_bflag); count_launch(); }
        if ((st = exclusive_scan_u32_to_i64(g, d_bflag, d_bpos, n))) return st;
        int64_t nmid = 0;
        HYP_CUDA(cudaMemcpyAsync(&nmid, d_bpos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HYP_CUDA(cudaStreamSynchronize(s));
        if (nmid > 0) {
            int32_t* d_mlist = nullptr;
            if ((st = tmp.alloc(&d_mlist, sizeof(int32_t) * (size_t)nmid))) return st;
            { k_big_list<<<grid_for(n, 256, sm), 256, 0, s>>>(n, d_bflag, d_bpos, d_mlist); count_launch(); }
            { k_profile_warp<kProfMidT, kPMWarps><<<grid_for(nmid * 32, kPMWarps * 32, sm), kPMWarps * 32, 0, s>>>(
                (int32_t)nmid, d_mlist, g->v_off, g->v_span, g->he_mem, g->tsum, g->id_bits, d_pairs, d_nl, d_deg,
                d_max); count_launch(); }
        }
    }
    if (n > 0) { k_big_flags<<<grid_for(n, 256, sm), 256, 0, s>>>(n, g->v_off, g->tsum, kProfMidT, 0x7FFFFFFF, d_bflag); count_launch(); }
    if ((st = exclusive_scan_u32_to_i64(g, d_bflag, d_bpos, n))) return st;
    int64_t nbig = 0;
    HYP_CUDA(cudaMemcpyAsync(&nbig, d_bpos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    if ((st = tmp.alloc(&d_blist, sizeof(int32_t) * (size_t)(nbig > 0 ? nbig : 1)))) return st;
    if (nbig > 0) {
        { k_big_list<<<grid_for(n, 256, sm), 256, 0, s>>>(n, d_bflag, d_bpos, d_blist); count_launch(); }
        // largest first (into the flag array, no longer needed: n >= nbig words)
        int32_t* d_border = reinterpret_cast<int32_t*>(d_bflag);
        if ((st = size_order(g, d_blist, nbig, false, d_border))) return st;
        { k_profile<<<(int)std::min<int64_t>(pblocks, nbig), kProfThreads, prof_smem, s>>>(
            I, g->v_span, d_border, (int32_t)nbig, g->id_bits, g->tsum, d_pairs, d_nl, d_deg, d_next, PS,
            g->d_status, d_max); count_launch(); }
    }
    if ((st = check_device_status(g, "layer profile"))) return st;
    HYP_CUDA(cudaMemcpyAsync(hmax, d_max, sizeof(hmax), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    g->max_layers = (int32_t)hmax[0];
    g->max_deg = (int64_t)hmax[1];
    g->max_layer_n = (int64_t)hmax[2];

    // --- profile offsets + pass 2
    int64_t* d_poff64 = nullptr;
    if ((st = tmp.alloc(&d_poff64, sizeof(int64_t) * ((size_t)n + 1)))) return st;
    if ((st = exclusive_scan_u32_to_i64(g, d_nl, d_poff64, n))) return st;
    int64_t L = 0;
    HYP_CUDA(cudaMemcpyAsync(&L, d_poff64 + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    g->profile_entries = L;
    if ((st = dev_alloc(g, (void**)&g->prof, 2 * sizeof(uint4) * (size_t)(L > 0 ? L : 1)))) return st;
    if ((st = dev_alloc(g, (void**)&g->prof_off, sizeof(int32_t) * ((size_t)n + 1)))) return st;
    if ((st = dev_alloc(g, (void**)&g->stratum, (size_t)n))) return st;
    // ln(l + 1) for the paper's layer probabilities, computed once on the host
    std::vector<double> ln_l1((size_t)g->max_layers + 2);
    for (size_t l = 0; l < ln_l1.size(); ++l) ln_l1[l] = std::log((double)l + 1.0);
    double* d_ln = nullptr;
    if ((st = tmp.alloc(&d_ln, sizeof(double) * ln_l1.size()))) return st;
    HYP_CUDA(cudaMemcpyAsync(d_ln, ln_l1.data(), sizeof(double) * ln_l1.size(),
                             cudaMemcpyHostToDevice, s));
    uint32_t* d_tlen = nullptr;
    int64_t* d_toff = nullptr;
    const size_t Lalloc = (size_t)(L > 0 ? L : 1);
    if ((st = tmp.alloc(&d_tlen, sizeof(uint32_t) * Lalloc))) return st;
    if ((st = tmp.alloc(&d_toff, sizeof(int64_t) * (Lalloc + 1)))) return st;
    { k_profile_write<<<grid_for(n, 256, sm), 256, 0, s>>>(n, g->v_off, d_pairs, d_poff64, d_deg,
                                                         g->model, g->uniform_thr, d_ln, g->prof,
                                                         d_tlen, g->prof_off, g->stratum); count_launch(); }
    if ((st = exclusive_scan_u32_to_i64(g, d_tlen, d_toff, L))) return st;
    int64_t tab_total = 0;
    HYP_CUDA(cudaMemcpyAsync(&tab_total, d_toff + L, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    if (tab_total >= (int64_t)0xFFFFFFFFll) return set_error(HYPERIM_EOVERFLOW, "CDF tables exceed 2^32 entries");
    g->table_entries = tab_total;
    if ((st = dev_alloc(g, (void**)&g->cdf_tab, sizeof(uint32_t) * (size_t)(tab_total > 0 ? tab_total : 1))))
        return st;
    if (L > 0)
        { k_table_fill<<<grid_for(L, 256, sm), 256, 0, s>>>(L, d_toff, g->prof, g->cdf_tab); count_launch(); }

    // --- theta(l*) from the histogram of l (Thm 2)
    const int hcap = g->max_layers + 1;
    unsigned long long* d_lh = nullptr;
    if ((st = tmp.alloc(&d_lh, sizeof(unsigned long long) * ((size_t)hcap + 1)))) return st;
    HYP_CUDA(cudaMemsetAsync(d_lh, 0, sizeof(unsigned long long) * ((size_t)hcap + 1), s));
    { k_hist_layers<<<grid_for(n, 256, sm), 256, 0, s>>>(d_poff64, n, d_lh, hcap); count_launch(); }
    std::vector<unsigned long long> lh((size_t)hcap + 1);
    HYP_CUDA(cudaMemcpyAsync(lh.data(), d_lh, sizeof(unsigned long long) * lh.size(),
                             cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    double lsum = 0.0;
    for (int l = 1; l < hcap; ++l)
        if (lh[l]) lsum += (double)lh[l] * ((double)l / std::log((double)l + 1.0));
    g->theta_lstar = lsum / (double)n;
    for (int s2 = 0; s2 < HYPERIM_NSTRATA; ++s2) g->stratum_size[s2] = 0;
    for (int l = 0; l < hcap; ++l)
        g->stratum_size[l < HYPERIM_NSTRATA - 1 ? l : HYPERIM_NSTRATA - 1] += (int64_t)lh[l];

    // --- per-vertex records for the RR kernel
    if ((st = dev_alloc(g, (void**)&g->vinfo, sizeof(int4) * (size_t)n))) return st;
    { k_build_vinfo<<<grid_for(n, 256, sm), 256, 0, s>>>(n, g->prof_off, g->v_off, g->vinfo); count_launch(); }
    if ((st = dev_alloc(g, (void**)&g->mat_sect, sizeof(uint32_t) * (size_t)n))) return st;
    { k_mat_sect<<<grid_for((int64_t)n * 32, 256, sm), 256, 0, s>>>(n, g->v_off, g->v_span, g->mat_sect); count_launch(); }

    // --- id directories of the larger hyperedges (read by the chunk path of the RR kernel)
    {
        uint32_t* d_dsize = nullptr;
        int64_t* d_doff = nullptr;
        if ((st = tmp.alloc(&d_dsize, sizeof(uint32_t) * ((size_t)m + 1)))) return st;
        if ((st = tmp.alloc(&d_doff, sizeof(int64_t) * ((size_t)m + 1)))) return st;
        if (m > 0) { k_dir_size<<<grid_for(m, 256, sm), 256, 0, s>>>(g->he_off, m, g->id_bits, d_dsize); count_launch(); }
        if ((st = exclusive_scan_u32_to_i64(g, d_dsize, d_doff, m))) return st;
        int64_t dtotal = 0;
        HYP_CUDA(cudaMemcpyAsync(&dtotal, d_doff + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HYP_CUDA(cudaStreamSynchronize(s));
        if (dtotal >= (int64_t)0xFFFFFFFFll) dtotal = 0;  // offsets must fit 32 bits: no directories
        g->dir_entries = dtotal;
        if ((st = dev_alloc(g, (void**)&g->v_dir, sizeof(uint2) * nnz_a))) return st;
        if (dtotal > 0) {
            if ((st = dev_alloc(g, (void**)&g->he_dir, sizeof(uint16_t) * (size_t)dtotal))) return st;
            { k_dir_fill<<<grid_for((int64_t)m * 32, 256, sm), 256, 0, s>>>(g->he_off, g->he_mem, m, g->id_bits, d_doff,
                                                                         g->he_dir); count_launch(); }
            if (nnz > 0)
                { k_dir_incidence<<<grid_for(nnz, 256, sm), 256, 0, s>>>(g->v_he, nnz, g->he_off, g->id_bits, d_doff,
                                                                       g->v_dir); count_launch(); }
        } else {
            HYP_CUDA(cudaMemsetAsync(g->v_dir, 0, sizeof(uint2) * nnz_a, s));
        }
    }
    if ((st = build_chunk_index(g))) return st;

    // --- strata lists V_s (ascending ids)
    if ((st = dev_alloc(g, (void**)&g->vs_off, sizeof(int32_t) * (HYPERIM_NSTRATA + 1)))) return st;
    if ((st = dev_alloc(g, (void**)&g->vs_list, sizeof(int32_t) * (size_t)n))) return st;
    int32_t hvs[HYPERIM_NSTRATA + 1];
    hvs[0] = 0;
    for (int s2 = 0; s2 < HYPERIM_NSTRATA; ++s2) hvs[s2 + 1] = hvs[s2] + (int32_t)g->stratum_size[s2];
    HYP_CUDA(cudaMemcpyAsync(g->vs_off, hvs, sizeof(hvs), cudaMemcpyHostToDevice, s));
    uint32_t* d_flags = d_cnt;
    for (int s2 = 0; s2 < HYPERIM_NSTRATA; ++s2) {
        if (g->stratum_size[s2] == 0) continue;
        { k_stratum_flags<<<grid_for(n, 256, sm), 256, 0, s>>>(g->stratum, n, s2, d_flags); count_launch(); }
        if ((st = exclusive_scan_u32_to_i64(g, d_flags, d_voff64, n))) return st;
        { k_stratum_scatter<<<grid_for(n, 256, sm), 256, 0, s>>>(d_flags, d_voff64, n, hvs[s2],
                                                               g->vs_list); count_launch(); }
    }
    HYP_CUDA(cudaGetLastError());
    if ((st = check_device_status(g, "profile write"))) return st;
    HYP_CUDA(cudaStreamSynchronize(s));
    return check_device_status(g, "load");
}

}  // namespace hyperim
