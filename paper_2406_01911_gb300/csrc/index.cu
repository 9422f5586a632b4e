// Chunk index of large neighbourhoods (a lookup structure over the layers of Sec. 3.1.1).
//
// A pick of Algorithm 3 is "the a-th member of layer L_i of A(mu) in id order". For a vertex
// whose hyperedges hold thousands of members, materialising all of A(mu) to find a handful of
// picks is most of the RR kernel's work. The index splits the id space into C = 2^c chunks (top
// c id bits) and stores, per layer and chunk, how many members of the layer lie in the earlier
// chunks. A pick's position then names its chunk, and the RR kernel reads only that id range of
// mu's hyperedges (each hyperedge's members are sorted, so the range is found by binary search).
// The index holds counts only (l x C words per indexed vertex), never neighbour lists.
//
// Build (after the layer profile):
//   k_idx_candidates  vertices with d_H >= 2, more than kIdxMinT members besides mu, l <= kIdxMaxL
//   k_idx_plan        per candidate: the expected picks per pop decide the chunk target (or
//                     no index); histogram of the members over 2^hb id bins (hb = min(12, id
//                     bits)); c = the fewest bits for which no chunk holds more than the target
//                     (0 bits: not indexed); entries = l 2^c
//   scan              table offsets
//   k_idx_fill        per indexed vertex: members sorted by id on chip (bucketed through a global
//                     scratch area when large), runs (multiplicity w -> layer) counted per
//                     (layer, chunk); each layer row becomes an exclusive prefix
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "mat.cuh"

namespace hyperim {
namespace {

constexpr int kThreads = 256;
constexpr int kBins = 1 << kIdxMaxBits;

__device__ __forceinline__ void dev_fail(DevStatus* st, int32_t code, int32_t detail) {
    if (atomicCAS(&st->code, 0, code) == 0) st->detail = detail;
}

__global__ void k_idx_candidates(int32_t n, const int4* __restrict__ vinfo, const int32_t* __restrict__ tsum,
                                 uint32_t* __restrict__ flag) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int4 vi = vinfo[v];
        const int T = tsum[v] - vi.w;
        flag[v] = (vi.w >= 2 && T > kIdxMinT && vi.y >= 1 && vi.y <= kIdxMaxL) ? 1u : 0u;
    }
}

__global__ void k_idx_list(int32_t n, const uint32_t* __restrict__ flag, const int64_t* __restrict__ pos,
                           int32_t* __restrict__ list) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        if (flag[v]) list[pos[v]] = (int32_t)v;
}

// exclusive scan of a[0, count) in place by warp 0 (count <= kBins); returns nothing, callers sync
__device__ void warp0_exclusive_scan(int* a, int count) {
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    int carry = 0;
    for (int base = 0; base < count; base += 32) {
        const int i = base + lane;
        const int v = i < count ? a[i] : 0;
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o) inc += t;
        }
        if (i < count) a[i] = carry + inc - v;
        carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
}

__global__ void __launch_bounds__(kThreads)
k_idx_plan(const int32_t* __restrict__ list, int32_t nlist, const int32_t* __restrict__ order,
           int* __restrict__ next, const int4* __restrict__ vinfo,
           const int2* __restrict__ v_span, const int32_t* __restrict__ he_mem,
           const int32_t* __restrict__ tsum, const uint4* __restrict__ prof, int id_bits,
           uint8_t* __restrict__ bits_out, uint32_t* __restrict__ entries) {
    __shared__ int hist_a[kBins];
    __shared__ int hist_b[kBins / 2];
    __shared__ int pre[2 * kThreads + 1];
    __shared__ int wmax[kThreads / 32];
    __shared__ int target_s, ticket_s;
    const int hb = id_bits < kIdxMaxBits ? id_bits : kIdxMaxBits;
    const int shift = id_bits - hb;
    for (;;) {
        // candidates largest first, from a counter
        if (threadIdx.x == 0) ticket_s = atomicAdd(next, 1);
        __syncthreads();
        const int ticket = ticket_s;
        __syncthreads();
        if (ticket >= nlist) break;
        const int i = order[ticket];
        const int32_t mu = list[i];
        const int4 vi = vinfo[mu];
        if (threadIdx.x == 0) {
            // expected picks per pop, sum_i n_i p_i, against kIdxFewPicks on the integers
            // n_i floor(p_i 2^32) (p = 1 counts 2^32), stopping once the bound is reached
            const unsigned long long cap = kIdxFewPicks << 32;
            unsigned long long acc = 0;
            for (int q = 0; q < vi.y && acc < cap; ++q) {
                const uint4 e = prof[2 * ((int64_t)vi.x + q)];
                const unsigned long long t = (e.x & kPOneFlag) ? (1ull << 32) : (unsigned long long)e.z;
                acc += (unsigned long long)e.y * t;
            }
            const bool few = acc < cap;
            const int T = tsum[mu] - vi.w;
            target_s = few ? kIdxTargetFew : (T > kIdxMinTMany ? kIdxTargetMany : 0);
        }
        __syncthreads();
        const int target = target_s;
        __syncthreads();
        if (target == 0) {  // many picks on a neighbourhood one warp sorts whole: no index
            if (threadIdx.x == 0) {
                bits_out[i] = 0;
                entries[i] = 0;
            }
            continue;
        }
        for (int b = threadIdx.x; b < (1 << hb); b += kThreads) hist_a[b] = 0;
        __syncthreads();
        for_each_member<kThreads>(v_span, he_mem, mu, vi.z, vi.w, pre,
                                  [&](uint32_t x) { atomicAdd(&hist_a[x >> shift], 1); });
        __syncthreads();
        int* hist = hist_a;
        int* half = hist_b;
        // level c = hb down to 1: the largest chunk at c bits; pairs are merged for c - 1
        int best = 0;
        for (int c = hb; c >= 1; --c) {
            const int nb = 1 << c;
            int mx = 0;
            for (int b = threadIdx.x; b < nb; b += kThreads) mx = max(mx, hist[b]);
            mx = __reduce_max_sync(0xFFFFFFFFu, mx);
            if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
            __syncthreads();
            int all = 0;
            for (int w = 0; w < kThreads / 32; ++w) all = max(all, wmax[w]);
            if (all <= target) best = c;  // uniform: every thread saw the same maxima
            for (int b = threadIdx.x; b < nb / 2; b += kThreads) half[b] = hist[2 * b] + hist[2 * b + 1];
            __syncthreads();
            int* tmp = hist;
            hist = half;
            half = tmp;
        }
        if (threadIdx.x == 0) {
            bits_out[i] = (uint8_t)best;
            entries[i] = best ? (uint32_t)vi.y << best : 0u;
        }
        __syncthreads();
    }
}

__global__ void k_idx_word(const int32_t* __restrict__ list, int32_t nlist, const uint8_t* __restrict__ bits,
                           const uint32_t* __restrict__ entries, const int64_t* __restrict__ off,
                           uint64_t* __restrict__ idx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlist;
         i += (int64_t)gridDim.x * blockDim.x)
        if (entries[i]) idx[list[i]] = ((uint64_t)bits[i] << kIdxBitsShift) | (uint64_t)off[i];
}

// Per indexed vertex (one block, vertices taken from a shared counter): the members of mu's
// hyperedges in ascending id order -- sorted whole on chip when at most kFillBuf of them, else
// bucketed by their top id bits (a bucket is 2^3 whole index chunks, so at most 8 x 1,024
// members) through a global scratch area and sorted bucket by bucket -- are walked run by run:
// each distinct neighbour (multiplicity w -> layer by search in the descending w list) adds one
// to its (layer, chunk) count, kept on chip when the l x 2^c table fits, else in the table
// itself. Every layer row then becomes an exclusive prefix along the chunks, one warp per row.
constexpr int kFillThreads = 512;  // two blocks (32 warps) per SM: the sorts are latency-bound
constexpr int kFillBuf = 8192;  // members sorted on chip at once (power of two)
constexpr int kFillCnt = 4096;  // (layer, chunk) counts kept on chip (more: in the table itself)
constexpr int kFillBkt = kBins;
constexpr int kFillTop = 1 << (kIdxMaxBits - 3);  // top-bit buckets: eight whole chunks each
// the shared memory above fits three 512-thread blocks per SM
constexpr int kFillCtrl = 64;
constexpr size_t kFillSmem = sizeof(uint32_t) * (kFillBuf + kFillCnt + kIdxMaxL) +
                             sizeof(int) * (kFillBkt + kFillTop + 2 * kFillThreads + 1 + kFillCtrl);

__global__ void __launch_bounds__(kFillThreads)
k_idx_fill(const int32_t* __restrict__ list, int32_t nlist, const uint8_t* __restrict__ bits_in,
           const uint32_t* __restrict__ entries, const int64_t* __restrict__ off,
           const int4* __restrict__ vinfo, const int2* __restrict__ v_span,
           const int32_t* __restrict__ he_mem, const int32_t* __restrict__ tsum,
           const uint4* __restrict__ prof, int id_bits, uint32_t* __restrict__ tab,
           uint32_t* __restrict__ scratch, int64_t scratch_cap, const int32_t* __restrict__ order,
           int* __restrict__ next, DevStatus* st) {
    extern __shared__ __align__(16) unsigned char fill_smem[];
    uint32_t* buf = reinterpret_cast<uint32_t*>(fill_smem);             // kFillBuf
    uint32_t* cnt_s = buf + kFillBuf;                                   // kFillCnt
    uint32_t* lw = cnt_s + kFillCnt;                                    // kIdxMaxL
    int* bkt = reinterpret_cast<int*>(lw + kIdxMaxL);                   // kFillBkt (on-chip sorts)
    int* bucket_end = bkt + kFillBkt;                                   // kFillBkt (top-bit buckets)
    int* pre = bucket_end + kFillTop;                                   // 2 kFillThreads + 1
    int* ctrl = pre + 2 * kFillThreads + 1;  // kFillCtrl: [0] ticket, [8, 8 + warps) maxima, [32, 48) sort scratch
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int kWarps = kFillThreads / 32;
    uint32_t* big = scratch + (int64_t)blockIdx.x * scratch_cap;
    for (;;) {
        if (threadIdx.x == 0) ctrl[0] = atomicAdd(next, 1);
        __syncthreads();
        const int ticket = ctrl[0];
        __syncthreads();
        if (ticket >= nlist) break;
        const int i = order[ticket];  // largest first
        if (entries[i] == 0) continue;
        const int32_t mu = list[i];
        const int4 vi = vinfo[mu];
        const int l = vi.y, c = bits_in[i];
        const int C = 1 << c, shift = id_bits - c;
        const int T = tsum[mu] - vi.w;
        uint32_t* t = tab + off[i];
        const int64_t cells = (int64_t)l * C;
        uint32_t* cnt = cells <= kFillCnt ? cnt_s : t;
        for (int q = threadIdx.x; q < l; q += kFillThreads) lw[q] = prof[2 * ((int64_t)vi.x + q)].x & ~kPOneFlag;
        for (int64_t k = threadIdx.x; k < cells; k += kFillThreads) cnt[k] = 0;
        __syncthreads();
        auto count_run = [&](bool start, uint32_t x, int mult) -> bool {
            if (start) {
                int lo = 0, hi = l;  // lw descends: first q with lw[q] <= mult
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (lw[mid] > (uint32_t)mult) lo = mid + 1; else hi = mid;
                }
                if (lo < l && lw[lo] == (uint32_t)mult) atomicAdd(&cnt[(int64_t)lo * C + (x >> shift)], 1u);
                else dev_fail(st, kErrProfile, mu);
            }
            return false;
        };
        if (T <= kFillBuf) {
            const int got = sorted_nbhd<kFillThreads>(v_span, he_mem, mu, vi.z, vi.w, T, id_bits, buf, bkt, 12,
                                                      pre, ctrl + 32);
            walk_runs<kFillThreads>(buf, got, count_run);
        } else {
            if ((int64_t)T > scratch_cap) {
                if (threadIdx.x == 0) dev_fail(st, kErrCapacity, mu);
                __syncthreads();
                continue;
            }
            const int b = c > 3 ? c - 3 : 0;
            const int nb = 1 << b, bshift = id_bits - b;
            for (int q = threadIdx.x; q < nb; q += kFillThreads) bucket_end[q] = 0;
            __syncthreads();
            for_each_member<kFillThreads>(v_span, he_mem, mu, vi.z, vi.w, pre,
                                          [&](uint32_t x) { atomicAdd(&bucket_end[x >> bshift], 1); });
            __syncthreads();
            int mx = 0;
            for (int q = threadIdx.x; q < nb; q += kFillThreads) mx = max(mx, bucket_end[q]);
            mx = __reduce_max_sync(0xFFFFFFFFu, mx);
            if (lane == 0) ctrl[8 + wid] = mx;
            __syncthreads();
            int all = 0;
            for (int w = 0; w < kWarps; ++w) all = max(all, ctrl[8 + w]);
            if (all > kFillBuf) {  // uniform; the plan's chunk bound rules this out
                if (threadIdx.x == 0) dev_fail(st, kErrBucket, mu);
                __syncthreads();
                continue;
            }
            warp0_exclusive_scan(bucket_end, nb);
            __syncthreads();
            for_each_member<kFillThreads>(v_span, he_mem, mu, vi.z, vi.w, pre,
                                          [&](uint32_t x) { big[atomicAdd(&bucket_end[x >> bshift], 1)] = x; });
            __threadfence_block();
            __syncthreads();
            // bucket_end[q] is now the end of bucket q
            int begin = 0;
            for (int q = 0; q < nb; ++q) {
                const int end = bucket_end[q];
                if (end > begin) {
                    sort_chunk<kFillThreads>(big + begin, end - begin, bshift, buf, bkt, 12, ctrl + 32);
                    walk_runs<kFillThreads>(buf, end - begin, count_run);
                    __syncthreads();
                }
                begin = end;
            }
        }
        __syncthreads();
        // counts -> exclusive prefix along the chunks, one warp per layer row
        for (int q = wid; q < l; q += kWarps) {
            const uint32_t* src = cnt + (int64_t)q * C;
            uint32_t* dst = t + (int64_t)q * C;
            uint32_t carry = 0;
            for (int k0 = 0; k0 < C; k0 += 32) {
                const int k = k0 + lane;
                const uint32_t v = k < C ? src[k] : 0u;
                uint32_t inc = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                    if (lane >= o) inc += u;
                }
                if (k < C) dst[k] = carry + inc - v;
                carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
            }
        }
        __syncthreads();
    }
}

int grid_for(int64_t items, int threads, int sm) {
    int64_t b = (items + threads - 1) / threads;
    int64_t cap = (int64_t)sm * 32;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

}  // namespace

hyperim_status build_chunk_index(hyperim_graph* g) {
    cudaStream_t s = g->stream;
    const int32_t n = g->n;
    const int sm = g->sm_count;
    hyperim_status st;
    CallBuffers tmp(g);
    if ((st = dev_alloc(g, (void**)&g->idx, sizeof(uint64_t) * (size_t)(n > 0 ? n : 1)))) return st;
    HYP_CUDA(cudaMemsetAsync(g->idx, 0, sizeof(uint64_t) * (size_t)(n > 0 ? n : 1), s));
    g->idx_entries = 0;
    g->idx_vertices = 0;
    if (n == 0 || g->max_tsum <= kIdxMinT) return HYPERIM_OK;

    uint32_t* d_flag = nullptr;
    int64_t* d_pos = nullptr;
    if ((st = tmp.alloc(&d_flag, sizeof(uint32_t) * (size_t)n))) return st;
    if ((st = tmp.alloc(&d_pos, sizeof(int64_t) * ((size_t)n + 1)))) return st;
    { k_idx_candidates<<<grid_for(n, 256, sm), 256, 0, s>>>(n, g->vinfo, g->tsum, d_flag); count_launch(); }
    if ((st = exclusive_scan_u32_to_i64(g, d_flag, d_pos, n))) return st;
    int64_t ncand = 0;
    HYP_CUDA(cudaMemcpyAsync(&ncand, d_pos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    if (ncand == 0) return HYPERIM_OK;
    int32_t* d_list = nullptr;
    uint8_t* d_bits = nullptr;
    uint32_t* d_entries = nullptr;
    int64_t* d_off = nullptr;
    if ((st = tmp.alloc(&d_list, sizeof(int32_t) * (size_t)ncand))) return st;
    if ((st = tmp.alloc(&d_bits, (size_t)ncand))) return st;
    if ((st = tmp.alloc(&d_entries, sizeof(uint32_t) * (size_t)ncand))) return st;
    if ((st = tmp.alloc(&d_off, sizeof(int64_t) * ((size_t)ncand + 1)))) return st;
    { k_idx_list<<<grid_for(n, 256, sm), 256, 0, s>>>(n, d_flag, d_pos, d_list); count_launch(); }
    const int nl = (int)ncand;
    // the candidates' indices, largest neighbourhood first (both passes take them in this order)
    int32_t* d_order = nullptr;
    int* d_next = nullptr;
    if ((st = tmp.alloc(&d_order, sizeof(int32_t) * (size_t)ncand))) return st;
    if ((st = tmp.alloc(&d_next, sizeof(int)))) return st;
    if ((st = size_order(g, d_list, ncand, true, d_order))) return st;
    HYP_CUDA(cudaMemsetAsync(d_next, 0, sizeof(int), s));
    const int pblocks = (int)std::min<int64_t>(ncand, (int64_t)sm * 8);  // 8 x 256 threads per SM
    { k_idx_plan<<<pblocks, kThreads, 0, s>>>(d_list, nl, d_order, d_next, g->vinfo, g->v_span, g->he_mem, g->tsum,
                                              g->prof, g->id_bits, d_bits, d_entries); count_launch(); }
    if ((st = exclusive_scan_u32_to_i64(g, d_entries, d_off, ncand))) return st;
    int64_t total = 0;
    HYP_CUDA(cudaMemcpyAsync(&total, d_off + ncand, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    if (total >= ((int64_t)1 << kIdxBitsShift)) return set_error(HYPERIM_EOVERFLOW, "chunk index too large");
    g->idx_entries = total;
    if (total > 0) {
        if ((st = dev_alloc(g, (void**)&g->idx_tab, sizeof(uint32_t) * (size_t)total))) return st;
        { k_idx_word<<<grid_for(ncand, 256, sm), 256, 0, s>>>(d_list, nl, d_bits, d_entries, d_off, g->idx); count_launch(); }
        // per resident block, room for the largest neighbourhood
        HYP_CUDA(cudaFuncSetAttribute(k_idx_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFillSmem));
        int per_sm = 0;
        HYP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_idx_fill, kFillThreads, kFillSmem));
        if (per_sm < 1) per_sm = 1;
        const int64_t cap = g->max_tsum;
        int fblocks = (int)std::min<int64_t>(ncand, (int64_t)sm * per_sm);
        // keep the scratch area within 2 GiB
        while (fblocks > sm && (int64_t)fblocks * cap * 4 > ((int64_t)2 << 30)) fblocks -= sm;
        uint32_t* d_scratch = nullptr;
        if ((st = tmp.alloc(&d_scratch, sizeof(uint32_t) * (size_t)cap * fblocks))) return st;
        HYP_CUDA(cudaMemsetAsync(d_next, 0, sizeof(int), s));
        { k_idx_fill<<<fblocks, kFillThreads, kFillSmem, s>>>(d_list, nl, d_bits, d_entries, d_off, g->vinfo, g->v_span,
                                                  g->he_mem, g->tsum, g->prof, g->id_bits, g->idx_tab, d_scratch,
                                                  cap, d_order, d_next, g->d_status); count_launch(); }
        if ((st = check_device_status(g, "chunk index"))) return st;
        // indexed vertices
        std::vector<uint32_t> e((size_t)ncand);
        HYP_CUDA(cudaMemcpyAsync(e.data(), d_entries, sizeof(uint32_t) * (size_t)ncand, cudaMemcpyDeviceToHost, s));
        HYP_CUDA(cudaStreamSynchronize(s));
        int32_t cnt = 0;
        for (uint32_t x : e) cnt += x ? 1 : 0;
        g->idx_vertices = cnt;
    }
    HYP_CUDA(cudaGetLastError());
    return HYPERIM_OK;
}

}  // namespace hyperim
