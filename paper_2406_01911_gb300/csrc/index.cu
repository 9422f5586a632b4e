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
//   k_idx_fill        per indexed vertex: members bucketed by chunk through a global scratch
//                     area, each chunk sorted on chip, its runs (multiplicity w -> layer) counted;
//                     before chunk k the running per-layer counts are written as column k
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
k_idx_plan(const int32_t* __restrict__ list, int32_t nlist, const int4* __restrict__ vinfo,
           const int2* __restrict__ v_span, const int32_t* __restrict__ he_mem,
           const int32_t* __restrict__ tsum, const uint4* __restrict__ prof, int id_bits,
           uint8_t* __restrict__ bits_out, uint32_t* __restrict__ entries) {
    __shared__ int hist_a[kBins];
    __shared__ int hist_b[kBins / 2];
    __shared__ int pre[2 * kThreads + 1];
    __shared__ int wmax[kThreads / 32];
    __shared__ int target_s;
    const int hb = id_bits < kIdxMaxBits ? id_bits : kIdxMaxBits;
    const int shift = id_bits - hb;
    for (int i = blockIdx.x; i < nlist; i += gridDim.x) {
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

// Per indexed vertex (one block): members bucketed by chunk through a global scratch area; the
// warps then take chunks in turn, sort one on chip (warp bucket sort), count its runs per layer
// (multiplicity w -> layer by search in the descending w list) and write the counts as column k;
// finally every layer row becomes an exclusive prefix along the chunks.
constexpr int kFillWarps = 4;
constexpr int kFillThreads = kFillWarps * 32;
constexpr size_t kFillSmem = sizeof(int) * kBins + sizeof(uint32_t) * kIdxMaxL +
                             sizeof(int) * (2 * kFillThreads + 1) +
                             kFillWarps * (sizeof(uint32_t) * (2 * kIdxTarget + kIdxMaxL) + sizeof(int) * 256);

__global__ void __launch_bounds__(kFillThreads)
k_idx_fill(const int32_t* __restrict__ list, int32_t nlist, const uint8_t* __restrict__ bits_in,
           const uint32_t* __restrict__ entries, const int64_t* __restrict__ off,
           const int4* __restrict__ vinfo, const int2* __restrict__ v_span,
           const int32_t* __restrict__ he_mem, const uint4* __restrict__ prof, int id_bits,
           uint32_t* __restrict__ tab, uint32_t* __restrict__ scratch, int64_t scratch_cap,
           DevStatus* st) {
    extern __shared__ __align__(16) unsigned char fill_smem[];
    int* chunk_end = reinterpret_cast<int*>(fill_smem);                 // kBins
    uint32_t* lw = reinterpret_cast<uint32_t*>(chunk_end + kBins);      // kIdxMaxL
    int* pre = reinterpret_cast<int*>(lw + kIdxMaxL);                   // 2 kFillThreads + 1
    uint32_t* wbase = reinterpret_cast<uint32_t*>(pre + 2 * kFillThreads + 1);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t* raw = wbase + (size_t)wid * (2 * kIdxTarget + kIdxMaxL);
    uint32_t* srt = raw + kIdxTarget;
    uint32_t* wcnt = srt + kIdxTarget;                                  // kIdxMaxL per warp
    int* bkt = reinterpret_cast<int*>(wbase + (size_t)kFillWarps * (2 * kIdxTarget + kIdxMaxL)) + wid * 256;
    uint32_t* big = scratch + (int64_t)blockIdx.x * scratch_cap;
    for (int i = blockIdx.x; i < nlist; i += gridDim.x) {
        if (entries[i] == 0) continue;
        const int32_t mu = list[i];
        const int4 vi = vinfo[mu];
        const int l = vi.y, c = bits_in[i];
        const int C = 1 << c, shift = id_bits - c;
        uint32_t* t = tab + off[i];
        for (int q = threadIdx.x; q < l; q += kFillThreads) lw[q] = prof[2 * ((int64_t)vi.x + q)].x & ~kPOneFlag;
        for (int k = threadIdx.x; k < C; k += kFillThreads) chunk_end[k] = 0;
        __syncthreads();
        for_each_member<kFillThreads>(v_span, he_mem, mu, vi.z, vi.w, pre,
                                      [&](uint32_t x) { atomicAdd(&chunk_end[x >> shift], 1); });
        __syncthreads();
        warp0_exclusive_scan(chunk_end, C);
        __syncthreads();
        for_each_member<kFillThreads>(v_span, he_mem, mu, vi.z, vi.w, pre, [&](uint32_t x) {
            const int p = atomicAdd(&chunk_end[x >> shift], 1);
            if (p < scratch_cap) big[p] = x;
        });
        __threadfence_block();
        __syncthreads();
        // chunk_end[k] is now the end of chunk k
        if (chunk_end[C - 1] > scratch_cap) {
            if (threadIdx.x == 0) dev_fail(st, kErrCapacity, mu);
            __syncthreads();
            continue;
        }
        for (int k = wid; k < C; k += kFillWarps) {
            const int begin = k ? chunk_end[k - 1] : 0;
            const int cnt = chunk_end[k] - begin;
            for (int q = lane; q < l; q += 32) wcnt[q] = 0;
            if (cnt > kIdxTarget) {
                if (lane == 0) dev_fail(st, kErrBucket, mu);
            } else if (cnt > 0) {
                const int nbits = bucket_bits(cnt, 8);
                const int nb = 1 << nbits;
                const int bshift = shift > nbits ? shift - nbits : 0;
                const uint32_t key_mask = (uint32_t)nb - 1;
                for (int b = lane; b < nb; b += 32) bkt[b] = 0;
                __syncwarp();
                for (int x = lane; x < cnt; x += 32) {
                    const uint32_t v = big[begin + x];
                    raw[x] = v;
                    atomicAdd(&bkt[(v >> bshift) & key_mask], 1);
                }
                __syncwarp();
                const int maxb = warp_bucket_scan(bkt, nb);
                warp_scatter_sort(raw, cnt, kSentinel, srt, cnt, bkt, nb, 0u, bshift, key_mask, maxb);
                walk_runs<32>(srt, cnt, [&](bool start, uint32_t, int mult) -> bool {
                    if (start) {
                        int lo = 0, hi = l;  // lw descends: first q with lw[q] <= mult
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (lw[mid] > (uint32_t)mult) lo = mid + 1; else hi = mid;
                        }
                        if (lo < l && lw[lo] == (uint32_t)mult) atomicAdd(&wcnt[lo], 1u);
                        else dev_fail(st, kErrProfile, mu);
                    }
                    return false;
                });
            }
            __syncwarp();
            for (int q = lane; q < l; q += 32) t[(int64_t)q * C + k] = wcnt[q];
            __syncwarp();
        }
        __syncthreads();
        // counts -> exclusive prefix along the chunks, one layer row per thread
        for (int q = threadIdx.x; q < l; q += kFillThreads) {
            uint32_t* row = t + (int64_t)q * C;
            uint32_t run = 0;
            for (int k = 0; k < C; ++k) {
                const uint32_t v = row[k];
                row[k] = run;
                run += v;
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
    if ((st = dev_alloc(g, (void**)&g->idx, sizeof(uint64_t) * (size_t)(n > 0 ? n : 1)))) return st;
    HYP_CUDA(cudaMemsetAsync(g->idx, 0, sizeof(uint64_t) * (size_t)(n > 0 ? n : 1), s));
    g->idx_entries = 0;
    g->idx_vertices = 0;
    if (n == 0 || g->max_tsum <= kIdxMinT) return HYPERIM_OK;

    uint32_t* d_flag = nullptr;
    int64_t* d_pos = nullptr;
    if ((st = dev_alloc(g, (void**)&d_flag, sizeof(uint32_t) * (size_t)n))) return st;
    if ((st = dev_alloc(g, (void**)&d_pos, sizeof(int64_t) * ((size_t)n + 1)))) return st;
    { k_idx_candidates<<<grid_for(n, 256, sm), 256, 0, s>>>(n, g->vinfo, g->tsum, d_flag); count_launch(); }
    if ((st = exclusive_scan_u32_to_i64(g, d_flag, d_pos, n))) return st;
    int64_t ncand = 0;
    HYP_CUDA(cudaMemcpyAsync(&ncand, d_pos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    if (ncand == 0) {
        dev_free(g, d_flag, sizeof(uint32_t) * (size_t)n);
        dev_free(g, d_pos, sizeof(int64_t) * ((size_t)n + 1));
        return HYPERIM_OK;
    }
    int32_t* d_list = nullptr;
    uint8_t* d_bits = nullptr;
    uint32_t* d_entries = nullptr;
    int64_t* d_off = nullptr;
    if ((st = dev_alloc(g, (void**)&d_list, sizeof(int32_t) * (size_t)ncand))) return st;
    if ((st = dev_alloc(g, (void**)&d_bits, (size_t)ncand))) return st;
    if ((st = dev_alloc(g, (void**)&d_entries, sizeof(uint32_t) * (size_t)ncand))) return st;
    if ((st = dev_alloc(g, (void**)&d_off, sizeof(int64_t) * ((size_t)ncand + 1)))) return st;
    { k_idx_list<<<grid_for(n, 256, sm), 256, 0, s>>>(n, d_flag, d_pos, d_list); count_launch(); }
    const int nl = (int)ncand;
    const int pblocks = (int)std::min<int64_t>(ncand, (int64_t)sm * 4);
    { k_idx_plan<<<pblocks, kThreads, 0, s>>>(d_list, nl, g->vinfo, g->v_span, g->he_mem, g->tsum, g->prof,
                                              g->id_bits, d_bits, d_entries); count_launch(); }
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
        // keep the scratch area within 1 GiB
        while (fblocks > sm && (int64_t)fblocks * cap * 4 > ((int64_t)1 << 30)) fblocks -= sm;
        uint32_t* d_scratch = nullptr;
        if ((st = dev_alloc(g, (void**)&d_scratch, sizeof(uint32_t) * (size_t)cap * fblocks))) return st;
        { k_idx_fill<<<fblocks, kFillThreads, kFillSmem, s>>>(d_list, nl, d_bits, d_entries, d_off, g->vinfo, g->v_span,
                                                  g->he_mem, g->prof, g->id_bits, g->idx_tab, d_scratch, cap,
                                                  g->d_status); count_launch(); }
        if ((st = check_device_status(g, "chunk index"))) return st;
        dev_free(g, d_scratch, sizeof(uint32_t) * (size_t)cap * fblocks);
        // indexed vertices
        std::vector<uint32_t> e((size_t)ncand);
        HYP_CUDA(cudaMemcpyAsync(e.data(), d_entries, sizeof(uint32_t) * (size_t)ncand, cudaMemcpyDeviceToHost, s));
        HYP_CUDA(cudaStreamSynchronize(s));
        int32_t cnt = 0;
        for (uint32_t x : e) cnt += x ? 1 : 0;
        g->idx_vertices = cnt;
    }
    dev_free(g, d_flag, sizeof(uint32_t) * (size_t)n);
    dev_free(g, d_pos, sizeof(int64_t) * ((size_t)n + 1));
    dev_free(g, d_list, sizeof(int32_t) * (size_t)ncand);
    dev_free(g, d_bits, (size_t)ncand);
    dev_free(g, d_entries, sizeof(uint32_t) * (size_t)ncand);
    dev_free(g, d_off, sizeof(int64_t) * ((size_t)ncand + 1));
    HYP_CUDA(cudaGetLastError());
    return HYPERIM_OK;
}

}  // namespace hyperim
