// Greedy max coverage over an RR pool (Algorithm 1; marginal coverage of Eq. 2) on the device.
//
// Scores are integers: an RR set of stratum s weighs W_s = floor(|V_s| 2^32 / n_s) (1 with plain
// roots), so sums do not depend on the order of the atomic updates. Each round: argmax over the
// vertices not picked yet (ties to the lowest id), then the RR sets containing the winner that
// are not covered yet are retired: marked covered, counted in Lambda_s, and their weight is
// subtracted from the score of every member. The k rounds run back to back on the stream; the
// winner of a round is read on the device by the next launch.
#include <algorithm>

#include "internal.h"

namespace hyperim {
namespace {

constexpr int kArgThreads = 256;

struct Weights {
    unsigned long long w[HYPERIM_NSTRATA];
};

__global__ void k_count_occ(const int32_t* __restrict__ mem, int64_t total, uint32_t* __restrict__ cnt) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[mem[x]], 1u);
}

// inverted index (vertex -> RR ids) and initial weighted scores; one warp per RR set
__global__ void k_scatter_inv(const int64_t* __restrict__ rr_off, const int32_t* __restrict__ mem,
                              const uint8_t* __restrict__ rr_stratum, int64_t N,
                              const int64_t* __restrict__ inv_off, uint32_t* __restrict__ cur,
                              uint32_t* __restrict__ inv, unsigned long long* __restrict__ score,
                              Weights W) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < N; r += nwarps) {
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

// argmax of score over unpicked vertices, lowest id on ties; the last block to finish reduces
// the per-block winners, records the seed and marks it picked.
__global__ void __launch_bounds__(kArgThreads)
k_argmax(const unsigned long long* __restrict__ score, uint8_t* __restrict__ picked, int32_t n,
         unsigned long long* __restrict__ bscore, uint32_t* __restrict__ bid,
         unsigned int* __restrict__ ticket, int32_t* __restrict__ best, int32_t* __restrict__ seeds,
         int round) {
    __shared__ unsigned long long ss[kArgThreads / 32];
    __shared__ uint32_t si[kArgThreads / 32];
    __shared__ bool last;
    unsigned long long bs = 0;
    uint32_t bi = 0xFFFFFFFFu;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (picked[v]) continue;
        const unsigned long long s = score[v];
        if (better(s, (uint32_t)v, bs, bi)) { bs = s; bi = (uint32_t)v; }
    }
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
        *ticket = 0;
    }
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
                           const uint8_t* __restrict__ rr_stratum, int64_t N,
                           const uint8_t* __restrict__ in_s, unsigned long long* __restrict__ lam) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < N; r += nwarps) {
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

int grid_cap(int64_t items, int threads, int sm, int per_sm) {
    int64_t b = (items + threads - 1) / threads;
    const int64_t cap = (int64_t)sm * per_sm;
    if (b < 1) b = 1;
    return (int)std::min(b, cap);
}

}  // namespace

hyperim_status greedy(hyperim_graph* g, hyperim_pool* p, int32_t k, int32_t* seeds_host,
                      uint64_t lambda_s[HYPERIM_NSTRATA]) {
    cudaStream_t s = g->stream;
    const int32_t n = g->n;
    const int64_t N = p->count, T = p->total;
    const int sm = g->sm_count;
    if (N >= (int64_t)0xFFFFFFFFll) return set_error(HYPERIM_EOVERFLOW, "more than 2^32 - 1 RR sets");
    Weights W;
    for (int i = 0; i < HYPERIM_NSTRATA; ++i)
        W.w[i] = stratum_weight(g, p->root_mode, p->n_s[i], i);
    hyperim_status st;
    uint32_t *cnt = nullptr, *inv = nullptr, *covered = nullptr, *bid = nullptr, *ticket = nullptr;
    int64_t* inv_off = nullptr;
    unsigned long long *score = nullptr, *lam = nullptr, *bscore = nullptr;
    uint8_t* picked = nullptr;
    int32_t *best = nullptr, *seeds_d = nullptr;
    const int ablocks = grid_cap(n, kArgThreads, sm, 2);
    const size_t bytes_cnt = sizeof(uint32_t) * ((size_t)n + 1);
    const size_t bytes_inv = sizeof(uint32_t) * (size_t)std::max<int64_t>(T, 1);
    const size_t bytes_cov = sizeof(uint32_t) * (size_t)std::max<int64_t>(N, 1);
    if ((st = dev_alloc(g, (void**)&cnt, bytes_cnt))) return st;
    if ((st = dev_alloc(g, (void**)&inv_off, sizeof(int64_t) * ((size_t)n + 1)))) return st;
    if ((st = dev_alloc(g, (void**)&inv, bytes_inv))) return st;
    if ((st = dev_alloc(g, (void**)&score, sizeof(unsigned long long) * (size_t)n))) return st;
    if ((st = dev_alloc(g, (void**)&picked, (size_t)n))) return st;
    if ((st = dev_alloc(g, (void**)&covered, bytes_cov))) return st;
    if ((st = dev_alloc(g, (void**)&lam, sizeof(unsigned long long) * HYPERIM_NSTRATA))) return st;
    if ((st = dev_alloc(g, (void**)&bscore, sizeof(unsigned long long) * ablocks))) return st;
    if ((st = dev_alloc(g, (void**)&bid, sizeof(uint32_t) * ablocks))) return st;
    if ((st = dev_alloc(g, (void**)&ticket, sizeof(uint32_t) * 2))) return st;
    if ((st = dev_alloc(g, (void**)&best, sizeof(int32_t) * 2))) return st;
    if ((st = dev_alloc(g, (void**)&seeds_d, sizeof(int32_t) * (size_t)k))) return st;
    HYP_CUDA(cudaMemsetAsync(cnt, 0, bytes_cnt, s));
    HYP_CUDA(cudaMemsetAsync(score, 0, sizeof(unsigned long long) * (size_t)n, s));
    HYP_CUDA(cudaMemsetAsync(picked, 0, (size_t)n, s));
    HYP_CUDA(cudaMemsetAsync(covered, 0, bytes_cov, s));
    HYP_CUDA(cudaMemsetAsync(lam, 0, sizeof(unsigned long long) * HYPERIM_NSTRATA, s));
    HYP_CUDA(cudaMemsetAsync(ticket, 0, sizeof(uint32_t) * 2, s));
    if (T > 0) { k_count_occ<<<grid_cap(T, 256, sm, 32), 256, 0, s>>>(p->rr_mem, T, cnt); count_launch(); }
    if ((st = exclusive_scan_u32_to_i64(g, cnt, inv_off, n))) return st;
    HYP_CUDA(cudaMemsetAsync(cnt, 0, bytes_cnt, s));
    if (N > 0)
        { k_scatter_inv<<<grid_cap(N * 32, 256, sm, 32), 256, 0, s>>>(p->rr_off, p->rr_mem, p->rr_stratum,
                                                                    N, inv_off, cnt, inv, score, W); count_launch(); }
    const int rblocks = sm * 8;
    for (int32_t round = 0; round < k; ++round) {
        { k_argmax<<<ablocks, kArgThreads, 0, s>>>(score, picked, n, bscore, bid, ticket, best, seeds_d,
                                                 round); count_launch(); }
        { k_retire<<<rblocks, 256, 0, s>>>(best, inv_off, inv, p->rr_off, p->rr_mem, p->rr_stratum,
                                         covered, score, lam, W); count_launch(); }
    }
    HYP_CUDA(cudaGetLastError());
    unsigned long long hl[HYPERIM_NSTRATA];
    HYP_CUDA(cudaMemcpyAsync(seeds_host, seeds_d, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaMemcpyAsync(hl, lam, sizeof(hl), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < HYPERIM_NSTRATA; ++i) lambda_s[i] = hl[i];
    dev_free(g, cnt, bytes_cnt);
    dev_free(g, inv_off, sizeof(int64_t) * ((size_t)n + 1));
    dev_free(g, inv, bytes_inv);
    dev_free(g, score, sizeof(unsigned long long) * (size_t)n);
    dev_free(g, picked, (size_t)n);
    dev_free(g, covered, bytes_cov);
    dev_free(g, lam, sizeof(unsigned long long) * HYPERIM_NSTRATA);
    dev_free(g, bscore, sizeof(unsigned long long) * ablocks);
    dev_free(g, bid, sizeof(uint32_t) * ablocks);
    dev_free(g, ticket, sizeof(uint32_t) * 2);
    dev_free(g, best, sizeof(int32_t) * 2);
    dev_free(g, seeds_d, sizeof(int32_t) * (size_t)k);
    return check_device_status(g, "greedy");
}

hyperim_status coverage(hyperim_graph* g, hyperim_pool* p, const int32_t* seeds_host, int32_t k,
                        uint64_t lambda_s[HYPERIM_NSTRATA]) {
    cudaStream_t s = g->stream;
    const int64_t N = p->count;
    hyperim_status st;
    uint8_t* in_s = nullptr;
    unsigned long long* lam = nullptr;
    int32_t* sd = nullptr;
    const size_t kk = (size_t)std::max(k, 1);
    if ((st = dev_alloc(g, (void**)&in_s, (size_t)g->n))) return st;
    if ((st = dev_alloc(g, (void**)&lam, sizeof(unsigned long long) * HYPERIM_NSTRATA))) return st;
    if ((st = dev_alloc(g, (void**)&sd, sizeof(int32_t) * kk))) return st;
    HYP_CUDA(cudaMemsetAsync(in_s, 0, (size_t)g->n, s));
    HYP_CUDA(cudaMemsetAsync(lam, 0, sizeof(unsigned long long) * HYPERIM_NSTRATA, s));
    if (k > 0) {
        HYP_CUDA(cudaMemcpyAsync(sd, seeds_host, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, s));
        { k_mark<<<grid_cap(k, 256, g->sm_count, 4), 256, 0, s>>>(sd, k, in_s); count_launch(); }
    }
    if (N > 0)
        { k_coverage<<<grid_cap(N * 32, 256, g->sm_count, 32), 256, 0, s>>>(p->rr_off, p->rr_mem,
                                                                          p->rr_stratum, N, in_s, lam); count_launch(); }
    HYP_CUDA(cudaGetLastError());
    unsigned long long hl[HYPERIM_NSTRATA];
    HYP_CUDA(cudaMemcpyAsync(hl, lam, sizeof(hl), cudaMemcpyDeviceToHost, s));
    HYP_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < HYPERIM_NSTRATA; ++i) lambda_s[i] = hl[i];
    dev_free(g, in_s, (size_t)g->n);
    dev_free(g, lam, sizeof(unsigned long long) * HYPERIM_NSTRATA);
    dev_free(g, sd, sizeof(int32_t) * kk);
    return check_device_status(g, "coverage");
}

}  // namespace hyperim
