// Exclusive prefix sums on the device (three passes: tile totals, scan of the totals in one
// block, per-tile scan plus offset). Used to turn counts into CSR offsets.
#include "internal.h"

namespace hyperim {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive scan of one value per thread across the block; returns the block total via *total
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* smem, int64_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t inc = warp_incl_scan(v);
    if (lane == 31) smem[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int64_t s = lane < nw ? smem[lane] : 0;
        const int64_t si = warp_incl_scan(s);
        if (lane < nw) smem[lane] = si - s;
        if (lane == nw - 1) smem[32] = si;
    }
    __syncthreads();
    const int64_t r = smem[warp] + inc - v;
    *total = smem[32];
    __syncthreads();
    return r;
}

template <typename T>
__global__ void k_tile_sums(const T* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
    __shared__ int64_t sm[33];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += (int64_t)in[base + i];
    int64_t tot;
    block_excl_scan(s, sm, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// single block: in-place exclusive scan of the tile totals; writes the grand total to *grand
__global__ void k_scan_sums(int64_t* sums, int64_t ntiles, int64_t* grand) {
    __shared__ int64_t sm[33];
    int64_t carry = 0;
    for (int64_t b = 0; b < ntiles; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        const int64_t v = i < ntiles ? sums[i] : 0;
        int64_t tot;
        const int64_t ex = block_excl_scan(v, sm, &tot);
        if (i < ntiles) sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *grand = carry;
}

template <typename T>
__global__ void k_tile_scan(const T* __restrict__ in, int64_t n, const int64_t* __restrict__ offs,
                            int64_t* __restrict__ out) {
    __shared__ int64_t sm[33];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? (int64_t)in[base + i] : 0;
        s += v[i];
    }
    int64_t tot;
    int64_t run = offs[blockIdx.x] + block_excl_scan(s, sm, &tot);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

template <typename T>
hyperim_status scan_impl(hyperim_graph* g, const T* in, int64_t* out, int64_t n) {
    if (n <= 0) {
        HYP_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), g->stream));
        return HYPERIM_OK;
    }
    const int64_t ntiles = (n + kTile - 1) / kTile;
    int64_t* sums = nullptr;
    hyperim_status st = dev_alloc(g, (void**)&sums, sizeof(int64_t) * (size_t)ntiles);
    if (st != HYPERIM_OK) return st;
    { k_tile_sums<T><<<(unsigned)ntiles, kScanThreads, 0, g->stream>>>(in, n, sums); count_launch(); }
    { k_scan_sums<<<1, 1024, 0, g->stream>>>(sums, ntiles, out + n); count_launch(); }
    { k_tile_scan<T><<<(unsigned)ntiles, kScanThreads, 0, g->stream>>>(in, n, sums, out); count_launch(); }
    cudaError_t e = cudaGetLastError();
    dev_free(g, sums, sizeof(int64_t) * (size_t)ntiles);
    if (e != cudaSuccess) return cuda_fail(e, "scan kernels");
    return HYPERIM_OK;
}

}  // namespace

hyperim_status exclusive_scan_u32_to_i64(hyperim_graph* g, const uint32_t* in, int64_t* out,
                                         int64_t n) {
    return scan_impl<uint32_t>(g, in, out, n);
}

hyperim_status exclusive_scan_i64(hyperim_graph* g, const int64_t* in, int64_t* out, int64_t n) {
    return scan_impl<int64_t>(g, in, out, n);
}

}  // namespace hyperim
