// hyperim_coverage_noalloc: the coverage step (RR sets of a pool hit by a seed set, per stratum)
// for callers that must not allocate device memory. Its only scratch is a fixed array of seed
// flags compiled into the library; every other buffer is the caller's.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace hyperim {
namespace {

// One flag per vertex id. Every GPU that loads the library holds these bytes until the process
// exits. All calls share them, so calls that overlap on the GPU race (see the header).
static __device__ __align__(256) uint8_t g_noalloc_seed_flags[HYPERIM_NOALLOC_MAX_N];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
uint8_t* g_addr[kMaxDevices] = {};

// Host code cannot use g_noalloc_seed_flags directly (in host code it names a host-side stand-in,
// not device memory): look its device address up once per device, with that device current.
hyperim_status flags_address(uint8_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(HYPERIM_EINVAL, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_seed_flags);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(seed flags)");
        g_addr[dev] = static_cast<uint8_t*>(p);
    }
    *out = g_addr[dev];
    return HYPERIM_OK;
}

// clear flags[0, n) and the 16 output counters
__global__ void k_na_clear(uint8_t* __restrict__ flags, int32_t n, unsigned long long* __restrict__ lam) {
    const int64_t words = ((int64_t)n + 15) / 16;  // n rounded up to 16-byte words (array is padded)
    uint4* f4 = reinterpret_cast<uint4*>(flags);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * blockDim.x)
        f4[i] = make_uint4(0, 0, 0, 0);
    if (blockIdx.x == 0 && threadIdx.x < HYPERIM_NSTRATA) lam[threadIdx.x] = 0;
}

// mark the seeds (ids outside [0, n) are ignored)
__global__ void k_na_mark(const int32_t* __restrict__ seeds, int32_t k, int32_t n,
                          uint8_t* __restrict__ flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const int32_t v = seeds[i];
        if (v >= 0 && v < n) flags[v] = 1;
    }
}

// one warp per RR set: counted in its stratum if any member is flagged
__global__ void k_na_cover(const int64_t* __restrict__ rr_off, const int32_t* __restrict__ rr_mem,
                           const uint8_t* __restrict__ rr_stratum, int64_t count, int32_t n,
                           const uint8_t* __restrict__ flags, unsigned long long* __restrict__ lam) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < count; r += nwarps) {
        const int64_t b = rr_off[r], e = rr_off[r + 1];
        bool hit = false;
        for (int64_t base = b; base < e; base += 32) {
            const int64_t x = base + lane;
            bool f = false;
            if (x < e) {
                const int32_t v = rr_mem[x];
                f = v >= 0 && v < n && flags[v] != 0;
            }
            if (__any_sync(0xFFFFFFFFu, f)) { hit = true; break; }
        }
        if (hit && lane == 0) atomicAdd(&lam[rr_stratum[r] & (HYPERIM_NSTRATA - 1)], 1ull);
    }
}

}  // namespace
}  // namespace hyperim

using namespace hyperim;

extern "C" hyperim_status hyperim_coverage_noalloc(int32_t n, const int64_t* rr_off, const int32_t* rr_mem,
                                                   const uint8_t* rr_stratum, int64_t count,
                                                   const int32_t* seeds, int32_t k,
                                                   unsigned long long* lambda_s, void* cuda_stream) {
    if (n < 1 || (uint32_t)n > HYPERIM_NOALLOC_MAX_N)
        return set_error(HYPERIM_EINVAL, "n = " + std::to_string(n) + " outside [1, " +
                                             std::to_string(HYPERIM_NOALLOC_MAX_N) +
                                             "]: the fixed seed-flag array is too small");
    if (count < 0 || k < 0) return set_error(HYPERIM_EINVAL, "count and k must be >= 0");
    if (!lambda_s || (count > 0 && (!rr_off || !rr_mem || !rr_stratum)) || (k > 0 && !seeds))
        return set_error(HYPERIM_EINVAL, "null pointer argument");
    uint8_t* flags = nullptr;
    hyperim_status st = flags_address(&flags);
    if (st != HYPERIM_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    if (sm < 1) sm = 1;
    const int64_t words = ((int64_t)n + 15) / 16;
    const int gclear = (int)((words + 255) / 256 < sm * 8 ? (words + 255) / 256 : sm * 8);
    { k_na_clear<<<gclear > 0 ? gclear : 1, 256, 0, s>>>(flags, n, lambda_s); count_launch(); }
    if (k > 0) { k_na_mark<<<(k + 255) / 256 < sm * 4 ? (k + 255) / 256 : sm * 4, 256, 0, s>>>(seeds, k, n, flags); count_launch(); }
    if (count > 0) {
        const int64_t want = (count * 32 + 255) / 256;
        const int g = (int)(want < (int64_t)sm * 32 ? want : (int64_t)sm * 32);
        { k_na_cover<<<g, 256, 0, s>>>(rr_off, rr_mem, rr_stratum, count, n, flags, lambda_s); count_launch(); }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "coverage kernels");
    return HYPERIM_OK;
}
