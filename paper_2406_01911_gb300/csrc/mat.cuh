// Neighbourhood materialisation of HyperIM (Sec. 3.1.1): for a vertex mu, the multiset of the
// members (other than mu) of every hyperedge containing mu, in ascending id order. A run of equal
// ids nu has length w(mu, nu), the number of hyperedges shared; the runs of length w_i form the
// layer L_i of A(mu), ordered by ascending id. The clique expansion is never stored: the multiset
// is rebuilt from the incidence lists on demand, in on-chip memory.
//
// Groups: the same routines run for a warp (G = 32) or a whole block (G = blockDim.x).
#pragma once
#include <cstdint>

namespace hyperim {

constexpr uint32_t kSentinel = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <int G>
struct Group;

template <>
struct Group<32> {
    static constexpr int size = 32;
    __device__ __forceinline__ static int rank() { return threadIdx.x & 31; }
    __device__ __forceinline__ static void sync() { __syncwarp(); }
    // exclusive count of true flags before this thread; *total = count over the group
    __device__ __forceinline__ static int excl_count(bool f, int* /*tmp*/, int* total) {
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, f);
        *total = __popc(b);
        return __popc(b & lanemask_lt());
    }
    __device__ __forceinline__ static bool any(bool f, int* /*tmp*/) {
        return __any_sync(0xFFFFFFFFu, f);
    }
};

template <int G>
struct Group {
    static constexpr int size = G;
    static constexpr int warps = G / 32;
    __device__ __forceinline__ static int rank() { return threadIdx.x; }
    __device__ __forceinline__ static void sync() { __syncthreads(); }
    // tmp: at least warps + 1 ints of shared memory
    __device__ __forceinline__ static int excl_count(bool f, int* tmp, int* total) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, f);
        if (lane == 0) tmp[warp] = __popc(b);
        __syncthreads();
        int before = 0, all = 0;
#pragma unroll
        for (int w = 0; w < warps; ++w) {
            const int c = tmp[w];
            before += w < warp ? c : 0;
            all += c;
        }
        __syncthreads();
        *total = all;
        return before + __popc(b & lanemask_lt());
    }
    __device__ __forceinline__ static bool any(bool f, int* tmp) {
        return __syncthreads_or(f) != 0;
    }
};

// Bitonic sort of buf[0, count) ascending in shared memory; buf must have room for the next
// power of two >= count (the tail is padded with the sentinel).
template <int G>
__device__ void group_sort(uint32_t* buf, int count) {
    using Gr = Group<G>;
    int P = 1;
    while (P < count) P <<= 1;
    for (int i = count + Gr::rank(); i < P; i += G) buf[i] = kSentinel;
    Gr::sync();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = Gr::rank(); t < (P >> 1); t += G) {
                const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                const int ixj = i | j;
                const uint32_t a = buf[i], b = buf[ixj];
                const bool up = (i & k) == 0;
                if ((a > b) == up) {
                    buf[i] = b;
                    buf[ixj] = a;
                }
            }
            Gr::sync();
        }
    }
}

// Incidence store view used by the device routines.
struct Incidence {
    const int32_t* he_off;
    const int32_t* he_mem;
    const int32_t* v_off;
    const int32_t* v_he;
};

// Copy the members != mu of mu's hyperedges into dst[0, T') (any order). Warps of the group take
// hyperedges round-robin; each reserves its output range with a shared atomic. Returns T' to
// every thread of the group. cursor: one shared int.
template <int G>
__device__ int gather_nbhd(const Incidence& I, int32_t mu, uint32_t* dst, int* cursor) {
    using Gr = Group<G>;
    if (Gr::rank() == 0) *cursor = 0;
    Gr::sync();
    const int lane = threadIdx.x & 31;
    const int wid = Gr::rank() >> 5;
    constexpr int nw = G / 32;
    const int e0 = I.v_off[mu], e1 = I.v_off[mu + 1];
    for (int e = e0 + wid; e < e1; e += nw) {
        const int he = I.v_he[e];
        const int b = I.he_off[he], len = I.he_off[he + 1] - b;
        int base = 0;
        if (lane == 0) base = atomicAdd(cursor, len - 1);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        for (int i = lane; i < len; i += 32) {
            const uint32_t x = (uint32_t)I.he_mem[b + i];
            if (x != (uint32_t)mu) {
                // members are sorted, so the ones after mu move down by one
                // (position of mu is unknown here; count it from the comparison)
                dst[base + i - (x > (uint32_t)mu ? 1 : 0)] = x;
            }
        }
    }
    Gr::sync();
    const int T = *cursor;
    Gr::sync();
    return T;
}

// Walk the runs of a sorted buffer buf[0, count) in ascending order, G positions at a time.
// For each chunk every thread of the group calls consume(is_start, value, run_length); the call
// is uniform across the group (threads past the end pass is_start = false). consume returns
// true to stop the walk (must be uniform too). Run lengths are taken by scanning forward, so a
// run that continues past the chunk is still measured in full at its start.
template <int G, typename F>
__device__ bool walk_runs(const uint32_t* buf, int count, F&& consume) {
    using Gr = Group<G>;
    for (int base = 0; base < count; base += G) {
        const int p = base + Gr::rank();
        bool start = false;
        uint32_t x = kSentinel;
        int mult = 0;
        if (p < count) {
            x = buf[p];
            start = (p == 0) || (buf[p - 1] != x);
            if (start) {
                mult = 1;
                while (p + mult < count && buf[p + mult] == x) ++mult;
            }
        }
        if (consume(start, x, mult)) return true;
    }
    return false;
}

}  // namespace hyperim
