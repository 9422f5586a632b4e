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

namespace hyperim {

// ------------------------------------------------------------------------------------------
// Flattened neighbourhood gather. Hyperedge spans (start, length into he_mem) of mu's
// incidences are read G at a time; their lengths are prefix-summed in shared memory and every
// thread then walks member positions p = rank, rank + G, ... of the group, locating its
// hyperedge by binary search in the prefix: all member loads of a group are independent.
// f(pos, x) is called for every position pos in [0, sum of the hyperedge sizes) of the
// concatenation of mu's hyperedges (in incidence order), x the member there (mu included).
// pre: 2 G + 1 ints of shared memory (prefix and starts).
// ------------------------------------------------------------------------------------------
template <int G, typename F>
__device__ __forceinline__ void for_each_position(const int2* __restrict__ v_span,
                                                  const int32_t* __restrict__ he_mem,
                                                  int32_t v_begin, int32_t dh, int* pre, F&& f) {
    using Gr = Group<G>;
    const int r = Gr::rank();
    const int lane = threadIdx.x & 31;
    int* start = pre + G + 1;  // G starts follow the G + 1 prefix entries
    int base = 0;              // positions of the earlier groups of incidences
    for (int c0 = 0; c0 < dh; c0 += G) {
        const int cnt = min(G, dh - c0);
        int2 sp = make_int2(0, 0);
        if (r < cnt) sp = v_span[v_begin + c0 + r];
        int inc = sp.y;  // inclusive prefix of the lengths across the group
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o) inc += t;
        }
        if constexpr (G > 32) {
            const int wid = r >> 5;
            if (lane == 31) start[wid] = inc;  // warp totals, before the starts are written
            __syncthreads();
            int off = 0;
            for (int w = 0; w < wid; ++w) off += start[w];
            __syncthreads();
            inc += off;
        }
        if (r == 0) pre[0] = 0;
        if (r < cnt) {
            pre[r + 1] = inc;
            start[r] = sp.x;
        }
        Gr::sync();
        const int total = pre[cnt];
        // positions of a thread increase by G: when hyperedges are long compared with G the
        // hyperedge index is advanced step by step, otherwise found by binary search
        const bool stepwise = total >= cnt * (G / 4);
        int j = 0;
        // two positions per round: both loads are issued before either result is used (more in
        // flight measured slower: the unrolled copies cost more issue slots than they hide)
        constexpr int U = 2;
        for (int p0 = r; p0 < total; p0 += U * G) {
            uint32_t xs[U] = {};
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int p = p0 + u * G;
                if (p < total) {
                    if (stepwise && p != r) {
                        while (pre[j + 1] <= p) ++j;
                    } else {
                        int lo = 0, hi = cnt;  // j with pre[j] <= p < pre[j + 1]
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if (pre[mid] <= p) lo = mid; else hi = mid;
                        }
                        j = lo;
                    }
                    xs[u] = (uint32_t)he_mem[start[j] + (p - pre[j])];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (p0 + u * G < total) f(base + p0 + u * G, xs[u]);
        }
        base += total;
        Gr::sync();
    }
}

// f(x) for every member x != mu of mu's hyperedges (duplicates across hyperedges included).
template <int G, typename F>
__device__ __forceinline__ void for_each_member(const int2* __restrict__ v_span,
                                                const int32_t* __restrict__ he_mem, int32_t mu,
                                                int32_t v_begin, int32_t dh, int* pre, F&& f) {
    for_each_position<G>(v_span, he_mem, v_begin, dh, pre, [&](int, uint32_t x) {
        if (x != (uint32_t)mu) f(x);
    });
}

// ------------------------------------------------------------------------------------------
// Sorted neighbourhood multiset by MSD bucketing: count members per bucket of their top id bits,
// scan, scatter (second read of the members), then sort every bucket by insertion. With the
// random vertex ids of real and synthetic hypergraphs buckets hold a handful of keys; if one
// holds more than kBucketSortMax the whole buffer is sorted by the bitonic network instead
// (capacity must then be a power of two >= count). Returns the number of keys (members != mu).
// bkt: nb ints of shared memory; pre: 2 G + 1 ints; scratch: G / 32 ints; buf: capacity keys.
// ------------------------------------------------------------------------------------------
constexpr int kBucketSortMax = 48;

// Number of bucket bits for count keys: about two keys per bucket, between 5 and max_bits.
__device__ __forceinline__ int bucket_bits(int count, int max_bits) {
    int b = 5;
    while (b < max_bits && (2 << b) < count) ++b;
    return b;
}

template <int G>
__device__ int sorted_nbhd(const int2* __restrict__ v_span, const int32_t* __restrict__ he_mem,
                           int32_t mu, int32_t v_begin, int32_t dh, int expected, int id_bits,
                           uint32_t* buf, int* bkt, int max_bits, int* pre, int* scratch) {
    using Gr = Group<G>;
    const int r = Gr::rank();
    const int nbits = bucket_bits(expected, max_bits);
    const int nb = 1 << nbits;
    const int shift = id_bits > nbits ? id_bits - nbits : 0;
    const uint32_t key_mask = (uint32_t)nb - 1;
    for (int b = r; b < nb; b += G) bkt[b] = 0;
    Gr::sync();
    for_each_member<G>(v_span, he_mem, mu, v_begin, dh, pre,
                       [&](uint32_t x) { atomicAdd(&bkt[(x >> shift) & key_mask], 1); });
    // exclusive scan of the bucket counts (chunks of G, carried)
    int carry = 0;
    int maxb = 0;
    for (int c0 = 0; c0 < nb; c0 += G) {
        const int b = c0 + r;
        const int v = b < nb ? bkt[b] : 0;
        maxb = max(maxb, v);
        int inc = v;
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o) inc += t;
        }
        int total;
        if constexpr (G > 32) {
            const int wid = r >> 5;
            if (lane == 31) scratch[wid] = inc;
            __syncthreads();
            int off = 0;
            total = 0;
            for (int w = 0; w < G / 32; ++w) {
                const int c = scratch[w];
                off += w < wid ? c : 0;
                total += c;
            }
            __syncthreads();
            inc += off;
        } else {
            total = __shfl_sync(0xFFFFFFFFu, inc, 31);
        }
        if (b < nb) bkt[b] = carry + inc - v;
        carry += total;
    }
    // largest bucket across the group
    maxb = __reduce_max_sync(0xFFFFFFFFu, maxb);
    if constexpr (G > 32) {
        if ((threadIdx.x & 31) == 0) scratch[r >> 5] = maxb;
        __syncthreads();
        int m = 0;
        for (int w = 0; w < G / 32; ++w) m = max(m, scratch[w]);
        __syncthreads();
        maxb = m;
    }
    const int count = carry;
    Gr::sync();
    for_each_member<G>(v_span, he_mem, mu, v_begin, dh, pre, [&](uint32_t x) {
        buf[atomicAdd(&bkt[(x >> shift) & key_mask], 1)] = x;
    });
    // bkt[b] is now the end of bucket b
    if (maxb > kBucketSortMax) {
        group_sort<G>(buf, count);
        return count;
    }
    for (int b = r; b < nb; b += G) {
        const int e = bkt[b], s = b ? bkt[b - 1] : 0;
        for (int i = s + 1; i < e; ++i) {
            const uint32_t x = buf[i];
            int j = i - 1;
            while (j >= s && buf[j] > x) {
                buf[j + 1] = buf[j];
                --j;
            }
            buf[j + 1] = x;
        }
    }
    Gr::sync();
    return count;
}

// Sort keys already in buf[0, count) (one id-range chunk) by the same bucketing, reading the
// keys from src (global) instead of the incidence lists.
// (key bits below the chunk's common prefix: rem_bits; the next bucket bits of them key the buckets)
template <int G>
__device__ void sort_chunk(const uint32_t* __restrict__ src, int count, int rem_bits, uint32_t* buf,
                           int* bkt, int max_bits, int* scratch) {
    using Gr = Group<G>;
    const int r = Gr::rank();
    const int nbits = bucket_bits(count, max_bits);
    const int nb = 1 << nbits;
    const int shift = rem_bits > nbits ? rem_bits - nbits : 0;
    const uint32_t key_mask = (uint32_t)nb - 1;
    for (int b = r; b < nb; b += G) bkt[b] = 0;
    Gr::sync();
    for (int i = r; i < count; i += G) atomicAdd(&bkt[(src[i] >> shift) & key_mask], 1);
    Gr::sync();
    int carry = 0, maxb = 0;
    for (int c0 = 0; c0 < nb; c0 += G) {
        const int b = c0 + r;
        const int v = b < nb ? bkt[b] : 0;
        maxb = max(maxb, v);
        int inc = v;
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o) inc += t;
        }
        int total;
        if constexpr (G > 32) {
            const int wid = r >> 5;
            if (lane == 31) scratch[wid] = inc;
            __syncthreads();
            int off = 0;
            total = 0;
            for (int w = 0; w < G / 32; ++w) {
                const int c = scratch[w];
                off += w < wid ? c : 0;
                total += c;
            }
            __syncthreads();
            inc += off;
        } else {
            total = __shfl_sync(0xFFFFFFFFu, inc, 31);
        }
        if (b < nb) bkt[b] = carry + inc - v;
        carry += total;
    }
    maxb = __reduce_max_sync(0xFFFFFFFFu, maxb);
    if constexpr (G > 32) {
        if ((threadIdx.x & 31) == 0) scratch[r >> 5] = maxb;
        __syncthreads();
        int m = 0;
        for (int w = 0; w < G / 32; ++w) m = max(m, scratch[w]);
        __syncthreads();
        maxb = m;
    }
    Gr::sync();
    for (int i = r; i < count; i += G) {
        const uint32_t x = src[i];
        buf[atomicAdd(&bkt[(x >> shift) & key_mask], 1)] = x;
    }
    Gr::sync();
    if (maxb > kBucketSortMax) {
        group_sort<G>(buf, count);
        return;
    }
    for (int b = r; b < nb; b += G) {
        const int e = bkt[b], s = b ? bkt[b - 1] : 0;
        for (int i = s + 1; i < e; ++i) {
            const uint32_t x = buf[i];
            int j = i - 1;
            while (j >= s && buf[j] > x) {
                buf[j + 1] = buf[j];
                --j;
            }
            buf[j + 1] = x;
        }
    }
    Gr::sync();
}

// ------------------------------------------------------------------------------------------
// Warp bucket sort pieces shared by the RR kernel and the load-time profile and index kernels.
// ------------------------------------------------------------------------------------------
// Exclusive scan of a warp's bucket counts bkt[0, nb) in place; returns the largest count.
static __device__ int warp_bucket_scan(int* bkt, int nb) {
    const int lane = threadIdx.x & 31;
    int carry = 0, maxb = 0;
    for (int c0 = 0; c0 < nb; c0 += 32) {
        const int b = c0 + lane;
        const int v = b < nb ? bkt[b] : 0;
        maxb = max(maxb, v);
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o) inc += t;
        }
        if (b < nb) bkt[b] = carry + inc - v;
        carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
    __syncwarp();
    return __reduce_max_sync(0xFFFFFFFFu, maxb);
}

// Scatter raw[0, nraw) (entries equal to skip left out; count remain) into buf by the bucket
// starts in bkt (key ((x - base) >> shift) & key_mask), then sort each bucket by insertion, or
// the whole buffer by the bitonic network when the largest bucket exceeds kBucketSortMax.
static __device__ void warp_scatter_sort(const uint32_t* raw, int nraw, uint32_t skip, uint32_t* buf, int count,
                                  int* bkt, int nb, uint32_t base, int shift, uint32_t key_mask, int maxb) {
    const int lane = threadIdx.x & 31;
    for (int p = lane; p < nraw; p += 32) {
        const uint32_t x = raw[p];
        if (x != skip) buf[atomicAdd(&bkt[((x - base) >> shift) & key_mask], 1)] = x;
    }
    __syncwarp();
    // bkt[b] is now the end of bucket b
    if (maxb > kBucketSortMax) {
        group_sort<32>(buf, count);
        return;
    }
    for (int b = lane; b < nb; b += 32) {
        const int e = bkt[b], s0 = b ? bkt[b - 1] : 0;
        for (int i = s0 + 1; i < e; ++i) {
            const uint32_t x = buf[i];
            int k = i - 1;
            while (k >= s0 && buf[k] > x) {
                buf[k + 1] = buf[k];
                --k;
            }
            buf[k + 1] = x;
        }
    }
    __syncwarp();
}

}  // namespace hyperim
