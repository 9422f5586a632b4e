// Device-side random stream and distribution draws of HyperIM's RR generation.
//
// Written for sm_103a. Floating point here is IEEE double through explicit round-to-nearest
// intrinsics (__dadd_rn, __dmul_rn, __ddiv_rn), never contracted, so every CDF threshold is the
// exact sequence of correctly rounded operations stated in the comments.
#pragma once
#include <cstdint>

namespace hyperim {

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64 multiplies
// whose halves are xored with the other counter words and the key; the key is bumped by the
// Weyl constants (golden ratio, sqrt(3)-1) between rounds.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Counter layout of one keyed stream (words consumed in order, four per Philox block):
//   x = RR index j within its stratum
//   y = pool tag << 24 | stratum field << 16 | block (block < 2^16)
//   z = popped vertex mu, or 0xFFFFFFFF for the root draw
//   w = layer index i (1-based), or 0 for the root draw
struct WordStream {
    uint32_t k0, k1, x, ybase, z, w;
    uint32_t cached_block;
    uint4 buf;
    bool overflow;

    __device__ __forceinline__ void init(uint64_t seed, uint32_t j, uint32_t ybase_, uint32_t z_,
                                         uint32_t w_) {
        k0 = (uint32_t)seed;
        k1 = (uint32_t)(seed >> 32);
        x = j; ybase = ybase_; z = z_; w = w_;
        cached_block = 0xFFFFFFFFu;
        overflow = false;
    }
    __device__ __forceinline__ uint32_t word(uint32_t idx) {
        const uint32_t block = idx >> 2;
        if (block > 0xFFFFu) { overflow = true; return 0u; }
        if (block != cached_block) {
            buf = philox10(make_uint4(x, ybase | block, z, w), k0, k1);
            cached_block = block;
        }
        const uint32_t lane = idx & 3u;
        return lane == 0 ? buf.x : lane == 1 ? buf.y : lane == 2 ? buf.z : buf.w;
    }
};

__device__ __forceinline__ uint32_t stream_ybase(uint32_t tag, uint32_t sfield) {
    return ((tag & 0xFFu) << 24) | ((sfield & 0xFFu) << 16);
}

// floor(cum * 2^32) for cum >= 0 (exact power-of-two scaling, truncation)
__device__ __forceinline__ uint64_t cdf_thr(double cum) {
    return __double2ull_rz(__dmul_rn(cum, 4294967296.0));
}

// exp(-x) for 0 < x <= 64 by scaling and squaring (Moler & Van Loan, "Nineteen dubious ways to
// compute the exponential of a matrix"): y = x / 2^s <= 2^-5, degree-10 Taylor polynomial of
// exp(-y) in Horner form (terms 10 down to 1), then s squarings.
__device__ __forceinline__ double exp_neg(double x) {
    int s = 0;
    double y = x;
    while (y > 0.03125) {
        y = __dmul_rn(y, 0.5);
        ++s;
    }
    double e = 1.0;
    for (int j = 10; j >= 1; --j) e = __dadd_rn(1.0, __ddiv_rn(__dmul_rn(-y, e), (double)j));
    for (int i = 0; i < s; ++i) e = __dmul_rn(e, e);
    return e;
}

constexpr uint64_t kPOne = 4294967296ull;  // threshold meaning p = 1

// P(h = 0) threshold floor(q^n 2^32) for the Binomial strategy (q = 1 - p, n multiplications).
__device__ __forceinline__ uint64_t binomial_t0(uint32_t n, uint64_t thr) {
    const double p = __dmul_rn((double)thr, 0x1p-32);
    const double q = __dsub_rn(1.0, p);
    double P = 1.0;
    for (uint32_t i = 0; i < n; ++i) P = __dmul_rn(P, q);
    return cdf_thr(P);
}

// Binomial(n, p) by inversion of one word: least h with w0 < floor(CDF(h) 2^32), else n.
// pmf: P(0) = q^n, P(h+1) = ((P(h) (n-h)) / (h+1)) r with r = p/q (Sec. 3.1.3, Binomial strategy).
static __device__ __noinline__ uint32_t binomial_h(uint32_t n, uint64_t thr, uint32_t w0) {
    if (thr == 0 || n == 0) return 0;
    if (thr >= kPOne) return n;
    const double p = __dmul_rn((double)thr, 0x1p-32);
    const double q = __dsub_rn(1.0, p);
    double P = 1.0;
    for (uint32_t i = 0; i < n; ++i) P = __dmul_rn(P, q);
    const double r = __ddiv_rn(p, q);
    double cum = P;
    if ((uint64_t)w0 < cdf_thr(cum)) return 0;
    for (uint32_t h = 0; h + 1 < n; ++h) {
        P = __dmul_rn(__ddiv_rn(__dmul_rn(P, (double)(n - h)), (double)(h + 1)), r);
        if (P == 0.0) return n;  // the CDF is constant from here on
        cum = __dadd_rn(cum, P);
        if ((uint64_t)w0 < cdf_thr(cum)) return h + 1;
    }
    return n;
}

// lambda = n p (one rounding); number of Poisson parts c = ceil(lambda / 64) (>= 1).
__device__ __forceinline__ double poisson_lambda(uint32_t n, uint64_t thr) {
    return __dmul_rn((double)n, __dmul_rn((double)thr, 0x1p-32));
}
__device__ __forceinline__ uint32_t poisson_parts(double lam) {
    const double q = __dmul_rn(lam, 0.015625);
    uint32_t c = (uint32_t)q;
    if ((double)c < q) ++c;
    return c == 0 ? 1u : c;
}
__device__ __forceinline__ double poisson_part_lambda(double lam, uint32_t c) {
    return c == 1 ? lam : __ddiv_rn(lam, (double)c);
}

// One Poisson(lam) part by inversion: P(0) = exp(-lam), P(h) = (P(h-1) lam) / h, stopped at n.
static __device__ __noinline__ uint32_t poisson_part(double lam, uint32_t n, uint32_t w) {
    double P = exp_neg(lam);
    double cum = P;
    if ((uint64_t)w < cdf_thr(cum)) return 0;
    for (uint32_t h = 1; h < n; ++h) {
        P = __ddiv_rn(__dmul_rn(P, lam), (double)h);
        if (P == 0.0) return n;
        cum = __dadd_rn(cum, P);
        if ((uint64_t)w < cdf_thr(cum)) return h;
    }
    return n;
}

// Thresholds T_0, T_1, ... of one inversion -- Binomial(n, p) as in binomial_h, or one
// Poisson(lam) part as in poisson_part -- computed by the same IEEE operation sequence and capped
// at 2^32 - 1. The table stops after T_{n-1}, where a pmf term underflows (the CDF is constant
// from there), once T_h >= kTailStop (the remaining mass is below 2^-16) or at cap entries.
// Returns the number of entries; writes them to T unless T is null. A draw w with w < T_k for a
// least k in the table has h = k; w >= the last entry means h = n if the table has n entries,
// otherwise the inversion itself must decide.
constexpr uint32_t kTailStop = 0xFFFF0000u;
constexpr uint32_t kTableCap = 64;

__device__ __forceinline__ uint32_t cdf_table(uint32_t n, uint64_t thr, bool poisson, double lam,
                                              uint32_t cap, uint32_t* T) {
    double P, r = 0.0;
    if (poisson) {
        P = exp_neg(lam);
    } else {
        const double p = __dmul_rn((double)thr, 0x1p-32);
        const double q = __dsub_rn(1.0, p);
        P = 1.0;
        for (uint32_t i = 0; i < n; ++i) P = __dmul_rn(P, q);
        r = __ddiv_rn(p, q);
    }
    double cum = P;
    uint32_t L = 0;
    for (uint32_t k = 0; k < n && L < cap; ++k) {
        if (k > 0) {
            P = poisson ? __ddiv_rn(__dmul_rn(P, lam), (double)k)
                        : __dmul_rn(__ddiv_rn(__dmul_rn(P, (double)(n - (k - 1))), (double)k), r);
            if (P == 0.0) break;
            cum = __dadd_rn(cum, P);
        }
        const uint64_t t = cdf_thr(cum);
        const uint32_t tk = (uint32_t)(t > 0xFFFFFFFFull ? 0xFFFFFFFFull : t);
        if (T) T[L] = tk;
        ++L;
        if (tk >= kTailStop) break;
    }
    return L;
}

// least k < L with w < T[k] (T non-decreasing), or L
__device__ __forceinline__ uint32_t table_find(const uint32_t* __restrict__ T, uint32_t L, uint32_t w) {
    uint32_t lo = 0, hi = L;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (w < T[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// P(h = 0) threshold for the (unsplit or first split) Poisson strategy: the whole draw is 0 iff
// every part draws 0; with one part this is w0 < floor(exp(-lam) 2^32).
__device__ __forceinline__ uint64_t poisson_t0(uint32_t n, uint64_t thr) {
    const double lam = poisson_lambda(n, thr);
    const uint32_t c = poisson_parts(lam);
    return cdf_thr(exp_neg(poisson_part_lambda(lam, c)));
}

}  // namespace hyperim
