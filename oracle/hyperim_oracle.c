/*
 * HyperIM CPU oracle -- TEST INFRASTRUCTURE ONLY (see hyperim_oracle.h).
 *
 * Plain, slow, single-threaded. Floating point is IEEE double with no contraction
 * (-ffp-contract=off) and only + - * / sqrt in a fixed order wherever a result must match the
 * CUDA library bit for bit. Each function names the passage of the paper (or the published
 * definition) it restates.
 *
 * Readings of the paper that this file implements (the paper is silent or self-contradictory
 * on these points):
 *   - layers of A(mu) are keyed by w(mu,nu), the number of hyperedges shared; L_1 holds the
 *     largest w (Sec. 3.1.1 rules (i)-(ii)); members of a layer are ordered by ascending id;
 *   - the per-vertex probability is p = P(L_i)/n(L_i) with P(L_i) = 1/(i ln(l+1)) clamped to 1
 *     (Sec. 3.1.1; Lemma 1's sum-to-at-most-one claim does not hold for l = 1);
 *   - Binomial(n_i, p) and Poisson(n_i p) draws use the per-vertex p (Sec. 3.1.3);
 *   - h members are picked from all of L_i; an already-activated pick is skipped (Alg. 3);
 *   - theta_max uses delta inside both logarithms, unsquared, as printed in Eq. (equation-max);
 *     theta_0 = theta_max eps^2 k / n (Sec. 4.3 text); the stop test is alpha >= 1-1/e-eps
 *     (Alg. 4), with at most ceil(log2(theta_max/theta_0)) doublings;
 *   - R1 and R2 are independent, equally sized pools; the upper bound comes from R1
 *     (Eq. upper_6 with p_max = 1), the lower bound from R2 (Sec. 4.2);
 *   - roots are stratified by l_mu (capped at 15) with proportional allocation
 *     n_s = ceil(theta |V_s| / n) and estimator weights |V_s| / n_s.
 */
#include "hyperim_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ===================================== Philox4x32-10 ========================================
 * Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11.
 * Ten rounds of the multiply/xor S-box on a 4-word counter with a 2-word Weyl-incremented key.
 */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u; /* golden ratio */
            k1 += 0xBB67AE85u; /* sqrt(3) - 1 */
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A keyed word stream: counter (c0, c1 | block, c2, c3), words consumed in order. */
typedef struct {
    uint32_t key[2];
    uint32_t c0, c1base, c2, c3;
    uint32_t next;      /* index of the next word */
    uint32_t buf[4];
    uint32_t buf_block; /* block held in buf, or UINT32_MAX */
    int overflow;
} word_stream;

static void ws_init(word_stream* w, uint64_t seed, uint32_t c0, uint32_t c1base, uint32_t c2,
                    uint32_t c3) {
    w->key[0] = (uint32_t)seed;
    w->key[1] = (uint32_t)(seed >> 32);
    w->c0 = c0; w->c1base = c1base; w->c2 = c2; w->c3 = c3;
    w->next = 0;
    w->buf_block = UINT32_MAX;
    w->overflow = 0;
}

static uint32_t ws_word(word_stream* w, uint32_t idx) {
    uint32_t block = idx >> 2;
    if (block > 0xFFFFu) { w->overflow = 1; return 0; }
    if (block != w->buf_block) {
        uint32_t ctr[4] = {w->c0, w->c1base | block, w->c2, w->c3};
        or_philox4x32_10(ctr, w->key, w->buf);
        w->buf_block = block;
    }
    return w->buf[idx & 3];
}

static uint32_t ws_next(word_stream* w) { return ws_word(w, w->next++); }

/* c1 field: pool tag in bits 24..31, stratum in bits 16..23, Philox block in bits 0..15. */
static uint32_t c1_field(uint32_t tag, uint32_t sfield) {
    return ((tag & 0xFFu) << 24) | ((sfield & 0xFFu) << 16);
}

/* ===================================== exp(-x), 0 < x <= 64 =================================
 * Scaling and squaring with a truncated Taylor series (Moler & Van Loan, "Nineteen dubious ways
 * to compute the exponential of a matrix", method 3): halve x until it is at most 2^-5, evaluate
 * the degree-10 Taylor polynomial of exp(-y) in Horner form, then square s times.
 */
double or_exp_neg(double x) {
    int s = 0;
    double y = x;
    while (y > 0.03125) {
        y = y * 0.5;
        s++;
    }
    double e = 1.0;
    for (int j = 10; j >= 1; --j) e = 1.0 + ((-y) * e) / (double)j;
    for (int i = 0; i < s; ++i) e = e * e;
    return e;
}

static uint64_t cdf_threshold(double cum) { return (uint64_t)(cum * 4294967296.0); }

/* ============================ Binomial-based strategy (Sec. 3.1.3) ===========================
 * h ~ Binomial(n, p) by inversion of one uniform 32-bit word w0: h is the least h with
 * w0 < floor(CDF(h) 2^32), else n. pmf by the recurrence P(h+1) = P(h) (n-h)/(h+1) p/q from
 * P(0) = q^n.
 */
uint32_t or_binomial_h(uint32_t n, uint64_t thr, uint32_t w0) {
    if (thr == 0 || n == 0) return 0;
    if (thr >= OR_P_ONE) return n;
    double p = (double)thr * 0x1p-32;
    double q = 1.0 - p;
    double P = 1.0;
    for (uint32_t i = 0; i < n; ++i) P = P * q;
    double r = p / q;
    double cum = P;
    if ((uint64_t)w0 < cdf_threshold(cum)) return 0;
    for (uint32_t h = 0; h + 1 < n; ++h) {
        P = ((P * (double)(n - h)) / (double)(h + 1)) * r;
        if (P == 0.0) return n; /* the CDF no longer moves: the search ends at n */
        cum = cum + P;
        if ((uint64_t)w0 < cdf_threshold(cum)) return h + 1;
    }
    return n;
}

/* ============================ Poisson-based strategy (Sec. 3.1.3) ============================
 * h ~ Poisson(lambda), lambda = n p, truncated to [0, n]. For lambda > 64 the draw is the sum of
 * c = ceil(lambda/64) independent Poisson(lambda/c) parts (one word each), each by inversion
 * from P(0) = exp(-lambda'), P(h+1) = P(h) lambda'/(h+1), each stopped at n.
 */
static double poisson_lambda(uint32_t n, uint64_t thr) {
    double p = (double)thr * 0x1p-32;
    return (double)n * p;
}

uint32_t or_poisson_parts(uint32_t n, uint64_t thr) {
    double lam = poisson_lambda(n, thr);
    double q = lam * 0.015625;
    uint32_t c = (uint32_t)q;
    if ((double)c < q) c++;
    if (c == 0) c = 1;
    return c;
}

static uint32_t poisson_part(double lam, uint32_t n, uint32_t w) {
    double P = or_exp_neg(lam);
    double cum = P;
    if ((uint64_t)w < cdf_threshold(cum)) return 0;
    for (uint32_t h = 1; h < n; ++h) {
        P = (P * lam) / (double)h;
        if (P == 0.0) return n;
        cum = cum + P;
        if ((uint64_t)w < cdf_threshold(cum)) return h;
    }
    return n;
}

uint32_t or_poisson_h(uint32_t n, uint64_t thr, const uint32_t* words, uint32_t nwords,
                      uint32_t* used) {
    if (thr == 0 || n == 0) { *used = 0; return 0; }
    if (thr >= OR_P_ONE) { *used = 0; return n; }
    uint32_t c = or_poisson_parts(n, thr);
    double lam = poisson_lambda(n, thr);
    double part = (c == 1) ? lam : lam / (double)c;
    uint64_t h = 0;
    for (uint32_t i = 0; i < c && i < nwords; ++i) h += poisson_part(part, n, words[i]);
    *used = c;
    return h > n ? n : (uint32_t)h;
}

/* ===================================== incidence store ====================================== */
struct or_graph {
    int32_t n, m;
    int model;
    uint64_t uniform_thr;
    int64_t* he_off;   /* m+1 */
    int32_t* he_mem;   /* members, each hyperedge sorted ascending, duplicates removed */
    int64_t* v_off;    /* n+1 */
    int32_t* v_he;     /* hyperedges of each vertex, ascending */
    int32_t* deg;      /* |A(v)| */
    int32_t* nlayers;  /* l_v */
    int64_t* prof_off; /* n+1 */
    uint32_t* lay_w;
    uint32_t* lay_n;
    uint64_t* lay_thr;
    int32_t* stratum;  /* min(l_v, 15) */
    int32_t vs_size[OR_NSTRATA];
    int32_t* vs[OR_NSTRATA];
    int32_t* all_v;    /* 0..n-1, the single stratum of plain roots */
    double theta_lstar;
    /* scratch (single-threaded) */
    int32_t* cnt;      /* n, zero between uses */
    uint8_t* seen;     /* n, zero between uses */
    int32_t* nb;       /* distinct neighbours */
    uint64_t* keys;
    int64_t nb_cap;
    int worker;        /* 1: a worker view (or_graph_worker) that owns only its scratch */
};

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}
static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

/* A(mu) (Sec. 3.1.1): the vertices sharing a hyperedge with mu, with w(mu,nu) the number of
 * shared hyperedges. Returns the distinct neighbours sorted by (w descending, id ascending) in
 * g->nb and their weights via g->cnt (caller must call nbhd_release). */
/* bytes of the 32-byte sectors that the byte range [a, a + len) overlaps */
static uint64_t sector_bytes(uint64_t a, uint64_t len) {
    if (len == 0) return 0;
    return 32u * ((a + len - 1) / 32u - a / 32u + 1u);
}

/* the cost-model bytes of one pop of mu (see or_stats.bytes_rr): its profile entries, and when
 * it materialises A(mu), v_he(mu) and every hyperedge of mu (two offsets plus its members) */
static uint64_t pop_bytes(const or_graph* g, int32_t mu, int materialises) {
    uint64_t b = sector_bytes(12u * (uint64_t)g->prof_off[mu],
                              12u * (uint64_t)(g->prof_off[mu + 1] - g->prof_off[mu]));
    if (!materialises) return b;
    b += sector_bytes(4u * (uint64_t)g->v_off[mu], 4u * (uint64_t)(g->v_off[mu + 1] - g->v_off[mu]));
    for (int64_t x = g->v_off[mu]; x < g->v_off[mu + 1]; ++x) {
        const int32_t he = g->v_he[x];
        b += 8u + sector_bytes(4u * (uint64_t)g->he_off[he], 4u * (uint64_t)(g->he_off[he + 1] - g->he_off[he]));
    }
    return b;
}

static int64_t nbhd_build(or_graph* g, int32_t mu, uint64_t* mat_members) {
    int64_t k = 0;
    uint64_t reads = 0;
    for (int64_t e = g->v_off[mu]; e < g->v_off[mu + 1]; ++e) {
        int32_t he = g->v_he[e];
        for (int64_t x = g->he_off[he]; x < g->he_off[he + 1]; ++x) {
            int32_t nu = g->he_mem[x];
            reads++;
            if (nu == mu) continue;
            if (g->cnt[nu]++ == 0) g->nb[k++] = nu;
        }
    }
    for (int64_t i = 0; i < k; ++i)
        g->keys[i] = ((uint64_t)(0xFFFFFFFFu - (uint32_t)g->cnt[g->nb[i]]) << 32) |
                     (uint32_t)g->nb[i];
    qsort(g->keys, (size_t)k, sizeof(uint64_t), cmp_u64);
    for (int64_t i = 0; i < k; ++i) g->nb[i] = (int32_t)(uint32_t)g->keys[i];
    if (mat_members) *mat_members += reads;
    return k;
}

/* The distinct neighbours of mu (unsorted) with w(mu,nu) in g->cnt (caller must release). */
static int64_t nbhd_count(or_graph* g, int32_t mu) {
    int64_t k = 0;
    for (int64_t e = g->v_off[mu]; e < g->v_off[mu + 1]; ++e) {
        int32_t he = g->v_he[e];
        for (int64_t x = g->he_off[he]; x < g->he_off[he + 1]; ++x) {
            int32_t nu = g->he_mem[x];
            if (nu == mu) continue;
            if (g->cnt[nu]++ == 0) g->nb[k++] = nu;
        }
    }
    return k;
}

static void nbhd_release(or_graph* g, int64_t k) {
    for (int64_t i = 0; i < k; ++i) g->cnt[g->nb[i]] = 0;
}

/* Threshold floor(p 2^32) of a member of layer i (1-based) of A(mu), for the three activation
 * settings: one p for every co-member pair; the weighted cascade p = 1/deg(mu); and the paper's
 * layer setting p = P(L_i)/n(L_i), P(L_i) = 1/(i ln(l+1)) (Sec. 3.1.1), clamped to 1. */
static uint64_t layer_threshold(const or_graph* g, int32_t deg, int32_t l, int32_t i,
                                uint32_t n_i) {
    switch (g->model) {
    case OR_MODEL_UNIFORM_PAIR:
        return g->uniform_thr;
    case OR_MODEL_WC:
        if (deg <= 1) return OR_P_ONE;
        return 4294967296ull / (uint64_t)deg;
    default: {
        double PL = 1.0 / ((double)i * log((double)l + 1.0));
        double pd = PL / (double)n_i;
        if (pd >= 1.0) return OR_P_ONE;
        return (uint64_t)(pd * 4294967296.0);
    }
    }
}

int or_graph_build(int32_t n, int32_t m, const int32_t* he_off, const int32_t* he_mem, int model,
                   uint64_t uniform_thr, or_graph** out) {
    if (n <= 0 || m < 0 || !he_off || (m > 0 && !he_mem) || !out) return OR_EINVAL;
    if (model < 0 || model > 2 || uniform_thr > OR_P_ONE) return OR_EINVAL;
    if (he_off[0] != 0) return OR_EINVAL;
    for (int32_t e = 0; e < m; ++e)
        if (he_off[e + 1] < he_off[e]) return OR_EINVAL;
    int64_t nnz_in = he_off[m];
    for (int64_t x = 0; x < nnz_in; ++x)
        if (he_mem[x] < 0 || he_mem[x] >= n) return OR_EINVAL;

    or_graph* g = (or_graph*)calloc(1, sizeof(or_graph));
    if (!g) return OR_ENOMEM;
    g->n = n; g->m = m; g->model = model; g->uniform_thr = uniform_thr;
    /* normalise: sort each member list, drop repeated ids (a hyperedge is a vertex set) */
    g->he_off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)m + 1));
    g->he_mem = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz_in > 0 ? nnz_in : 1));
    int64_t w = 0;
    g->he_off[0] = 0;
    for (int32_t e = 0; e < m; ++e) {
        int64_t b = he_off[e], len = he_off[e + 1] - he_off[e];
        memcpy(g->he_mem + w, he_mem + b, sizeof(int32_t) * (size_t)len);
        qsort(g->he_mem + w, (size_t)len, sizeof(int32_t), cmp_i32);
        int64_t u = 0;
        for (int64_t x = 0; x < len; ++x)
            if (u == 0 || g->he_mem[w + x] != g->he_mem[w + u - 1]) g->he_mem[w + u++] = g->he_mem[w + x];
        w += u;
        g->he_off[e + 1] = w;
    }
    int64_t nnz = w;
    /* vertex -> hyperedge lists (ascending hyperedge id) */
    g->v_off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    g->v_he = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    for (int64_t x = 0; x < nnz; ++x) g->v_off[g->he_mem[x] + 1]++;
    for (int32_t v = 0; v < n; ++v) g->v_off[v + 1] += g->v_off[v];
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    for (int32_t v = 0; v < n; ++v) cur[v] = g->v_off[v];
    for (int32_t e = 0; e < m; ++e)
        for (int64_t x = g->he_off[e]; x < g->he_off[e + 1]; ++x) g->v_he[cur[g->he_mem[x]]++] = e;
    free(cur);

    g->cnt = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    g->seen = (uint8_t*)calloc((size_t)n, 1);
    g->nb_cap = n;
    g->nb = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    g->keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    g->deg = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    g->nlayers = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    g->stratum = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    g->prof_off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!g->he_off || !g->he_mem || !g->v_off || !g->v_he || !g->cnt || !g->seen || !g->nb ||
        !g->keys || !g->deg || !g->nlayers || !g->stratum || !g->prof_off) {
        or_graph_free(g);
        return OR_ENOMEM;
    }
    /* layer profile (Sec. 3.1.1): the number of distinct neighbours per multiplicity w; the
     * distinct w values in descending order are the layers. Pass 1 counts layers, pass 2 stores
     * (w_i, n_i, threshold). */
    int32_t maxdh = 0;
    for (int32_t v = 0; v < n; ++v) {
        int32_t d = (int32_t)(g->v_off[v + 1] - g->v_off[v]);
        if (d > maxdh) maxdh = d;
    }
    int64_t* hist = (int64_t*)calloc((size_t)maxdh + 2, sizeof(int64_t));
    if (!hist) { or_graph_free(g); return OR_ENOMEM; }
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            int64_t L = g->prof_off[n];
            g->lay_w = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(L > 0 ? L : 1));
            g->lay_n = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(L > 0 ? L : 1));
            g->lay_thr = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(L > 0 ? L : 1));
            if (!g->lay_w || !g->lay_n || !g->lay_thr) { free(hist); or_graph_free(g); return OR_ENOMEM; }
        }
        for (int32_t v = 0; v < n; ++v) {
            int64_t k = nbhd_count(g, v);
            int32_t dh = (int32_t)(g->v_off[v + 1] - g->v_off[v]);
            for (int64_t i = 0; i < k; ++i) hist[g->cnt[g->nb[i]]]++;
            nbhd_release(g, k);
            int32_t l = 0;
            int64_t base = g->prof_off[v];
            for (int32_t w = dh; w >= 1; --w) {
                if (hist[w] == 0) continue;
                if (pass == 1) {
                    g->lay_w[base + l] = (uint32_t)w;
                    g->lay_n[base + l] = (uint32_t)hist[w];
                }
                l++;
                hist[w] = 0;
            }
            if (pass == 0) {
                g->deg[v] = (int32_t)k;
                g->nlayers[v] = l;
                g->prof_off[v + 1] = g->prof_off[v] + l;
            }
        }
    }
    free(hist);
    double lsum = 0.0;
    for (int32_t v = 0; v < n; ++v) {
        int32_t l = g->nlayers[v];
        int64_t base = g->prof_off[v];
        for (int32_t i = 0; i < l; ++i)
            g->lay_thr[base + i] = layer_threshold(g, g->deg[v], l, i + 1, g->lay_n[base + i]);
        g->stratum[v] = l < OR_NSTRATA - 1 ? l : OR_NSTRATA - 1;
        if (l > 0) lsum += (double)l / log((double)l + 1.0);
    }
    g->theta_lstar = lsum / (double)n; /* Thm 2: theta(l*) = (1/|V|) sum l/ln(l+1) */
    /* root strata: V_s in ascending id order */
    for (int32_t v = 0; v < n; ++v) g->vs_size[g->stratum[v]]++;
    for (int s = 0; s < OR_NSTRATA; ++s) {
        g->vs[s] = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->vs_size[s] > 0 ? g->vs_size[s] : 1));
        g->vs_size[s] = 0;
    }
    for (int32_t v = 0; v < n; ++v) {
        int s = g->stratum[v];
        g->vs[s][g->vs_size[s]++] = v;
    }
    g->all_v = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t v = 0; v < n; ++v) g->all_v[v] = v;
    *out = g;
    return OR_OK;
}

void or_graph_free(or_graph* g) {
    if (!g) return;
    if (g->worker) {
        free(g->cnt); free(g->seen); free(g->nb); free(g->keys);
        free(g);
        return;
    }
    free(g->he_off); free(g->he_mem); free(g->v_off); free(g->v_he); free(g->deg);
    free(g->nlayers); free(g->prof_off); free(g->lay_w); free(g->lay_n); free(g->lay_thr);
    free(g->stratum); free(g->all_v); free(g->cnt); free(g->seen); free(g->nb); free(g->keys);
    for (int s = 0; s < OR_NSTRATA; ++s) free(g->vs[s]);
    free(g);
}

/* A second view of g for another thread: the same (read-only) graph arrays, its own scratch.
 * Freed with or_graph_free before g. */
int or_graph_worker(const or_graph* g, or_graph** out) {
    or_graph* w = (or_graph*)malloc(sizeof(or_graph));
    if (!w) return OR_ENOMEM;
    memcpy(w, g, sizeof(or_graph));
    w->worker = 1;
    w->cnt = (int32_t*)calloc((size_t)g->n, sizeof(int32_t));
    w->seen = (uint8_t*)calloc((size_t)g->n, 1);
    w->nb_cap = g->n;
    w->nb = (int32_t*)malloc(sizeof(int32_t) * (size_t)g->n);
    w->keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)g->n);
    if (!w->cnt || !w->seen || !w->nb || !w->keys) {
        or_graph_free(w);
        return OR_ENOMEM;
    }
    *out = w;
    return OR_OK;
}

int32_t or_graph_n(const or_graph* g) { return g->n; }
int64_t or_graph_nnz(const or_graph* g) { return g->he_off[g->m]; }
int32_t or_graph_he_size(const or_graph* g, int32_t he) {
    return (int32_t)(g->he_off[he + 1] - g->he_off[he]);
}
int32_t or_graph_dh(const or_graph* g, int32_t v) { return (int32_t)(g->v_off[v + 1] - g->v_off[v]); }
int32_t or_graph_deg(const or_graph* g, int32_t v) { return g->deg[v]; }
int32_t or_graph_nlayers(const or_graph* g, int32_t v) { return g->nlayers[v]; }
int32_t or_graph_stratum(const or_graph* g, int32_t v) { return g->stratum[v]; }
int32_t or_graph_stratum_size(const or_graph* g, int32_t s) { return g->vs_size[s]; }
double or_graph_theta_lstar(const or_graph* g) { return g->theta_lstar; }

int or_graph_layer(const or_graph* g, int32_t v, int32_t i, uint32_t* w, uint32_t* n_i,
                   uint64_t* thr) {
    if (v < 0 || v >= g->n || i < 1 || i > g->nlayers[v]) return OR_EINVAL;
    int64_t x = g->prof_off[v] + i - 1;
    *w = g->lay_w[x]; *n_i = g->lay_n[x]; *thr = g->lay_thr[x];
    return OR_OK;
}

int64_t or_graph_layer_members(const or_graph* g, int32_t v, int32_t i, int32_t* out, int64_t cap) {
    if (v < 0 || v >= g->n || i < 1 || i > g->nlayers[v]) return OR_EINVAL;
    or_graph* gm = (or_graph*)g;
    int64_t k = nbhd_build(gm, v, NULL);
    int32_t li = 0;
    int64_t c = 0;
    for (int64_t x = 0; x < k; ++x) {
        if (x > 0 && gm->cnt[gm->nb[x]] != gm->cnt[gm->nb[x - 1]]) li++;
        if (li == i - 1) {
            if (c < cap) out[c] = gm->nb[x];
            c++;
        }
    }
    nbhd_release(gm, k);
    return c;
}

/* ================================ allocation and root draw ==================================
 * Roots are drawn uniformly from a stratum V_s (Alg. 3 first step, restricted to the stratum).
 * Stratified roots: strata by s(mu) = min(l_mu, 15); stratum s receives n_s = ceil(theta |V_s|/n)
 * RR sets (at least one per nonempty stratum, monotone in theta). Plain roots: one stratum V.
 */
int or_allocate(const or_graph* g, int root_mode, uint64_t theta, uint64_t n_s[OR_NSTRATA]) {
    memset(n_s, 0, sizeof(uint64_t) * OR_NSTRATA);
    if (root_mode == OR_ROOTS_PLAIN) {
        n_s[0] = theta;
        return OR_OK;
    }
    if (root_mode != OR_ROOTS_STRATIFIED) return OR_EINVAL;
    for (int s = 0; s < OR_NSTRATA; ++s) {
        if (g->vs_size[s] == 0 || theta == 0) continue;
        unsigned __int128 num = (unsigned __int128)theta * (uint64_t)g->vs_size[s];
        n_s[s] = (uint64_t)((num + (uint64_t)g->n - 1) / (uint64_t)g->n);
    }
    return OR_OK;
}

static uint32_t stratum_field(int root_mode, uint32_t stratum) {
    return root_mode == OR_ROOTS_PLAIN ? 0xFFu : stratum;
}

static const int32_t* stratum_list(const or_graph* g, int root_mode, uint32_t s, int32_t* size) {
    if (root_mode == OR_ROOTS_PLAIN) { *size = g->n; return g->all_v; }
    *size = g->vs_size[s];
    return g->vs[s];
}

int32_t or_root(const or_graph* g, uint64_t seed, uint32_t tag, int root_mode, uint32_t stratum,
                uint32_t j) {
    int32_t size;
    const int32_t* list = stratum_list(g, root_mode, stratum, &size);
    if (size <= 0) return -1;
    word_stream ws;
    ws_init(&ws, seed, j, c1_field(tag, stratum_field(root_mode, stratum)), 0xFFFFFFFFu, 0u);
    uint32_t w0 = ws_next(&ws);
    uint64_t idx = ((uint64_t)w0 * (uint64_t)(uint32_t)size) >> 32;
    return list[idx];
}

/* ============================== RR-set generation (Algorithm 3) =============================
 * Reverse BFS from the root. Each popped mu: for every layer i of A(mu), draw the number h of
 * activators (Binomial if n(L_i) <= 20, else Poisson; Sec. 3.1.3), then pick h distinct members
 * of L_i by sequential selection from the remainder (Sec. 3.1.3): at step r a word x gives
 * a = floor(x (n_i - r) / 2^32) and the pick is the a-th (0-based) not-yet-picked position of
 * L_i in ascending id order. Picks already in R are skipped; new ones join R and the queue.
 * Draws are keyed by (RR, popped vertex, layer), so R does not depend on the pop order.
 */
typedef struct {
    int32_t* v;
    int64_t len, cap;
} ivec;

static int ivec_push(ivec* a, int32_t x) {
    if (a->len == a->cap) {
        int64_t nc = a->cap ? a->cap * 2 : 64;
        int32_t* nv = (int32_t*)realloc(a->v, sizeof(int32_t) * (size_t)nc);
        if (!nv) return OR_ENOMEM;
        a->v = nv; a->cap = nc;
    }
    a->v[a->len++] = x;
    return OR_OK;
}

/* the a-th (0-based) position of [0, n) not in the sorted list sel[0..r) */
static uint32_t nth_unpicked(const uint32_t* sel, uint32_t r, uint32_t a) {
    uint32_t idx = a;
    for (uint32_t t = 0; t < r; ++t) {
        if (sel[t] <= idx) idx++;
        else break;
    }
    return idx;
}

static void sorted_insert(uint32_t* sel, uint32_t r, uint32_t x) {
    uint32_t t = r;
    while (t > 0 && sel[t - 1] > x) { sel[t] = sel[t - 1]; t--; }
    sel[t] = x;
}

static int rr_pop(or_graph* g, uint64_t seed, uint32_t j, uint32_t c1base, int strategy,
                  int32_t mu, ivec* R, or_stats* st, uint32_t** selbuf, uint32_t* selcap) {
    /* A(mu) and its layers, from the incidence lists (never from a stored expansion) */
    uint64_t reads = 0;
    int64_t k = nbhd_build(g, mu, &reads);
    int32_t l = 0;
    for (int64_t i = 0; i < k; ++i)
        if (i == 0 || g->cnt[g->nb[i]] != g->cnt[g->nb[i - 1]]) l++;
    st->pops++;
    st->layers_seen += (uint64_t)l;
    int any = 0;
    int rc = OR_OK;
    int64_t start = 0;
    for (int32_t i = 1; i <= l; ++i) {
        int64_t end = start;
        while (end < k && g->cnt[g->nb[end]] == g->cnt[g->nb[start]]) end++;
        uint32_t n_i = (uint32_t)(end - start);
        const int32_t* Li = g->nb + start;
        uint64_t thr = layer_threshold(g, (int32_t)k, l, i, n_i);
        word_stream ws;
        ws_init(&ws, seed, j, c1base, (uint32_t)mu, (uint32_t)i);
        uint32_t h = 0;
        if (thr == 0) {
            h = 0;
        } else if (thr >= OR_P_ONE) {
            h = n_i;
        } else if (n_i <= 20 || strategy == OR_STRAT_BINOMIAL_ONLY) {
            st->draws++;
            h = or_binomial_h(n_i, thr, ws_next(&ws));
        } else {
            st->draws++;
            uint32_t c = or_poisson_parts(n_i, thr);
            double lam = poisson_lambda(n_i, thr);
            double part = (c == 1) ? lam : lam / (double)c;
            uint64_t hh = 0;
            for (uint32_t t = 0; t < c; ++t) hh += poisson_part(part, n_i, ws_next(&ws));
            h = hh > n_i ? n_i : (uint32_t)hh;
        }
        if (h > 0) any = 1;
        st->selected += h;
        if (h == n_i) {
            for (uint32_t x = 0; x < n_i; ++x) {
                int32_t nu = Li[x];
                if (!g->seen[nu]) { g->seen[nu] = 1; if ((rc = ivec_push(R, nu))) goto done; }
            }
        } else if (h > 0) {
            if (h > *selcap) {
                uint32_t* nb2 = (uint32_t*)realloc(*selbuf, sizeof(uint32_t) * h);
                if (!nb2) { rc = OR_ENOMEM; goto done; }
                *selbuf = nb2; *selcap = h;
            }
            uint32_t* sel = *selbuf;
            for (uint32_t r = 0; r < h; ++r) {
                uint32_t x = ws_next(&ws);
                uint32_t a = (uint32_t)(((uint64_t)x * (uint64_t)(n_i - r)) >> 32);
                uint32_t idx = nth_unpicked(sel, r, a);
                sorted_insert(sel, r, idx);
                int32_t nu = Li[idx];
                if (!g->seen[nu]) { g->seen[nu] = 1; if ((rc = ivec_push(R, nu))) goto done; }
            }
        }
        if (ws.overflow) { rc = OR_EOVERFLOW; goto done; }
        start = end;
    }
    if (any) {
        st->mats++;
        st->mat_he += (uint64_t)(g->v_off[mu + 1] - g->v_off[mu]);
        st->mat_members += reads;
    }
    st->bytes_rr += pop_bytes(g, mu, any);
done:
    nbhd_release(g, k);
    return rc;
}

/* LT cascade (Sec. 2.2, LT model) in its live-edge form: a popped mu keeps at most one
 * in-neighbour, nu with probability p(nu, mu). With the layers of A(mu) and t_i = floor(p_i 2^32)
 * (2^32 for p = 1): masses m_i = n_i t_i, cumulated C_i = m_1 + ... + m_i, total M = C_l (exact
 * 128-bit integers). One word x of the (RR, mu, layer 0) stream: if M <= 2^32, y = x and no
 * in-neighbour is kept when y >= M; otherwise (sum of p above 1, which standard LT forbids)
 * y = floor(x M / 2^32) always lands, so the probabilities are normalised by M. The kept vertex
 * is position a = floor((y - C_{i-1}) / t_i) of the layer L_i with C_{i-1} <= y < C_i (members
 * in ascending id order): each member of L_i owns t_i consecutive values of y. */
static int rr_pop_lt(or_graph* g, uint64_t seed, uint32_t j, uint32_t c1base, int32_t mu, ivec* R,
                     or_stats* st) {
    uint64_t reads = 0;
    int64_t k = nbhd_build(g, mu, &reads);
    int32_t l = 0;
    for (int64_t i = 0; i < k; ++i)
        if (i == 0 || g->cnt[g->nb[i]] != g->cnt[g->nb[i - 1]]) l++;
    st->pops++;
    st->layers_seen += (uint64_t)l;
    int rc = OR_OK;
    int kept = 0;
    unsigned __int128 M = 0;
    for (int64_t px = g->prof_off[mu]; px < g->prof_off[mu + 1]; ++px)
        M += (unsigned __int128)g->lay_n[px] * (unsigned __int128)g->lay_thr[px];
    if (M == 0) goto done;
    {
        word_stream ws;
        ws_init(&ws, seed, j, c1base, (uint32_t)mu, 0u);
        st->draws++;
        const uint32_t x = ws_next(&ws);
        unsigned __int128 y = x;
        if (M > ((unsigned __int128)1 << 32)) y = ((unsigned __int128)x * M) >> 32;
        else if (y >= M) goto done;
        unsigned __int128 C = 0;
        int64_t start = 0;
        for (int32_t i = 1; i <= l; ++i) {
            const int64_t px = g->prof_off[mu] + i - 1;
            const uint32_t n_i = g->lay_n[px];
            const uint64_t t_i = g->lay_thr[px];
            const unsigned __int128 m_i = (unsigned __int128)n_i * t_i;
            if (y < C + m_i) {
                const uint64_t a = (uint64_t)((y - C) / t_i);
                const int32_t nu = g->nb[start + (int64_t)a];
                st->selected += 1;
                kept = 1;
                st->mats++;
                st->mat_he += (uint64_t)(g->v_off[mu + 1] - g->v_off[mu]);
                st->mat_members += reads;
                if (!g->seen[nu]) { g->seen[nu] = 1; rc = ivec_push(R, nu); }
                break;
            }
            C += m_i;
            start += n_i;
        }
    }
done:
    st->bytes_rr += pop_bytes(g, mu, kept);
    nbhd_release(g, k);
    return rc;
}

static int rr_generate(or_graph* g, uint64_t seed, uint32_t tag, int root_mode, uint32_t stratum,
                       uint32_t j, int strategy, ivec* R, or_stats* st) {
    R->len = 0;
    int32_t root = or_root(g, seed, tag, root_mode, stratum, j);
    if (root < 0) return OR_EINVAL;
    uint32_t c1base = c1_field(tag, stratum_field(root_mode, stratum));
    g->seen[root] = 1;
    int rc = ivec_push(R, root);
    uint32_t* selbuf = NULL;
    uint32_t selcap = 0;
    for (int64_t head = 0; rc == OR_OK && head < R->len; ++head)
        rc = strategy == OR_STRAT_LT ? rr_pop_lt(g, seed, j, c1base, R->v[head], R, st)
                                     : rr_pop(g, seed, j, c1base, strategy, R->v[head], R, st, &selbuf, &selcap);
    free(selbuf);
    for (int64_t i = 0; i < R->len; ++i) g->seen[R->v[i]] = 0;
    if (rc != OR_OK) return rc;
    qsort(R->v, (size_t)R->len, sizeof(int32_t), cmp_i32);
    st->rr_sets++;
    st->members_out += (uint64_t)R->len;
    st->bytes_rr += 4u * (uint64_t)R->len + 8u;
    return OR_OK;
}

int64_t or_rr_set(const or_graph* g, uint64_t seed, uint32_t tag, int root_mode, uint32_t stratum,
                  uint32_t j, int strategy, int32_t* out, int64_t cap, or_stats* st) {
    or_stats local;
    memset(&local, 0, sizeof(local));
    ivec R = {0, 0, 0};
    int rc = rr_generate((or_graph*)g, seed, tag, root_mode, stratum, j, strategy, &R,
                         st ? st : &local);
    if (rc != OR_OK) { free(R.v); return rc; }
    for (int64_t i = 0; i < R.len && i < cap; ++i) out[i] = R.v[i];
    int64_t len = R.len;
    free(R.v);
    return len;
}

/* ============================== forward Monte-Carlo influence ===============================
 * The discrete-time cascade of Sec. 2.2 under the IC model: at time 0 the seeds are active;
 * a vertex u activated at time i gets one chance, at time i + 1, to activate each neighbour v
 * (each nu sharing a hyperedge with u), with probability p(u, v); the cascade stops when no
 * vertex is newly activated. p(u, v) is the probability the layer setting gives u in A(v) --
 * the layer of A(v) keyed by w(u, v) (Sec. 3.1.1) -- i.e. the probability of the same live edge
 * u -> v that the reverse sampler draws for a pop of v, so that the expected number of activated
 * vertices equals sigma(S) of Eq. 1. Coins: one word per directed pair and simulation,
 * Philox4x32-10 with key (seed_lo, seed_hi) and counter (r, u, v, 0xFFFFFFFE); the edge is live
 * iff p = 1, or p > 0 and word < floor(p 2^32). counts[r] = vertices activated in simulation r. */
static uint64_t pair_threshold(const or_graph* g, int32_t v, uint32_t w) {
    for (int64_t x = g->prof_off[v]; x < g->prof_off[v + 1]; ++x)
        if (g->lay_w[x] == w) return g->lay_thr[x];
    return 0; /* unreachable: every w(u, v) > 0 keys a layer of A(v) */
}

int or_forward_spread(const or_graph* g_, const int32_t* seeds, int32_t k, uint64_t sims,
                      uint64_t seed, uint32_t* counts) {
    or_graph* g = (or_graph*)g_;
    if (k < 0 || (k > 0 && !seeds) || (sims > 0 && !counts) || sims > 0x100000000ull)
        return OR_EINVAL;
    for (int32_t i = 0; i < k; ++i)
        if (seeds[i] < 0 || seeds[i] >= g->n) return OR_EINVAL;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    ivec A = {0, 0, 0};
    int rc = OR_OK;
    for (uint64_t r = 0; r < sims && rc == OR_OK; ++r) {
        A.len = 0;
        for (int32_t i = 0; i < k && rc == OR_OK; ++i)
            if (!g->seen[seeds[i]]) { g->seen[seeds[i]] = 1; rc = ivec_push(&A, seeds[i]); }
        for (int64_t head = 0; rc == OR_OK && head < A.len; ++head) {
            const int32_t u = A.v[head];
            const int64_t kn = nbhd_count(g, u);
            for (int64_t x = 0; x < kn && rc == OR_OK; ++x) {
                const int32_t v = g->nb[x];
                const uint64_t thr = pair_threshold(g, v, (uint32_t)g->cnt[v]);
                int live;
                if (thr >= OR_P_ONE) {
                    live = 1;
                } else if (thr == 0) {
                    live = 0;
                } else {
                    const uint32_t ctr[4] = {(uint32_t)r, (uint32_t)u, (uint32_t)v, 0xFFFFFFFEu};
                    uint32_t out[4];
                    or_philox4x32_10(ctr, key, out);
                    live = (uint64_t)out[0] < thr;
                }
                if (live && !g->seen[v]) { g->seen[v] = 1; rc = ivec_push(&A, v); }
            }
            nbhd_release(g, kn);
        }
        counts[r] = (uint32_t)A.len;
        for (int64_t i = 0; i < A.len; ++i) g->seen[A.v[i]] = 0;
    }
    free(A.v);
    return rc;
}

/* ======================================== RR pools ========================================== */
struct or_pool {
    const or_graph* g;
    uint64_t seed;
    uint32_t tag;
    int root_mode, strategy;
    uint64_t n_s[OR_NSTRATA];
    int32_t** sets[OR_NSTRATA]; /* sets[s][j] -> members, sizes in len[s][j] */
    int64_t* len[OR_NSTRATA];
    uint64_t cap_s[OR_NSTRATA];
    or_stats stats;
};

int or_pool_create(const or_graph* g, uint64_t seed, uint32_t tag, int root_mode, int strategy,
                   or_pool** out) {
    if (!g || !out || tag > 0xFF || (root_mode != 0 && root_mode != 1)) return OR_EINVAL;
    if (strategy < OR_STRAT_PAPER || strategy > OR_STRAT_LT) return OR_EINVAL;
    or_pool* p = (or_pool*)calloc(1, sizeof(or_pool));
    if (!p) return OR_ENOMEM;
    p->g = g; p->seed = seed; p->tag = tag; p->root_mode = root_mode; p->strategy = strategy;
    *out = p;
    return OR_OK;
}

void or_pool_free(or_pool* p) {
    if (!p) return;
    for (int s = 0; s < OR_NSTRATA; ++s) {
        for (uint64_t j = 0; j < p->n_s[s]; ++j) free(p->sets[s][j]);
        free(p->sets[s]);
        free(p->len[s]);
    }
    free(p);
}

/* Extends the pool to n_s sets per stratum; sets (s, j) already present are kept as they are. */
int or_pool_grow(or_pool* p, const uint64_t n_s[OR_NSTRATA]) {
    ivec R = {0, 0, 0};
    for (int s = 0; s < OR_NSTRATA; ++s) {
        if (n_s[s] <= p->n_s[s]) continue;
        if (n_s[s] > 0xFFFFFFFFull) { free(R.v); return OR_EOVERFLOW; }
        int32_t sz;
        stratum_list(p->g, p->root_mode, (uint32_t)s, &sz);
        if (sz <= 0) { free(R.v); return OR_EINVAL; }
        if (n_s[s] > p->cap_s[s]) {
            int32_t** ns = (int32_t**)realloc(p->sets[s], sizeof(int32_t*) * n_s[s]);
            if (!ns) { free(R.v); return OR_ENOMEM; }
            p->sets[s] = ns;
            int64_t* nl = (int64_t*)realloc(p->len[s], sizeof(int64_t) * n_s[s]);
            if (!nl) { free(R.v); return OR_ENOMEM; }
            p->len[s] = nl;
            p->cap_s[s] = n_s[s];
        }
        for (uint64_t j = p->n_s[s]; j < n_s[s]; ++j) {
            int rc = rr_generate((or_graph*)p->g, p->seed, p->tag, p->root_mode, (uint32_t)s,
                                 (uint32_t)j, p->strategy, &R, &p->stats);
            if (rc != OR_OK) { p->n_s[s] = j; free(R.v); return rc; }
            p->sets[s][j] = (int32_t*)malloc(sizeof(int32_t) * (size_t)(R.len > 0 ? R.len : 1));
            if (!p->sets[s][j]) { p->n_s[s] = j; free(R.v); return OR_ENOMEM; }
            memcpy(p->sets[s][j], R.v, sizeof(int32_t) * (size_t)R.len);
            p->len[s][j] = R.len;
            p->n_s[s] = j + 1;
        }
    }
    free(R.v);
    return OR_OK;
}

/* The same growth as or_pool_grow, driven by `nworkers` threads over disjoint (s, j): thread t
 * takes the new sets whose rank in the stratum-major order of the growth is t modulo nworkers,
 * each with its own worker view of the pool's graph (or_graph_worker). Every set is the single-
 * threaded rr_generate of (seed, tag, s, j), so the pool is identical to or_pool_grow's. */
typedef struct {
    or_pool* p;
    or_graph* g;
    const uint64_t* first;  /* per stratum: first new j */
    const uint64_t* last;   /* per stratum: end of the new j */
    int t, nworkers;
    int rc;
    or_stats stats;
} grow_job;

static void* grow_worker(void* arg) {
    grow_job* J = (grow_job*)arg;
    ivec R = {0, 0, 0};
    uint64_t rank = 0;
    for (int s = 0; s < OR_NSTRATA && J->rc == OR_OK; ++s)
        for (uint64_t j = J->first[s]; j < J->last[s] && J->rc == OR_OK; ++j, ++rank) {
            if ((int)(rank % (uint64_t)J->nworkers) != J->t) continue;
            or_pool* p = J->p;
            int rc = rr_generate(J->g, p->seed, p->tag, p->root_mode, (uint32_t)s, (uint32_t)j, p->strategy,
                                 &R, &J->stats);
            if (rc != OR_OK) { J->rc = rc; break; }
            int32_t* set = (int32_t*)malloc(sizeof(int32_t) * (size_t)(R.len > 0 ? R.len : 1));
            if (!set) { J->rc = OR_ENOMEM; break; }
            memcpy(set, R.v, sizeof(int32_t) * (size_t)R.len);
            p->sets[s][j] = set;
            p->len[s][j] = R.len;
        }
    free(R.v);
    return NULL;
}

static void add_stats(or_stats* a, const or_stats* b) {
    a->rr_sets += b->rr_sets; a->pops += b->pops; a->layers_seen += b->layers_seen;
    a->draws += b->draws; a->mats += b->mats; a->mat_he += b->mat_he;
    a->mat_members += b->mat_members; a->selected += b->selected;
    a->members_out += b->members_out; a->bytes_rr += b->bytes_rr;
}

int or_pool_grow_mt(or_pool* p, const uint64_t n_s[OR_NSTRATA], or_graph* const* workers, int nworkers) {
    if (nworkers <= 1 || !workers) return or_pool_grow(p, n_s);
    uint64_t first[OR_NSTRATA], last[OR_NSTRATA];
    for (int s = 0; s < OR_NSTRATA; ++s) {
        first[s] = p->n_s[s];
        last[s] = n_s[s] > p->n_s[s] ? n_s[s] : p->n_s[s];
        if (last[s] == first[s]) continue;
        if (last[s] > 0xFFFFFFFFull) return OR_EOVERFLOW;
        int32_t sz;
        stratum_list(p->g, p->root_mode, (uint32_t)s, &sz);
        if (sz <= 0) return OR_EINVAL;
        if (last[s] > p->cap_s[s]) {
            int32_t** ns = (int32_t**)realloc(p->sets[s], sizeof(int32_t*) * last[s]);
            if (!ns) return OR_ENOMEM;
            p->sets[s] = ns;
            int64_t* nl = (int64_t*)realloc(p->len[s], sizeof(int64_t) * last[s]);
            if (!nl) return OR_ENOMEM;
            p->len[s] = nl;
            p->cap_s[s] = last[s];
        }
        for (uint64_t j = first[s]; j < last[s]; ++j) p->sets[s][j] = NULL;
    }
    grow_job* jobs = (grow_job*)calloc((size_t)nworkers, sizeof(grow_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nworkers, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return OR_ENOMEM; }
    int started = 0, rc = OR_OK;
    for (int t = 0; t < nworkers; ++t) {
        jobs[t] = (grow_job){p, workers[t], first, last, t, nworkers, OR_OK, {0}};
        if (pthread_create(&th[t], NULL, grow_worker, &jobs[t]) != 0) { rc = OR_ENOMEM; break; }
        started++;
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < started; ++t) {
        if (jobs[t].rc != OR_OK && rc == OR_OK) rc = jobs[t].rc;
        add_stats(&p->stats, &jobs[t].stats);
    }
    if (started < nworkers && rc == OR_OK) rc = OR_ENOMEM;
    if (rc != OR_OK) {  /* drop the partial growth */
        for (int s = 0; s < OR_NSTRATA; ++s)
            for (uint64_t j = first[s]; j < last[s]; ++j) { free(p->sets[s][j]); p->sets[s][j] = NULL; }
    } else {
        for (int s = 0; s < OR_NSTRATA; ++s) p->n_s[s] = last[s];
    }
    free(jobs);
    free(th);
    return rc;
}

int64_t or_pool_count(const or_pool* p) {
    int64_t c = 0;
    for (int s = 0; s < OR_NSTRATA; ++s) c += (int64_t)p->n_s[s];
    return c;
}

int64_t or_pool_total(const or_pool* p) {
    int64_t t = 0;
    for (int s = 0; s < OR_NSTRATA; ++s)
        for (uint64_t j = 0; j < p->n_s[s]; ++j) t += p->len[s][j];
    return t;
}

void or_pool_counts(const or_pool* p, uint64_t n_s[OR_NSTRATA]) {
    memcpy(n_s, p->n_s, sizeof(uint64_t) * OR_NSTRATA);
}

int or_pool_copy(const or_pool* p, int64_t* off, int32_t* mem, uint8_t* stratum, uint32_t* j) {
    int64_t r = 0, w = 0;
    off[0] = 0;
    for (int s = 0; s < OR_NSTRATA; ++s)
        for (uint64_t jj = 0; jj < p->n_s[s]; ++jj) {
            memcpy(mem + w, p->sets[s][jj], sizeof(int32_t) * (size_t)p->len[s][jj]);
            w += p->len[s][jj];
            if (stratum) stratum[r] = (uint8_t)s;
            if (j) j[r] = (uint32_t)jj;
            off[++r] = w;
        }
    return OR_OK;
}

void or_pool_stats(const or_pool* p, or_stats* st) { *st = p->stats; }

/* Estimator weight of an RR set of stratum s, in 2^-32 units: floor(|V_s| 2^32 / n_s); plain
 * roots weigh 1 (every set stands for |V|/theta vertices). */
static uint64_t stratum_weight(const or_pool* p, int s) {
    if (p->root_mode == OR_ROOTS_PLAIN) return 1;
    if (p->n_s[s] == 0) return 0;
    return ((uint64_t)(uint32_t)p->g->vs_size[s] << 32) / p->n_s[s];
}

/* ================================ greedy max coverage (Algorithm 1) =========================
 * k rounds: pick the vertex with the largest marginal coverage (Eq. 2) -- each uncovered RR set
 * containing it counts with its stratum weight -- ties to the lowest id, among vertices not yet
 * picked; add it to S and retire the RR sets it covers.
 */
static int cmp_u64_desc(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x < y) - (x > y);
}

/* Eq. upper_2 with p_max = 1: min over the greedy prefixes S_i (0 <= i <= k) of the coverage of
 * S_i plus the sum of the k largest marginal coverages given S_i (maxC(S_i, k)), all in the
 * greedy's integer weights; the k largest are taken among the vertices not in S_i. */
static unsigned __int128 topk_sum(const uint64_t* score, const uint8_t* picked, int32_t n, int32_t k,
                                  uint64_t* tmp) {
    int32_t c = 0;
    for (int32_t v = 0; v < n; ++v)
        if (!picked[v]) tmp[c++] = score[v];
    qsort(tmp, (size_t)c, sizeof(uint64_t), cmp_u64_desc);
    unsigned __int128 sum = 0;
    for (int32_t i = 0; i < c && i < k; ++i) sum += tmp[i];
    return sum;
}

int or_greedy(const or_pool* p, int32_t k, int32_t* seeds, uint64_t lambda_s[OR_NSTRATA],
              uint64_t* gains) {
    return or_greedy_upper(p, k, seeds, lambda_s, gains, NULL);
}

int or_greedy_upper(const or_pool* p, int32_t k, int32_t* seeds, uint64_t lambda_s[OR_NSTRATA],
                    uint64_t* gains, uint64_t prefix_upper[2]) {
    const int32_t n = p->g->n;
    if (k < 0 || k > n) return OR_EINVAL;
    int64_t N = or_pool_count(p);
    /* flatten */
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N + 1));
    int32_t* mem = (int32_t*)malloc(sizeof(int32_t) * (size_t)(or_pool_total(p) + 1));
    uint8_t* sof = (uint8_t*)malloc((size_t)(N + 1));
    uint64_t* score = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));
    int64_t* ioff = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    uint8_t* covered = (uint8_t*)calloc((size_t)(N + 1), 1);
    uint8_t* picked = (uint8_t*)calloc((size_t)n, 1);
    if (!off || !mem || !sof || !score || !ioff || !covered || !picked) {
        free(off); free(mem); free(sof); free(score); free(ioff); free(covered); free(picked);
        return OR_ENOMEM;
    }
    or_pool_copy(p, off, mem, sof, NULL);
    uint64_t W[OR_NSTRATA];
    for (int s = 0; s < OR_NSTRATA; ++s) W[s] = stratum_weight(p, s);
    /* inverted index vertex -> RR sets */
    for (int64_t x = 0; x < off[N]; ++x) ioff[mem[x] + 1]++;
    for (int32_t v = 0; v < n; ++v) ioff[v + 1] += ioff[v];
    int64_t* inv = (int64_t*)malloc(sizeof(int64_t) * (size_t)(off[N] + 1));
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)n + 1);
    for (int32_t v = 0; v < n; ++v) cur[v] = ioff[v];
    for (int64_t r = 0; r < N; ++r)
        for (int64_t x = off[r]; x < off[r + 1]; ++x) {
            inv[cur[mem[x]]++] = r;
            score[mem[x]] += W[sof[r]];
        }
    memset(lambda_s, 0, sizeof(uint64_t) * OR_NSTRATA);
    uint64_t* tmp = prefix_upper ? (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1)) : NULL;
    unsigned __int128 cover = 0, best_u = ~(unsigned __int128)0;
    for (int32_t round = 0; round <= k; ++round) {
        if (prefix_upper) {
            const unsigned __int128 u = cover + topk_sum(score, picked, n, k, tmp);
            if (u < best_u) best_u = u;
        }
        if (round == k) break;
        int32_t best = -1;
        for (int32_t v = 0; v < n; ++v) {
            if (picked[v]) continue;
            if (best < 0 || score[v] > score[best]) best = v;
        }
        picked[best] = 1;
        seeds[round] = best;
        uint64_t gain = 0;
        for (int64_t t = ioff[best]; t < ioff[best + 1]; ++t) {
            int64_t r = inv[t];
            if (covered[r]) continue;
            covered[r] = 1;
            lambda_s[sof[r]]++;
            gain += W[sof[r]];
            for (int64_t x = off[r]; x < off[r + 1]; ++x) score[mem[x]] -= W[sof[r]];
        }
        if (gains) gains[round] = gain;
        cover += gain;
    }
    if (prefix_upper) {
        prefix_upper[0] = (uint64_t)best_u;
        prefix_upper[1] = (uint64_t)(best_u >> 64);
    }
    free(tmp);
    free(off); free(mem); free(sof); free(score); free(ioff); free(covered); free(picked);
    free(inv); free(cur);
    return OR_OK;
}

/* Coverage Lambda_R(S) per stratum: RR sets with at least one member in S (Sec. 2.2). */
int or_coverage(const or_pool* p, const int32_t* seeds, int32_t k, uint64_t lambda_s[OR_NSTRATA]) {
    const int32_t n = p->g->n;
    uint8_t* in = (uint8_t*)calloc((size_t)n, 1);
    if (!in) return OR_ENOMEM;
    for (int32_t i = 0; i < k; ++i) {
        if (seeds[i] < 0 || seeds[i] >= n) { free(in); return OR_EINVAL; }
        in[seeds[i]] = 1;
    }
    memset(lambda_s, 0, sizeof(uint64_t) * OR_NSTRATA);
    for (int s = 0; s < OR_NSTRATA; ++s)
        for (uint64_t j = 0; j < p->n_s[s]; ++j)
            for (int64_t x = 0; x < p->len[s][j]; ++x)
                if (in[p->sets[s][j][x]]) { lambda_s[s]++; break; }
    free(in);
    return OR_OK;
}

/* Eq. 1 with the coverage fraction estimated per stratum: sigma = sum_s |V_s|/n_s Lambda_s. */
double or_estimate(const or_pool* p, const uint64_t lambda_s[OR_NSTRATA]) {
    double sigma = 0.0;
    for (int s = 0; s < OR_NSTRATA; ++s) {
        if (p->n_s[s] == 0) continue;
        double vs = p->root_mode == OR_ROOTS_PLAIN ? (double)p->g->n : (double)p->g->vs_size[s];
        sigma = sigma + (vs / (double)p->n_s[s]) * (double)lambda_s[s];
    }
    return sigma;
}

/* ====================================== theta (Sec. 4.3) ====================================
 * delta = n^-ell; ln C(n,k) as a sum of logarithms of ratios; theta_max per Eq. (equation-max):
 *   2 n (sqrt(ln(2/delta)) + sqrt(ln C(n,k) + ln(6/delta))) / (eps^2 k);
 * theta_0 = ceil(theta_max eps^2 k / n); at most i_max = ceil(log2(theta_max/theta_0)) doublings.
 */
int or_plan_theta(int64_t n, int32_t k, double eps, double ell, or_plan* out) {
    if (n < 2 || k < 1 || k > n || !(eps > 0.0 && eps < 1.0) || !(ell > 0.0)) return OR_EINVAL;
    double dn = (double)n, dk = (double)k;
    double delta = pow(dn, -ell);
    /* ln C(n,k) = sum_{i=1..k'} ln((n - k' + i) / i), k' = min(k, n - k): no cancellation */
    int64_t kk = k < n - k ? k : n - k;
    double lnc = 0.0;
    for (int64_t i = 1; i <= kk; ++i) lnc = lnc + log((double)(n - kk + i) / (double)i);
    double tmax = 2.0 * dn * (sqrt(log(2.0 / delta)) + sqrt(lnc + log(6.0 / delta))) /
                  (eps * eps * dk);
    double t0 = tmax * eps * eps * dk / dn;
    uint64_t tmc = (uint64_t)ceil(tmax);
    uint64_t t0c = (uint64_t)ceil(t0);
    if (t0c < 1) t0c = 1;
    int32_t imax = 0;
    while (((double)t0c * ldexp(1.0, imax)) < tmax) imax++;
    out->delta = delta; out->ln_binom = lnc; out->theta_max = tmax;
    out->theta_max_ceil = tmc; out->theta0 = t0c; out->i_max = imax;
    return OR_OK;
}

/* Eq. upper_6 with p_max = 1: Lambda_R1(S_k)/(1 - (1 - 1/k)^k), scaled by n/|R1|. */
double or_upper_bound(double lambda1, int32_t k, int64_t n, uint64_t theta) {
    double base = 1.0 - 1.0 / (double)k;
    double pw = 1.0;
    for (int32_t i = 0; i < k; ++i) pw = pw * base;
    return lambda1 / (1.0 - pw) * (double)n / (double)theta;
}

/* Sec. 4.2 lower bound from R2:
 * ((sqrt(Lambda_R2 + 2 ln(1/delta)/9) - sqrt(ln(1/delta)/2))^2 - ln(1/delta)/18) n/|R2|. */
double or_lower_bound(double lambda2, double delta, int64_t n, uint64_t theta) {
    double L = log(1.0 / delta);
    double a = sqrt(lambda2 + 2.0 * L / 9.0) - sqrt(L / 2.0);
    return (a * a - L / 18.0) * (double)n / (double)theta;
}

/* ================================ HyperIM_BRR (Algorithm 4) =================================
 * Round i uses theta_i = theta_0 2^i RR sets in each of R1 (tag 0) and R2 (tag 1). Greedy on R1
 * gives S_k; the upper bound comes from R1, the lower bound from S_k's coverage of R2; stop when
 * alpha = lower/upper >= 1 - 1/e - eps or after i_max doublings.
 */
/* Eq. upper_2 (integer greedy weights, two 64-bit words) in the units of sigma: the weights
 * are floor(|V_s| 2^32 / n_s) with stratified roots (scale 2^-32), 1 with plain roots (scale n/N). */
double or_prefix_upper_sigma(uint64_t lo, uint64_t hi, int root_mode, int64_t n, uint64_t N) {
    const double u = (double)(((unsigned __int128)hi << 64) | lo);
    if (root_mode == 1) return u * 0x1p-32;
    return (u * (double)n) / (double)N;
}

int or_brr(const or_graph* g, uint64_t seed, int32_t k, double eps, double ell, uint64_t cap,
           int root_mode, int strategy, int32_t* seeds, or_brr_result* res, or_stats* st) {
    return or_brr_upper(g, seed, k, eps, ell, cap, root_mode, strategy, 0, seeds, res, st);
}

int or_brr_upper(const or_graph* g, uint64_t seed, int32_t k, double eps, double ell, uint64_t cap,
                 int root_mode, int strategy, int upper_mode, int32_t* seeds, or_brr_result* res,
                 or_stats* st) {
    return or_brr_upper_mt(g, seed, k, eps, ell, cap, root_mode, strategy, upper_mode, seeds, res, st, NULL, 0);
}

int or_brr_upper_mt(const or_graph* g, uint64_t seed, int32_t k, double eps, double ell, uint64_t cap,
                    int root_mode, int strategy, int upper_mode, int32_t* seeds, or_brr_result* res,
                    or_stats* st, or_graph* const* workers, int nworkers) {
    or_plan plan;
    int rc = or_plan_theta(g->n, k, eps, ell, &plan);
    if (rc != OR_OK) return rc;
    or_pool *r1 = NULL, *r2 = NULL;
    if ((rc = or_pool_create(g, seed, 0, root_mode, strategy, &r1))) return rc;
    if ((rc = or_pool_create(g, seed, 1, root_mode, strategy, &r2))) { or_pool_free(r1); return rc; }
    memset(res, 0, sizeof(*res));
    double target = 1.0 - exp(-1.0) - eps;
    for (int32_t i = 0;; ++i) {
        uint64_t theta = plan.theta0 << i;
        if (cap && theta > cap) { rc = OR_EOVERFLOW; break; }
        uint64_t ns[OR_NSTRATA];
        or_allocate(g, root_mode, theta, ns);
        if ((rc = or_pool_grow_mt(r1, ns, workers, nworkers))) break;
        if ((rc = or_pool_grow_mt(r2, ns, workers, nworkers))) break;
        uint64_t N1 = (uint64_t)or_pool_count(r1), N2 = (uint64_t)or_pool_count(r2);
        uint64_t pu[2] = {0, 0};
        if ((rc = or_greedy_upper(r1, k, seeds, res->lambda_r1, NULL, upper_mode ? pu : NULL))) break;
        if ((rc = or_coverage(r2, seeds, k, res->lambda_r2))) break;
        double s1 = or_estimate(r1, res->lambda_r1);
        double s2 = or_estimate(r2, res->lambda_r2);
        double lam1 = s1 * (double)N1 / (double)g->n;
        double lam2 = s2 * (double)N2 / (double)g->n;
        double up = upper_mode ? or_prefix_upper_sigma(pu[0], pu[1], root_mode, g->n, N1)
                               : or_upper_bound(lam1, k, g->n, N1);
        double lo = or_lower_bound(lam2, plan.delta, g->n, N2);
        double alpha = lo / up;
        res->rounds = i + 1;
        res->theta = theta;
        res->pool_r1 = N1; res->pool_r2 = N2;
        res->sigma_r1 = s1; res->sigma_r2 = s2;
        res->upper = up; res->lower = lo; res->alpha = alpha;
        if (i < 64) res->alpha_round[i] = alpha;
        if (alpha >= target || i >= plan.i_max) break;
    }
    if (st) {
        or_stats a, b;
        or_pool_stats(r1, &a);
        or_pool_stats(r2, &b);
        memset(st, 0, sizeof(*st));
        add_stats(st, &a);
        add_stats(st, &b);
    }
    or_pool_free(r1);
    or_pool_free(r2);
    return rc;
}
