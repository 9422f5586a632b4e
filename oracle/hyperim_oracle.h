/*
 * HyperIM CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded restatement of the HyperIM hot path (stratified RR-set
 * generation over a hypergraph, Algorithm 3, and greedy max coverage, Algorithm 1, with the
 * RR-count bound of Eq. (equation-max) and the doubling schedule of Algorithm 4). It exists to
 * check the CUDA library bit for bit. Only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the product path never does.
 *
 * It shares no code with the CUDA library: every routine (Philox, exp, distributions, layers,
 * sampling, greedy, bounds) is written here independently from the paper and from the published
 * definitions it names.
 */
#ifndef HYPERIM_ORACLE_H
#define HYPERIM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2, OR_EOVERFLOW = -3 };
enum { OR_MODEL_UNIFORM_PAIR = 0, OR_MODEL_WC = 1, OR_MODEL_PAPER_LAYER = 2 };
enum { OR_ROOTS_PLAIN = 0, OR_ROOTS_STRATIFIED = 1 };
enum { OR_STRAT_PAPER = 0, OR_STRAT_BINOMIAL_ONLY = 1, OR_STRAT_LT = 2 };
/* OR_STRAT_LT: the LT cascade's live-edge sampler instead of the IC one -- each popped vertex keeps
 * at most one in-neighbour (see rr_pop_lt in hyperim_oracle.c). */

#define OR_NSTRATA 16
#define OR_P_ONE 4294967296ull /* threshold value meaning p = 1 */

typedef struct or_graph or_graph;
typedef struct or_pool or_pool;

typedef struct {
    uint64_t rr_sets;       /* RR sets generated */
    uint64_t pops;          /* vertices popped from the queue (Alg. 3 loop) */
    uint64_t layers_seen;   /* sum of l_mu over pops (profile entries read) */
    uint64_t draws;         /* layer-size draws with 0 < p < 1 (the paper's sampling operations) */
    uint64_t mats;          /* pops where some layer drew h > 0 (A(mu) must be materialised) */
    uint64_t mat_he;        /* sum of d_H(mu) over materialising pops */
    uint64_t mat_members;   /* sum over materialising pops of sum_{he in mu} |he| */
    uint64_t selected;      /* activations drawn (sum of h) */
    uint64_t members_out;   /* sum of |R| */
    /* Algorithmic bytes of RR generation (the cost model behind Thms 2-3: what a pop must read),
     * at 32-byte-sector granularity, over one layout of the method's data: the layer profile as
     * 12-byte entries of one array in vertex order, v_he and the normalised hyperedge members as
     * 4-byte ids at their CSR offsets. Per pop the sectors of mu's profile entries; per
     * materialising pop also those of v_he(mu) and, for every hyperedge he containing mu, its two
     * offsets (8 bytes) and the sectors of its member ids; per RR set its output ids (4 |R|), its
     * root draw and its offset (8). */
    uint64_t bytes_rr;
} or_stats;

/* ---- primitives ---- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_exp_neg(double x);
uint32_t or_binomial_h(uint32_t n, uint64_t thr, uint32_t w0);
/* Poisson h with lambda = n*p split into ceil(lambda/64) parts; consumes *used words. */
uint32_t or_poisson_h(uint32_t n, uint64_t thr, const uint32_t* words, uint32_t nwords,
                      uint32_t* used);
uint32_t or_poisson_parts(uint32_t n, uint64_t thr);

/* ---- incidence store + layer profile ---- */
int or_graph_build(int32_t n, int32_t m, const int32_t* he_off, const int32_t* he_mem, int model,
                   uint64_t uniform_thr, or_graph** out);
void or_graph_free(or_graph* g);
int32_t or_graph_n(const or_graph* g);
int64_t or_graph_nnz(const or_graph* g);
int32_t or_graph_he_size(const or_graph* g, int32_t he);
int32_t or_graph_dh(const or_graph* g, int32_t v);
int32_t or_graph_deg(const or_graph* g, int32_t v);
int32_t or_graph_nlayers(const or_graph* g, int32_t v);
int32_t or_graph_stratum(const or_graph* g, int32_t v);
int32_t or_graph_stratum_size(const or_graph* g, int32_t s);
double or_graph_theta_lstar(const or_graph* g);
/* layer i (1-based) of A(v): weight w_i, size n_i and threshold floor(p*2^32) (OR_P_ONE = 1). */
int or_graph_layer(const or_graph* g, int32_t v, int32_t i, uint32_t* w, uint32_t* n_i,
                   uint64_t* thr);
/* members of layer i of A(v), ascending ids; returns count or <0 on error. */
int64_t or_graph_layer_members(const or_graph* g, int32_t v, int32_t i, int32_t* out, int64_t cap);

/* A worker view of g for another thread: the same read-only graph, its own scratch (an oracle
 * graph is not safe for concurrent calls). Free it with or_graph_free before g. */
int or_graph_worker(const or_graph* g, or_graph** out);

/* ---- roots, allocation, RR sets ---- */
int or_allocate(const or_graph* g, int root_mode, uint64_t theta, uint64_t n_s[OR_NSTRATA]);
int32_t or_root(const or_graph* g, uint64_t seed, uint32_t tag, int root_mode, uint32_t stratum,
                uint32_t j);
int64_t or_rr_set(const or_graph* g, uint64_t seed, uint32_t tag, int root_mode, uint32_t stratum,
                  uint32_t j, int strategy, int32_t* out, int64_t cap, or_stats* st);

/* ---- pools ---- */
int or_pool_create(const or_graph* g, uint64_t seed, uint32_t tag, int root_mode, int strategy,
                   or_pool** out);
void or_pool_free(or_pool* p);
int or_pool_grow(or_pool* p, const uint64_t n_s[OR_NSTRATA]);
/* The same growth driven by nworkers threads over disjoint (s, j), each with its own worker view
 * (workers[t], views of the pool's graph); the resulting pool is identical to or_pool_grow's. */
int or_pool_grow_mt(or_pool* p, const uint64_t n_s[OR_NSTRATA], or_graph* const* workers, int nworkers);
int64_t or_pool_count(const or_pool* p);
int64_t or_pool_total(const or_pool* p);
void or_pool_counts(const or_pool* p, uint64_t n_s[OR_NSTRATA]);
/* copies the pool in stratum-major, j-ascending order */
int or_pool_copy(const or_pool* p, int64_t* off, int32_t* mem, uint8_t* stratum, uint32_t* j);
void or_pool_stats(const or_pool* p, or_stats* st);

/* ---- greedy, estimate ---- */
int or_greedy(const or_pool* p, int32_t k, int32_t* seeds, uint64_t lambda_s[OR_NSTRATA],
              uint64_t* gains);
int or_coverage(const or_pool* p, const int32_t* seeds, int32_t k, uint64_t lambda_s[OR_NSTRATA]);
double or_estimate(const or_pool* p, const uint64_t lambda_s[OR_NSTRATA]);

/* Forward Monte-Carlo influence of a seed set (Sec. 2.2 cascade, IC model; keyed coins, see the
 * definition in hyperim_oracle.c): counts[r] = vertices activated in simulation r, r < sims
 * (sims <= 2^32). OR_EINVAL on a seed outside [0, n). */
int or_forward_spread(const or_graph* g, const int32_t* seeds, int32_t k, uint64_t sims,
                      uint64_t seed, uint32_t* counts);

/* ---- theta plan + BRR ---- */
typedef struct {
    double delta, ln_binom, theta_max;
    uint64_t theta_max_ceil, theta0;
    int32_t i_max;
} or_plan;
int or_plan_theta(int64_t n, int32_t k, double eps, double ell, or_plan* out);
double or_upper_bound(double lambda1, int32_t k, int64_t n, uint64_t theta);
double or_lower_bound(double lambda2, double delta, int64_t n, uint64_t theta);

typedef struct {
    int32_t rounds;
    uint64_t theta;          /* target theta of the last round */
    uint64_t pool_r1, pool_r2;
    double sigma_r1, sigma_r2;
    double upper, lower, alpha;
    double alpha_round[64];
    uint64_t lambda_r1[OR_NSTRATA], lambda_r2[OR_NSTRATA];
} or_brr_result;
int or_brr(const or_graph* g, uint64_t seed, int32_t k, double eps, double ell, uint64_t cap,
           int root_mode, int strategy, int32_t* seeds, or_brr_result* res, or_stats* st);
/* Greedy that also returns Eq. upper_2 (p_max = 1): min over i in [0, k] of the weighted
 * coverage of the first i seeds plus the k largest weighted marginal coverages of the vertices
 * not among them, as an unsigned 128-bit integer {low, high} in the greedy's weights. */
int or_greedy_upper(const or_pool* p, int32_t k, int32_t* seeds, uint64_t lambda_s[OR_NSTRATA],
                    uint64_t* gains, uint64_t prefix_upper[2]);
/* or_brr_upper with the pools grown by or_pool_grow_mt over `workers` (NULL / 0: one thread) */
int or_brr_upper_mt(const or_graph* g, uint64_t seed, int32_t k, double eps, double ell, uint64_t cap,
                    int root_mode, int strategy, int upper_mode, int32_t* seeds, or_brr_result* res,
                    or_stats* st, or_graph* const* workers, int nworkers);
/* that bound in the units of sigma (stratified: x 2^-32; plain: x n / N) */
double or_prefix_upper_sigma(uint64_t lo, uint64_t hi, int root_mode, int64_t n, uint64_t N);
/* BRR with the upper bound of Eq. upper_6 (upper_mode 0, the closed form Alg. 4 uses) or of
 * Eq. upper_2 (upper_mode 1, its definition: the prefix minimum). */
int or_brr_upper(const or_graph* g, uint64_t seed, int32_t k, double eps, double ell, uint64_t cap,
                 int root_mode, int strategy, int upper_mode, int32_t* seeds, or_brr_result* res,
                 or_stats* st);

#ifdef __cplusplus
}
#endif
#endif
