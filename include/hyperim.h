/*
 * hyperim.h -- C ABI of the GB300 (sm_103a) HyperIM library.
 *
 * HyperIM ("Influence Maximization in Hypergraphs by Stratified Sampling for Efficient Generation
 * of Reverse Reachable Sets", arXiv 2406.01911) picks k seed vertices of a hypergraph G = (V, HE)
 * with the largest expected influence (Def. 1). Its hot path, implemented here in CUDA kernels:
 *
 *   load      -- incidence store (he -> members, v -> he; never the clique expansion G_w of
 *                Sec. 2.1) and the per-vertex layer profile of A(mu) (Sec. 3.1.1);
 *   plan      -- the RR-set budget theta_max, theta_0 and the doubling count (Eq. equation-max,
 *                Sec. 4.3);
 *   sample    -- stratified random RR sets (Algorithm 3 with the Binomial/Poisson strategies of
 *                Sec. 3.1.3), roots drawn per stratum, output compacted to CSR;
 *   select    -- greedy max coverage (Algorithm 1) over a pool, fixed theta or the adaptive
 *                HyperIM_BRR schedule (Algorithm 4) with the bounds of Sec. 4.2;
 *   spread    -- the RR estimate of a seed set's influence (Eq. 1).
 *
 * Conventions (all entry points):
 *   - Every call returns a hyperim_status; no C++ exception crosses this boundary. On a non-OK
 *     status hyperim_last_error() returns a thread-local message.
 *   - Input pointers are borrowed for the duration of the call only. Handles own all device
 *     memory they allocate (stream-ordered cudaMallocAsync on the graph's stream).
 *   - All device work is ordered on the graph's CUDA stream (hyperim_load_args.cuda_stream, or
 *     the legacy default stream when NULL). Calls that return host results synchronise it.
 *   - Randomness: every draw is a word of Philox4x32-10 (Salmon et al., SC'11) keyed by the
 *     graph's 64-bit seed and a counter built from (pool tag, stratum, RR index, popped vertex,
 *     layer, block). Results therefore do not depend on launch configuration or scheduling.
 *   - Vertex ids are int32 in [0, n); n < 2^31 - 1. Hyperedges are vertex sets: repeated ids in
 *     one hyperedge are collapsed on load; a hyperedge with fewer than two members links nobody.
 */
#ifndef HYPERIM_H
#define HYPERIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HYPERIM_OK = 0,
    HYPERIM_EINVAL = -1,     /* bad argument: id out of range, k > n, eps not in (0,1), ... */
    HYPERIM_ENOMEM = -2,     /* device allocation failed or the HBM budget would be exceeded */
    HYPERIM_EOVERFLOW = -3,  /* theta cap or a fixed-size arena exceeded; results discarded */
    HYPERIM_ETIMEDOUT = -4,  /* a bounded device-side wait gave up */
    HYPERIM_ECUDA = -5,      /* a CUDA runtime call failed */
    HYPERIM_ESTATE = -6      /* handle used in the wrong state (e.g. pool of another graph) */
} hyperim_status;

/* Activation probability of nu -> mu for nu in layer L_i of A(mu). */
typedef enum {
    HYPERIM_P_UNIFORM_PAIR = 0, /* one p for every co-member pair: p = uniform_threshold / 2^32 */
    HYPERIM_P_WC = 1,           /* weighted cascade: p = floor(2^32 / deg(mu)) / 2^32, 1 if deg=1 */
    HYPERIM_P_PAPER_LAYER = 2   /* Sec. 3.1.1: p = P(L_i)/n(L_i), P(L_i) = 1/(i ln(l_mu + 1)),
                                   clamped to 1 */
} hyperim_prob_model;

typedef enum {
    HYPERIM_ROOTS_PLAIN = 0,      /* roots uniform over V (Alg. 3, first step) */
    HYPERIM_ROOTS_STRATIFIED = 1  /* roots uniform within strata s(mu) = min(l_mu, 15), with
                                     n_s = ceil(theta |V_s| / n) sets per nonempty stratum */
} hyperim_root_mode;

typedef enum {
    HYPERIM_STRAT_PAPER = 0,         /* Binomial if n(L_i) <= 20, else Poisson (Sec. 3.1.3) */
    HYPERIM_STRAT_BINOMIAL_ONLY = 1, /* Binomial for every layer (exact IC semantics, Lemma 3) */
    HYPERIM_STRAT_LT = 2             /* the LT cascade (Sec. 2.2) in live-edge form: a popped mu
                                        keeps at most one in-neighbour; one word w against the
                                        layers' masses n_i floor(p_i 2^32) cumulated as C_i (sum
                                        M): y = w if M <= 2^32 (nothing kept when y >= M), else
                                        floor(w M / 2^32); kept: position floor((y - C_{i-1}) /
                                        t_i) of the layer with C_{i-1} <= y < C_i. Stream (RR, mu,
                                        layer field 0). */
} hyperim_strategy;

typedef struct hyperim_graph* hyperim_graph_t;
typedef struct hyperim_pool* hyperim_pool_t;

#define HYPERIM_NSTRATA 16
#define HYPERIM_P_ONE 4294967296ull /* uniform_threshold value meaning p = 1 */

/* ------------------------------------------------------------------------------------------
 * hyperim_load -- build the incidence store and layer profile of G on the device.
 *   Sec. 2.1 (G, V(he), w(mu,nu), deg(mu)); Sec. 3.1.1 (layers of A(mu), l_mu, n(L_i), P(L_i)).
 *   he_off[m+1], he_mem[he_off[m]]: hyperedge -> member CSR, int32; host pointers, or device
 *   pointers when ptrs_on_device != 0 (read during the call only). Members of a hyperedge may
 *   come in any order and may repeat.
 *   EINVAL: n < 1, n >= 2^31 - 1, m < 0, he_off not monotone from 0, a member outside [0, n),
 *   model out of range, uniform_threshold > 2^32, only one of dev_alloc / dev_free given.
 *   ENOMEM: allocation failed or the device footprint would exceed hbm_budget_bytes (0 = no
 *   budget). On success *out owns the graph.
 *   Device memory: with dev_alloc and dev_free both NULL every device buffer of the graph, its
 *   shares and its pools comes from cudaMallocAsync / cudaFreeAsync on the handle's stream. A
 *   caller that owns the GPU's memory (PyTorch's caching allocator, a server that hands memory
 *   out by budget) passes both: dev_alloc(bytes, stream, alloc_ctx) returns a device pointer
 *   aligned to at least 256 bytes, or NULL (the call then fails with ENOMEM); dev_free(ptr,
 *   stream, alloc_ctx) releases one, ordered after the work queued on `stream` before it (the
 *   way cudaFreeAsync is). `stream` is the cudaStream_t of the handle making the call (a share
 *   passes its own). The hooks may be called from any thread that calls into the library
 *   (query server workers included) and must outlive the graph, its shares and its pools. The
 *   HBM budget still counts every byte requested through them.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t n;                   /* |V| */
    int32_t m;                   /* |HE| */
    const int32_t* he_off;       /* m + 1 offsets */
    const int32_t* he_mem;       /* he_off[m] members */
    int32_t ptrs_on_device;      /* 0: host pointers; 1: device pointers */
    int32_t model;               /* hyperim_prob_model */
    uint64_t uniform_threshold;  /* floor(p 2^32) for HYPERIM_P_UNIFORM_PAIR, <= 2^32 */
    uint64_t seed;               /* Philox key (seed_lo, seed_hi) */
    void* cuda_stream;           /* cudaStream_t, may be NULL */
    size_t hbm_budget_bytes;     /* 0 = unlimited */
    void* (*dev_alloc)(size_t bytes, void* cuda_stream, void* alloc_ctx);  /* NULL: cudaMallocAsync */
    void (*dev_free)(void* ptr, void* cuda_stream, void* alloc_ctx);       /* NULL: cudaFreeAsync */
    void* alloc_ctx;             /* passed to both hooks */
} hyperim_load_args;

hyperim_status hyperim_load(const hyperim_load_args* args, hyperim_graph_t* out);

/* ------------------------------------------------------------------------------------------
 * hyperim_graph_share -- a second handle on a loaded graph, for calls from another host thread
 *   on another stream at the same time (a query server, one worker per handle). It reads g's
 *   incidence store, layer profile and chunk index (never copied) and owns its own stream
 *   (cuda_stream, may be NULL), RR-kernel scratch, device status word and counters. Handles of
 *   one graph share its HBM budget, its seed and its RR schedule at the time of sharing, and
 *   any of them may grow or read the pools created on any other: a pool is grown under an
 *   exclusive lock and read (greedy, coverage, views, copies) under a shared one, so concurrent
 *   calls see whole growth steps. The result of a call does not depend on other calls running
 *   beside it (RR sets are keyed by (stratum, index); BRR rounds read the prefix of a pool that
 *   their theta names). g may itself be a share; every share is freed with hyperim_graph_free.
 *   EINVAL: g or out NULL. ENOMEM: budget or allocation.
 * ------------------------------------------------------------------------------------------ */
hyperim_status hyperim_graph_share(hyperim_graph_t g, void* cuda_stream, hyperim_graph_t* out);

/* hyperim_graph_free -- releases a handle. The loaded graph's device data stays until it, all of
 * its shares and all of its pools are freed (in any order). Synchronises the handle's stream.
 * NULL is ignored. A freed handle must not be used again (its shares and pools may). */
void hyperim_graph_free(hyperim_graph_t g);

/* ------------------------------------------------------------------------------------------
 * hyperim_graph_stats -- scalar statistics of a loaded graph (host struct, filled on return).
 *   theta_lstar is Thm 2's theta(l*) = (1/|V|) sum_v l_v / ln(l_v + 1).
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t n, m;
    int64_t nnz;                           /* members after normalisation */
    int64_t profile_entries;               /* sum_v l_v */
    int32_t max_layers, max_dh;
    int64_t max_deg;
    int64_t stratum_size[HYPERIM_NSTRATA]; /* |V_s| */
    double theta_lstar;
    size_t device_bytes;                   /* device memory held by the graph */
    int32_t index_vertices;                /* vertices with a chunk index (hyperim_graph_chunk_index) */
    int64_t index_entries;                 /* uint32 entries of all chunk-index tables */
} hyperim_graph_stats_t;

hyperim_status hyperim_graph_stats(hyperim_graph_t g, hyperim_graph_stats_t* out);

/* ------------------------------------------------------------------------------------------
 * hyperim_graph_profile -- copy the layer profile to host buffers (Sec. 3.1.1).
 *   Any pointer may be NULL to skip it. deg[n] = |A(v)|, nlayers[n] = l_v, stratum[n],
 *   prof_off[n+1] (int64), and for each profile entry x in [prof_off[v], prof_off[v+1]) the
 *   layer i = x - prof_off[v] + 1 of A(v): layer_w[x] = w_i (descending in i), layer_n[x] = n_i,
 *   layer_thr[x] = floor(p_i 2^32) with 2^32 meaning p = 1. Buffers are caller-owned and sized
 *   from hyperim_graph_stats. Synchronises the stream.
 * ------------------------------------------------------------------------------------------ */
hyperim_status hyperim_graph_profile(hyperim_graph_t g, int32_t* deg, int32_t* nlayers,
                                     int32_t* stratum, int64_t* prof_off, uint32_t* layer_w,
                                     uint32_t* layer_n, uint64_t* layer_thr);

/* ------------------------------------------------------------------------------------------
 * hyperim_graph_chunk_index -- copy one vertex's chunk index to host (a lookup structure of this
 *   library over the layers of Sec. 3.1.1, not a quantity of the paper).
 *   Ids are split into C = 2^bits chunks by their top bits (chunk of u = u >> (B - bits),
 *   B = ceil(log2 n), at least 1), and table[(i - 1) C + k] = number of members of layer L_i of
 *   A(v) whose chunk is < k (i = 1..l_v, k = 0..C-1). Which vertices have one: d_H(v) >= 2,
 *   1 <= l_v <= 1024, and, with T = members of v's hyperedges other than v (repeats counted) and
 *   lambda = sum_i n_i p_i the expected picks per pop (decided on the integers
 *   sum_i n_i floor(p_i 2^32) against 4 2^32): T > 1024 if lambda < 4, else T > 2048; bits is the
 *   fewest (1..min(12, B)) for which no chunk holds more than 512 (lambda < 4) or 1024 of those
 *   members, and no index if none does. *bits = 0 and *entries = 0 when v has no index. table may
 *   be NULL (then only *bits and *entries are set); otherwise it must hold cap >= *entries =
 *   l_v C entries (EINVAL if not). EINVAL: v outside [0, n). Synchronises the stream.
 * ------------------------------------------------------------------------------------------ */
hyperim_status hyperim_graph_chunk_index(hyperim_graph_t g, int32_t v, int32_t* bits,
                                         uint32_t* table, int64_t cap, int64_t* entries);

/* ------------------------------------------------------------------------------------------
 * hyperim_graph_set_schedule -- how RR generation (Alg. 3) is scheduled on the GPU for every
 *   later hyperim_sample_rr / hyperim_select_seeds call on g. The RR sets are identical under
 *   both (their draws are keyed by RR id, vertex and layer); only the time differs.
 *   HYPERIM_SCHED_PERSISTENT (the default): one launch per growth step, a persistent grid whose
 *     blocks take RR sets from a device counter until none is left.
 *   HYPERIM_SCHED_PLAIN: the comparison form, one launch per batch of as many RR sets as blocks
 *     fit on the GPU, one set per block, the next batch launched after the slowest set of the
 *     previous one finishes.
 *   EINVAL: g NULL or an unknown schedule. No device work.
 * ------------------------------------------------------------------------------------------ */
typedef enum { HYPERIM_SCHED_PERSISTENT = 0, HYPERIM_SCHED_PLAIN = 1 } hyperim_schedule;
hyperim_status hyperim_graph_set_schedule(hyperim_graph_t g, int32_t schedule);

/* ------------------------------------------------------------------------------------------
 * hyperim_graph_set_tuning / hyperim_graph_get_tuning -- scheduling parameters of RR generation
 *   on this handle (shares made afterwards inherit them). None changes any RR set, seed or
 *   estimate: the draws are keyed by (RR, vertex, layer), so only the time differs.
 *   warp_set_limit: in the persistent schedule every RR set is first built by one warp alone
 *     (its members in on-chip memory) while it has at most this many members (1..128) and no
 *     pop needs the block path; larger sets are built again by a whole block. 0: every set by a
 *     block (no warp phase), the default (hyperim_graph_autotune measures the alternatives).
 *   early_sets_per_block: BRR (hyperim_select_seeds) grows R1 and R2 in its first launch to at
 *     least this many sets per resident block of the RR kernel per pool (the rounds up to that
 *     theta read their prefixes of it). >= 1; default 4.
 *   arena_entries_per_set: the output arena of a growth step starts at this many entries per
 *     new RR set (0, the default: 1.25 x the pool's mean set size so far, or the handle's last
 *     growth's, or min(sets x n, 2^27) entries with no history). A set that does not fit is
 *     built again by a repair launch and written to the slot the first launch reserved for it,
 *     so a small value costs time, never results. 0..2^20.
 *   EINVAL: g or t NULL, a value out of range. No device work.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t warp_set_limit;
    int32_t early_sets_per_block;
    int32_t arena_entries_per_set;
} hyperim_tuning;
hyperim_status hyperim_graph_set_tuning(hyperim_graph_t g, const hyperim_tuning* t);
hyperim_status hyperim_graph_get_tuning(hyperim_graph_t g, hyperim_tuning* out);

/* ------------------------------------------------------------------------------------------
 * hyperim_graph_autotune -- choose g's tuning for RR generation by measurement (not part of
 *   the paper: an autotuner of this library). The graph's degree profile (the model and its
 *   threshold, n and nnz, the shares of the 16 strata, the largest neighbourhood and degree, in
 *   logarithmic buckets) and (root_mode, strategy) form a key; if the process has tuned a graph
 *   of that key before, its choice is applied at once (from_cache = 1). Otherwise every
 *   candidate -- warp_set_limit in {0 (no warp phase), 16, 32, 64, 128} -- grows a scratch
 *   pool (tag 255) to `sets` RR sets (0: 8 per SM), the same sets each time since they are keyed
 *   by (stratum, index), and the candidate with the least RR-kernel time (CUDA events, best of
 *   two) is applied to g and cached under the key, with the per-set SM cycles (mean, maximum)
 *   the candidate without warp phase measured; a graph that takes a cached choice and has no
 *   launch of its own yet starts with those cycles (used by BRR's growing ahead, see
 *   hyperim_select_seeds). early_sets_per_block is left as it is. The RR sets, seeds and
 *   estimates never depend on the choice. EINVAL: g or out NULL, bad mode or
 *   strategy. Synchronises the stream.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    hyperim_tuning chosen;
    int32_t from_cache;
    int32_t candidates;          /* timed now (0 when from_cache) */
    int32_t warp_set_limit[8];   /* per candidate */
    double seconds[8];           /* RR-kernel seconds of the candidate's growth */
    uint64_t profile_key;
} hyperim_autotune_result;
hyperim_status hyperim_graph_autotune(hyperim_graph_t g, int32_t root_mode, int32_t strategy, uint64_t sets,
                                      hyperim_autotune_result* out);

/* ------------------------------------------------------------------------------------------
 * hyperim_graph_set_wait_limit -- bound of the device-side waits of this handle's kernels (a
 *   warp of the RR or forward kernel waiting for its block's work queue: a claimable vertex, or
 *   the id of a claimed slot still being stored). A wait that runs `iterations` rounds without
 *   progress gives up: the kernel records it, every block leaves its current set and the
 *   launch ends; the call returns HYPERIM_ETIMEDOUT and its results are discarded (the handle
 *   stays usable, pools keep the sets of earlier growth steps). 0 restores the default of 2^24
 *   rounds (about a second of sleeping per wait). Not part of the paper: a failure detector of
 *   this library. Shares made afterwards inherit the value. EINVAL: g NULL. No device work.
 * ------------------------------------------------------------------------------------------ */
hyperim_status hyperim_graph_set_wait_limit(hyperim_graph_t g, uint32_t iterations);

/* ------------------------------------------------------------------------------------------
 * hyperim_plan_theta -- RR budget of Sec. 4.3 (host arithmetic, IEEE double).
 *   delta = n^-ell (Sec. 6: delta = 1/|V| for ell = 1); ln C(n,k) = sum_{i<=k'} ln((n-k'+i)/i)
 *   with k' = min(k, n-k);
 *   theta_max = 2n (sqrt(ln(2/delta)) + sqrt(ln C(n,k) + ln(6/delta))) / (eps^2 k)
 *   (Eq. equation-max, delta inside both logarithms); theta0 = ceil(theta_max eps^2 k / n);
 *   i_max = ceil(log2(theta_max / theta0)).  EINVAL: k < 1, k > n, eps not in (0,1), ell <= 0.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    double delta;
    double ln_binom;
    double theta_max;         /* real value */
    uint64_t theta_max_ceil;
    uint64_t theta0;
    int32_t i_max;
} hyperim_theta_plan;

hyperim_status hyperim_plan_theta(hyperim_graph_t g, int32_t k, double eps, double ell,
                                  hyperim_theta_plan* out);

/* ------------------------------------------------------------------------------------------
 * hyperim_sample_rr -- grow an RR pool to the allocation of theta (Algorithm 3).
 *   If *inout is NULL a pool is created with (pool_tag, root_mode, strategy); otherwise those
 *   arguments must match the pool's (ESTATE if not). Stratum s holds n_s(theta) sets, n_s as in
 *   hyperim_root_mode; RR set (s, j) is a pure function of (seed, tag, s, j), so sets already in
 *   the pool are kept and only j in [old n_s, new n_s) are generated. pool_tag < 256. Device
 *   CSR output; the call synchronises the stream once to size the CSR.
 *   EOVERFLOW: some n_s >= 2^32, or one layer draw needs more than 2^18 Philox words.
 *   ETIMEDOUT: a bounded device wait gave up (hyperim_graph_set_wait_limit); the pool keeps the
 *   sets it held before the call.
 * ------------------------------------------------------------------------------------------ */
hyperim_status hyperim_sample_rr(hyperim_graph_t g, uint32_t pool_tag, uint64_t theta,
                                 int32_t root_mode, int32_t strategy, hyperim_pool_t* inout);
void hyperim_pool_free(hyperim_pool_t p);

/* ------------------------------------------------------------------------------------------
 * hyperim_sample_rr_shard -- like hyperim_sample_rr for one shard of a pool split over `world`
 *   ranks (processes or GPUs): the shard holds the sets (s, j) of the allocation of theta with
 *   j = rank (mod world), so the shards of ranks 0..world-1 together hold exactly the pool
 *   hyperim_sample_rr would build (every set is keyed by (seed, tag, s, j)), with no exchange.
 *   The shard's n_s (pool view) is the whole allocation it covers; its count is its own sets.
 *   A pool made by this call is a shard for good (ESTATE if grown with another rank or world,
 *   or by hyperim_sample_rr). EINVAL: world < 1, rank outside [0, world), others as
 *   hyperim_sample_rr.
 * ------------------------------------------------------------------------------------------ */
hyperim_status hyperim_sample_rr_shard(hyperim_graph_t g, uint32_t pool_tag, uint64_t theta, int32_t root_mode,
                                       int32_t strategy, int32_t rank, int32_t world, hyperim_pool_t* inout);

/* ------------------------------------------------------------------------------------------
 * Greedy max coverage one round at a time (Algorithm 1), for pools split into shards: each
 *   round every rank hands its shard's weighted marginal scores (Eq. 2) to an all-reduce (sum),
 *   and each rank picks the argmax of the sum -- the same vertex everywhere: integer weights,
 *   ties to the lowest id -- and retires the RR sets of its own shard that it covers.
 *   hyperim_greedy_begin: the state of a pool's prefix view (the sets a pool grown to theta
 *     holds; theta = 0: every set of the pool): inverted index and initial scores, weights
 *     floor(|V_s| 2^32 / n_s) from the view's allocation (1 with plain roots). The pool must not
 *     grow while the state lives (it holds the pool's read lock).
 *   hyperim_greedy_scores: copies the shard's n current scores (uint64, device) to dev_out
 *     (caller-owned device memory, n entries), ordered on the graph's stream.
 *   hyperim_greedy_pick: argmax over the vertices not picked yet of dev_total (device, n uint64:
 *     the summed scores; NULL: this shard's own), ties to the lowest id; marks it picked,
 *     retires this shard's uncovered sets that contain it; *picked = the vertex (host).
 *     Synchronises the stream.
 *   hyperim_greedy_end: this shard's coverage per stratum of the picks (Lambda_s) and frees the
 *     state. EINVAL: null arguments.
 * ------------------------------------------------------------------------------------------ */
typedef struct hyperim_greedy* hyperim_greedy_t;
hyperim_status hyperim_greedy_begin(hyperim_graph_t g, hyperim_pool_t pool, uint64_t theta, hyperim_greedy_t* out);
hyperim_status hyperim_greedy_scores(hyperim_greedy_t s, uint64_t* dev_out);
hyperim_status hyperim_greedy_pick(hyperim_greedy_t s, const uint64_t* dev_total, int32_t* picked);
hyperim_status hyperim_greedy_end(hyperim_greedy_t s, uint64_t lambda_s[HYPERIM_NSTRATA]);

/* ------------------------------------------------------------------------------------------
 * hyperim_coverage_view -- Lambda_s of a seed set (host ids) on a pool's prefix view of theta
 *   (0: the whole pool): the RR sets of each stratum with a member in the set (Sec. 2.2); for a
 *   shard, its own sets. Synchronises the stream. EINVAL: a seed outside [0, n).
 * ------------------------------------------------------------------------------------------ */
hyperim_status hyperim_coverage_view(hyperim_graph_t g, hyperim_pool_t pool, uint64_t theta, const int32_t* seeds_host,
                                     int32_t k, uint64_t lambda_s[HYPERIM_NSTRATA]);

/* ------------------------------------------------------------------------------------------
 * hyperim_brr_round -- the host arithmetic of one HyperIM_BRR round (Algorithm 4) from the
 *   coverages summed over every shard: with theta_i = theta0 2^i and n_s = its allocation,
 *   sigma_r = sum_s |V_s|/n_s Lambda_s (Eq. 1) on R1 and R2, the Eq. upper_6 bound (p_max = 1)
 *   from R1, the Sec. 4.2 lower bound from R2, alpha = lower / upper, and stop = 1 when alpha >=
 *   1 - 1/e - eps or round >= i_max -- exactly what hyperim_select_seeds does per round.
 *   EINVAL: bad k, eps, ell, root mode or a round beyond 62.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    uint64_t theta;
    double sigma_r1, sigma_r2, upper, lower, alpha;
    int32_t stop;
} hyperim_brr_round_t;
hyperim_status hyperim_brr_round(hyperim_graph_t g, int32_t k, double eps, double ell, int32_t root_mode, int32_t round,
                                 const uint64_t lambda_r1[HYPERIM_NSTRATA], const uint64_t lambda_r2[HYPERIM_NSTRATA],
                                 hyperim_brr_round_t* out);

/* ------------------------------------------------------------------------------------------
 * hyperim_pool_view -- read-only device view of a pool (valid until the pool grows or is freed).
 *   RR set r has members rr_mem[rr_off[r] .. rr_off[r+1]) (ascending ids), stratum rr_stratum[r]
 *   and index rr_j[r] within its stratum. Sets are stored in generation order: one stratum-major
 *   block per growth step.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int64_t count;                         /* RR sets */
    int64_t total;                         /* sum of sizes */
    const int64_t* rr_off;                 /* device, count + 1 */
    const int32_t* rr_mem;                 /* device, total */
    const uint8_t* rr_stratum;             /* device, count */
    const uint32_t* rr_j;                  /* device, count */
    uint64_t n_s[HYPERIM_NSTRATA];         /* sets per stratum */
    uint32_t pool_tag;
    int32_t root_mode, strategy;
    /* work counters of all generation launches so far: vertices popped, profile entries read,
       layer draws with 0 < p < 1, pops that materialised A(mu), hyperedges and members read by
       those materialisations, activations drawn (sum of h) */
    uint64_t pops, layers_seen, draws, mats, mat_he, mat_members, selected;
    /* member ids the library actually read for those materialisations (one pass: sum of |he|
       over mu's hyperedges, or only the id ranges of the chunks that hold picks when mu has a
       chunk index), and 4-byte words read to locate those ranges (span entries, binary-search
       probes into hyperedges, chunk-index probes) */
    uint64_t gathered, search_words;
    uint64_t rr_launches;     /* RR-generation kernel launches that grew this pool first (a launch
                                 growing R1 and R2 of a BRR round together counts once, on R1) */
    double rr_kernel_seconds; /* this pool's share (by RR sets) of those launches' duration,
                                 CUDA events on the graph's stream */
    /* 32-byte sectors of the method's own data that generation touches, whatever this library
       actually reads: per pop the sectors spanned by mu's profile (l_mu entries of 12 bytes at
       entry offset prof_off[mu] of one array over all vertices); per materialising pop also
       those spanned by v_he(mu) (4-byte ids at v_off[mu]) and by mem(he) (4-byte ids at
       he_off[he]) of every he containing mu, offsets of the normalised incidence store. With
       the pool's other counters it gives the algorithmic bytes of RR generation,
       B = 32 sectors + 8 mat_he + 4 total + 8 count (the two offsets read per hyperedge, the
       output ids, the root draw and the set's offset). */
    uint64_t sectors;
} hyperim_pool_view_t;

hyperim_status hyperim_pool_view(hyperim_pool_t p, hyperim_pool_view_t* out);

/* ------------------------------------------------------------------------------------------
 * hyperim_pool_copy -- copy a pool's CSR to caller-owned HOST buffers (any may be NULL):
 *   rr_off[count + 1], rr_mem[total], rr_stratum[count], rr_j[count], in the layout of
 *   hyperim_pool_view. Synchronises the stream.
 * ------------------------------------------------------------------------------------------ */
hyperim_status hyperim_pool_copy(hyperim_pool_t p, int64_t* rr_off, int32_t* rr_mem,
                                 uint8_t* rr_stratum, uint32_t* rr_j);

/* ------------------------------------------------------------------------------------------
 * hyperim_select_seeds -- greedy max coverage (Algorithm 1) and, in BRR mode, HyperIM_BRR.
 *   FIXED: greedy on r1 as it is (r2 may be NULL; if given, S_k's coverage of r2 is reported).
 *   BRR:   r1 and r2 (distinct pools of this graph, pool tags 0 and 1 by convention, possibly
 *          empty) are grown round by round to theta_i = theta0 2^i (Algorithm 4); greedy on r1
 *          gives S_k; upper bound Lambda_R1(S_k)/(1 - (1 - 1/k)^k) n/|R1| (Eq. upper_6,
 *          p_max = 1); lower bound ((sqrt(Lambda_R2 + 2 ln(1/delta)/9) - sqrt(ln(1/delta)/2))^2 -
 *          ln(1/delta)/18) n/|R2| (Sec. 4.2); stop once lower/upper >= 1 - 1/e - eps or after
 *          i_max doublings. theta_cap > 0 bounds theta_i (EOVERFLOW beyond it).
 *          Round i reads only the sets (s, j) with j < n_s(theta_i) of each pool, so the pools
 *          may be grown further than a round needs without changing any result: the first
 *          growth reaches at least early_sets_per_block sets per resident RR block, and in the
 *          persistent schedule a growth goes on to later rounds' theta (doubling, at most
 *          theta0 2^i_max and the cap) while its new sets' work per block stays below the
 *          longest set of the handle's last RR launch (per-set SM cycles recorded by the RR
 *          kernel, or those of the autotuner's cache entry for the graph's profile).
 *          upper_mode HYPERIM_UPPER_PREFIX replaces the closed form (the one Alg. 4 uses) by
 *          the bound it closes, Eq. upper_2 with p_max = 1: the minimum over the greedy's
 *          prefixes S_i (0 <= i <= k) of the weighted coverage of S_i plus the k largest
 *          weighted marginal coverages of the vertices not in S_i, computed exactly on the
 *          integer greedy weights and scaled to sigma units (x 2^-32 with stratified roots,
 *          x n/|R1| with plain roots); never larger than the closed form (Lemma 5), so BRR
 *          stops no later. Also usable in FIXED mode (reported in `upper`).
 *          seconds_sample / seconds_select split the call's host wall time between growing
 *          the pools and running greedy + coverage.
 *   Greedy: marginal coverage (Eq. 2) weighted per stratum by floor(|V_s| 2^32 / n_s) (1 with
 *   plain roots), ties to the lowest vertex id, never a vertex twice; when every marginal is 0
 *   the lowest unpicked id is taken. seeds_host[k] receives S_k in pick order.
 *   Estimate: sigma = sum_s |V_s|/n_s Lambda_s (Eq. 1 per stratum).
 *   EINVAL: k < 1, k > n, bad mode; ESTATE: pools of another graph or r1 == r2.
 * ------------------------------------------------------------------------------------------ */
typedef enum { HYPERIM_SELECT_FIXED = 0, HYPERIM_SELECT_BRR = 1 } hyperim_select_mode;
typedef enum { HYPERIM_UPPER_CLOSED = 0, HYPERIM_UPPER_PREFIX = 1 } hyperim_upper_mode;

typedef struct {
    int32_t mode;        /* hyperim_select_mode */
    double eps, ell;     /* BRR only */
    uint64_t theta_cap;  /* BRR only; 0 = no cap (the i_max doublings bound theta) */
    int32_t root_mode;   /* BRR only: used when the pools are created empty */
    int32_t strategy;    /* BRR only */
    int32_t upper_mode;  /* hyperim_upper_mode (0: Eq. upper_6, the default) */
} hyperim_select_opts;

typedef struct {
    int32_t rounds;                          /* BRR rounds run (1 in FIXED mode) */
    uint64_t theta;                          /* target theta of the last round */
    uint64_t pool_r1, pool_r2;               /* RR sets of r1 / r2 the last round used: all of
                                                the pool in FIXED mode; in BRR the sets (s, j)
                                                with j < n_s(theta) (a pool another query grew
                                                further holds more) */
    uint64_t lambda_r1[HYPERIM_NSTRATA];     /* coverage of S_k in r1 per stratum */
    uint64_t lambda_r2[HYPERIM_NSTRATA];     /* coverage of S_k in r2 per stratum */
    double sigma_r1, sigma_r2;               /* Eq. 1 estimates on r1 and r2 */
    double upper, lower, alpha;              /* last round's bounds (BRR) */
    double alpha_round[64];
    double seconds_sample, seconds_select;   /* host wall time inside the call */
} hyperim_select_result;

hyperim_status hyperim_select_seeds(hyperim_graph_t g, hyperim_pool_t r1, hyperim_pool_t r2,
                                    int32_t k, const hyperim_select_opts* opts,
                                    int32_t* seeds_host, hyperim_select_result* out);

/* ------------------------------------------------------------------------------------------
 * hyperim_select_seeds_batch -- HyperIM_BRR (Alg. 4, Sec. 4.3) for many queries at once, on one
 *   GPU, round by round: in round i every query still running grows its pools to
 *   theta_i = theta_0 2^i, and the growth of all of them -- across graphs, k values and batches
 *   of uneven size -- is ONE persistent RR-kernel launch whose blocks take (graph, pool, stratum,
 *   j) jobs from a device work counter; then ONE launch runs greedy max coverage (Alg. 1, Eq. 2)
 *   on every running query's R1 view and the coverage of its seeds on its R2 view (a block per
 *   query); the host then takes each query's bounds and stop test (Eq. 1, Eq. upper_6, the
 *   Sec. 4.2 lower bound). Each query's result is the one hyperim_select_seeds in BRR mode
 *   gives it (closed upper bound, no theta cap): seeds, rounds, theta, Lambda per stratum and
 *   bounds are identical, since every round reads the prefix view j < n_s(theta_i) of its pools.
 *   queries[nq]: graph (a loaded graph or a share), r1 and r2 (two distinct empty or grown pools
 *   of that graph, same root mode and strategy), k (1 <= k <= n), eps and ell as in
 *   hyperim_select_opts; out: seeds_host[k] and *result. Queries may share pools (a graph's
 *   queries with several k: the pools grow to the largest theta any of them needs). The pools
 *   are held exclusively for the whole call. The device work runs on the first query's graph
 *   stream, which waits for the work queued on the other graphs' streams; the call returns
 *   after all of it. result->seconds_sample / seconds_select are the host wall time of the
 *   whole batch's growth and greedy steps in the rounds the query ran (shared, not its own).
 *   EINVAL: nq < 1, a null graph/pool/output, k out of range, bad eps/ell; ESTATE: a pool of
 *   another graph, r1 == r2, pools of one query that differ in root mode or strategy;
 *   EOVERFLOW: theta doubling past 2^62; errors of growth or greedy as in hyperim_sample_rr.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    hyperim_graph_t graph;
    hyperim_pool_t r1, r2;
    int32_t k;
    double eps, ell;
    int32_t* seeds_host;              /* out: k entries, S_k in pick order */
    hyperim_select_result* result;    /* out */
} hyperim_batch_query;

hyperim_status hyperim_select_seeds_batch(const hyperim_batch_query* queries, int32_t nq);

/* ------------------------------------------------------------------------------------------
 * hyperim_spread -- Eq. 1 estimate of the influence of seeds_host[k] from a pool:
 *   sigma = sum_s |V_s|/n_s Lambda_s, std_err^2 = sum_s (|V_s|/n_s)^2 n_s f_s (1 - f_s),
 *   f_s = Lambda_s / n_s. Seeds may repeat. EINVAL: a seed outside [0, n).
 * ------------------------------------------------------------------------------------------ */
hyperim_status hyperim_spread(hyperim_graph_t g, const int32_t* seeds_host, int32_t k,
                              hyperim_pool_t pool, double* sigma_hat, double* std_err);

/* ------------------------------------------------------------------------------------------
 * hyperim_forward_spread -- forward Monte-Carlo estimate of the influence of a seed set: the
 *   discrete-time cascade of Sec. 2.2 under the IC model, simulated `simulations` times.
 *   Simulation r starts with the seeds active; a vertex u activated at step i tries once, at
 *   step i + 1, each vertex v sharing a hyperedge with it; the pair u -> v is live with the
 *   probability of u's layer in A(v) (the layer keyed by w(u, v), Sec. 3.1.1) -- the same live
 *   edge the RR sampler draws for a pop of v, so E[activated] = sigma(S) of Eq. 1. Each pair
 *   draws one coin: word 0 of Philox4x32-10 with key (seed_lo, seed_hi) and counter (r, u, v,
 *   0xFFFFFFFE), live iff p = 1, or word < floor(p 2^32). Results do not depend on the order in
 *   which the GPU processes activations.
 *   seeds_host: k vertex ids (host; repeats allowed); counts_host: NULL or `simulations` entries
 *   receiving each simulation's activated count; mean / std_err: NULL or the sample mean of the
 *   counts and its standard error (sample standard deviation / sqrt(simulations); 0 when
 *   simulations = 1). EINVAL: k < 0, a seed outside [0, n), simulations = 0 or > 2^32.
 *   Synchronises the stream.
 * ------------------------------------------------------------------------------------------ */
hyperim_status hyperim_forward_spread(hyperim_graph_t g, const int32_t* seeds_host, int32_t k,
                                      uint64_t simulations, uint64_t seed, uint32_t* counts_host,
                                      double* mean, double* std_err);

/* ------------------------------------------------------------------------------------------
 * hyperim_coverage_noalloc -- per-stratum coverage of a seed set on an RR pool, computed without
 *   allocating any memory. The paper has no counterpart: it is the coverage step behind
 *   hyperim_spread and the BRR lower bound, offered to callers that cannot allocate device
 *   memory -- a serving loop whose device memory was handed out up front by its admission
 *   budget, a host application whose own allocator owns the GPU, or a latency-critical path
 *   where an allocation may wait on the device or fail under memory pressure.
 *   Inputs (device pointers, caller-owned): rr_off[count + 1] (int64), rr_mem[rr_off[count]]
 *   (int32 vertex ids), rr_stratum[count] (0..15) -- e.g. the CSR of hyperim_pool_view -- and
 *   seeds[k] (ids outside [0, n) are ignored). Inputs taken from hyperim_pool_view must stay
 *   valid until this call's work on cuda_stream has finished: no thread may grow or free that
 *   pool in the meantime (growth moves the pool's arrays and frees the old ones). Output (device, caller-owned): lambda_s[16] gets
 *   the number of RR sets of each stratum that contain a seed; the call zeroes it first.
 *   Scratch: one flag byte per vertex in a fixed array of HYPERIM_NOALLOC_MAX_N bytes built into
 *   the library; every GPU that loads the library holds those bytes until the process exits.
 *   EINVAL: n < 1 or n > HYPERIM_NOALLOC_MAX_N (the scratch is too small), count < 0, k < 0,
 *   null pointers. Never calls cudaMalloc, cudaFree or any other allocating routine.
 *   The first call on a device looks up the scratch array's device address and caches it (a
 *   set-up step): make that first call before any stream capture. The cached address belongs
 *   to the device's current context: after cudaDeviceReset the library must be reloaded (the
 *   process restarted) before this entry point is used on that device again. The work is queued on
 *   cuda_stream (NULL = legacy default stream) and the call returns without waiting. Every call
 *   uses the same scratch array, which keeps the last call's flags until the next call clears
 *   it: calls whose work overlaps on the GPU (other streams, other threads) race and return wrong
 *   counts, so order them on one stream.
 * ------------------------------------------------------------------------------------------ */
#define HYPERIM_NOALLOC_MAX_N (1u << 24)
hyperim_status hyperim_coverage_noalloc(int32_t n, const int64_t* rr_off, const int32_t* rr_mem,
                                        const uint8_t* rr_stratum, int64_t count,
                                        const int32_t* seeds, int32_t k,
                                        unsigned long long* lambda_s, void* cuda_stream);

/* ------------------------------------------------------------------------------------------
 * Query server -- influence-maximisation queries (HyperIM_BRR, Alg. 4, stratified roots) on
 *   graphs resident in HBM, served with continuous batching: `workers` host threads each run one
 *   query at a time on their own CUDA stream and their own share of each graph
 *   (hyperim_graph_share), so the kernels of up to `workers` queries overlap on the GPU; a worker
 *   that finishes takes the next queued query at once. Queries on one graph use one R1/R2 pool
 *   pair (tags 0 and 1), grown by whichever query needs more sets first; every query reads the
 *   prefix its own theta names, so its seeds, theta and estimates equal those of the same query
 *   run alone (hyperim_select_seeds on fresh pools).
 *   A worker keeps one share at a time (the RR kernel's scratch of a share holds a queue of n
 *   entries per resident block), replacing it when its next query is on another graph.
 *   Admission by HBM budget: before a query starts, if the device bytes held by the server's
 *   graphs exceed hbm_budget_bytes (0 = no limit), the pools of graphs with no running query are
 *   released (least recently used first; they are regrown on demand, with the same sets); if the
 *   total is still above the budget the query waits until a running one finishes (it starts
 *   anyway when nothing runs). Latency = submit to completion (host steady clock).
 * ------------------------------------------------------------------------------------------ */
typedef struct hyperim_server* hyperim_server_t;

typedef struct {
    int32_t workers;              /* 1..64 */
    size_t hbm_budget_bytes;      /* 0 = no admission limit */
} hyperim_server_args;

typedef struct {
    int32_t graph_id;             /* from hyperim_server_add_graph */
    int32_t k;                    /* 1 <= k <= n */
    double eps, ell;              /* as in hyperim_select_opts (BRR) */
    int32_t upper_mode;           /* hyperim_upper_mode */
} hyperim_query;

typedef struct {
    hyperim_status status;        /* the query's own status (OK or the error it met) */
    int32_t k;
    hyperim_select_result result; /* as hyperim_select_seeds fills it */
    double queued_seconds;        /* submit to start */
    double run_seconds;           /* start to completion */
    double latency_seconds;       /* submit to completion */
    int32_t worker;
} hyperim_query_result;

typedef struct {
    uint64_t submitted, completed, failed, evictions;
    double p50_latency_seconds, p99_latency_seconds, mean_latency_seconds, max_latency_seconds;
    double span_seconds;          /* first submit to last completion */
    double queries_per_second;    /* completed / span_seconds */
    uint64_t rr_sets_generated;   /* RR sets the server's pools generated (evicted pools included) */
    size_t device_bytes;          /* held by the server's graphs now */
    int32_t max_running;          /* most queries that ran at once */
} hyperim_server_stats_t;

/* EINVAL: args NULL or workers outside [1, 64]. Workers start at once. */
hyperim_status hyperim_server_create(const hyperim_server_args* args, hyperim_server_t* out);
/* Registers a loaded graph (not a share); it must outlive the server. *graph_id: 0, 1, ... */
hyperim_status hyperim_server_add_graph(hyperim_server_t s, hyperim_graph_t g, int32_t* graph_id);
/* Queues a query; returns at once. EINVAL: unknown graph_id, k outside [1, n], eps outside
 * (0, 1), ell <= 0, unknown upper_mode. */
hyperim_status hyperim_server_submit(hyperim_server_t s, const hyperim_query* q, uint64_t* ticket);
/* Blocks until the ticket's query is done; seeds_host (k entries, may be NULL) receives S_k.
 * Each ticket is waited for once. EINVAL: unknown or already collected ticket. The call
 * returns OK when the result was collected; the query's own status is out->status. */
hyperim_status hyperim_server_wait(hyperim_server_t s, uint64_t ticket, int32_t* seeds_host,
                                   hyperim_query_result* out);
hyperim_status hyperim_server_stats(hyperim_server_t s, hyperim_server_stats_t* out);
/* Finishes the running queries, drops the queued ones, frees the pools and shares. */
void hyperim_server_free(hyperim_server_t s);

/* Number of CUDA kernels this library has launched in this process (all threads, all graphs). */
uint64_t hyperim_kernel_launches(void);

/* Thread-local message describing the last non-OK status returned on this thread. */
const char* hyperim_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HYPERIM_H */
