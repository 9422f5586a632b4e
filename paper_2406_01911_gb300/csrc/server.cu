// Query server: HyperIM_BRR queries (Alg. 4 over stratified RR sets, Alg. 3, and greedy, Alg. 1)
// on resident graphs, served with continuous batching.
//
// Host code only. `workers` threads each own a CUDA stream and, per graph, a share of it
// (hyperim_graph_share): a worker runs one query at a time through hyperim_select_seeds on its
// stream, so the kernels of up to `workers` queries overlap on the GPU, and a worker that
// finishes takes the next queued query at once (no batch boundary to wait for). Queries on one
// graph grow and read one R1/R2 pool pair; a BRR round reads the prefix of the pools that its
// own theta names, so a query's result does not depend on the queries that ran before or beside
// it. Admission by HBM budget releases the pools of idle graphs (least recently used first) and
// otherwise holds a query until a running one finishes.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using clk = std::chrono::steady_clock;

struct ServerGraph {
    hyperim_graph* g = nullptr;   // the loaded graph (not a share)
    hyperim_pool* r1 = nullptr;   // tag 0, stratified roots
    hyperim_pool* r2 = nullptr;   // tag 1
    int running = 0;              // queries on this graph now
    uint64_t last_use = 0;        // logical clock of the last admission (LRU order)
    uint64_t evicted_sets = 0;    // RR sets held by pools released so far
};

struct Job {
    uint64_t ticket;
    hyperim_query q;
    clk::time_point submit;
};

struct Done {
    hyperim_query_result r;
    std::vector<int32_t> seeds;
    std::string message;          // the error text of a failed query
};

double seconds(clk::time_point a, clk::time_point b) { return std::chrono::duration<double>(b - a).count(); }

}  // namespace

struct hyperim_server {
    int workers = 0;
    size_t budget = 0;
    int device = 0;
    std::vector<cudaStream_t> streams;
    std::vector<std::map<int32_t, hyperim_graph*>> shares;  // [worker]: graph id -> its share (one at a time)
    std::deque<ServerGraph> graphs;                         // stable addresses
    std::mutex mu;
    std::condition_variable cv_job, cv_done, cv_slot;
    std::deque<Job> queue;
    std::map<uint64_t, Done> done;
    std::set<uint64_t> open;                                // submitted, not yet collected
    uint64_t next_ticket = 1, clock = 0;
    bool stop = false;
    int running = 0, max_running = 0;
    uint64_t submitted = 0, completed = 0, failed = 0, evictions = 0;
    std::vector<double> latencies;
    bool any_submit = false;
    clk::time_point first_submit, last_done;
    std::vector<std::thread> threads;

    size_t held_bytes() const {
        size_t b = 0;
        for (const ServerGraph& sg : graphs) b += sg.g->device_bytes.load();
        return b;
    }

    // releases the pools of idle graphs, least recently used first, until the budget holds
    void evict_idle() {
        std::vector<ServerGraph*> idle;
        for (ServerGraph& sg : graphs)
            if (sg.running == 0 && (sg.r1 || sg.r2)) idle.push_back(&sg);
        std::sort(idle.begin(), idle.end(),
                  [](const ServerGraph* a, const ServerGraph* b) { return a->last_use < b->last_use; });
        for (ServerGraph* sg : idle) {
            if (held_bytes() <= budget) return;
            for (hyperim_pool** p : {&sg->r1, &sg->r2}) {
                if (!*p) continue;
                sg->evicted_sets += (uint64_t)(*p)->count;
                hyperim_pool_free(*p);
                *p = nullptr;
            }
            ++evictions;
        }
    }

    void worker_main(int w);
};

void hyperim_server::worker_main(int w) {
    cudaSetDevice(device);
    for (;;) {
        Job job;
        ServerGraph* sg = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            for (;;) {
                if (stop) return;
                if (queue.empty()) {
                    cv_job.wait(lk);
                    continue;
                }
                if (budget && held_bytes() > budget) {
                    evict_idle();
                    if (held_bytes() > budget && running > 0) {
                        cv_slot.wait(lk);  // admission: wait for a running query to finish
                        continue;
                    }
                }
                job = queue.front();
                queue.pop_front();
                break;
            }
            sg = &graphs[(size_t)job.q.graph_id];
            ++sg->running;
            ++running;
            max_running = std::max(max_running, running);
            sg->last_use = ++clock;
        }
        const clk::time_point start = clk::now();
        Done d{};
        d.r.k = job.q.k;
        d.r.worker = w;
        d.seeds.assign((size_t)job.q.k, -1);
        hyperim_status st = HYPERIM_OK;
        {
            // the pools of this graph: created by the first query that needs them (host only)
            std::lock_guard<std::mutex> lk(mu);
            if (!sg->r1) st = hyperim_sample_rr(sg->g, 0, 0, HYPERIM_ROOTS_STRATIFIED, HYPERIM_STRAT_PAPER, &sg->r1);
            if (st == HYPERIM_OK && !sg->r2)
                st = hyperim_sample_rr(sg->g, 1, 0, HYPERIM_ROOTS_STRATIFIED, HYPERIM_STRAT_PAPER, &sg->r2);
        }
        // the worker's share of the graph; a worker keeps one share at a time, since the RR
        // kernel's scratch of a share grows with the graph (a queue of n entries per resident block)
        hyperim_graph* h = nullptr;
        if (st == HYPERIM_OK) {
            auto& mine = shares[(size_t)w];
            auto it = mine.find(job.q.graph_id);
            if (it != mine.end()) {
                h = it->second;
            } else {
                for (auto& kv : mine) hyperim_graph_free(kv.second);
                mine.clear();
                if ((st = hyperim_graph_share(sg->g, streams[(size_t)w], &h)) == HYPERIM_OK) mine[job.q.graph_id] = h;
            }
        }
        if (st == HYPERIM_OK) {
            hyperim_select_opts o{};
            o.mode = HYPERIM_SELECT_BRR;
            o.eps = job.q.eps;
            o.ell = job.q.ell;
            o.root_mode = HYPERIM_ROOTS_STRATIFIED;
            o.strategy = HYPERIM_STRAT_PAPER;
            o.upper_mode = job.q.upper_mode;
            st = hyperim_select_seeds(h, sg->r1, sg->r2, job.q.k, &o, d.seeds.data(), &d.r.result);
        }
        if (st != HYPERIM_OK) d.message = hyperim_last_error();
        const clk::time_point end = clk::now();
        d.r.status = st;
        d.r.queued_seconds = seconds(job.submit, start);
        d.r.run_seconds = seconds(start, end);
        d.r.latency_seconds = seconds(job.submit, end);
        {
            std::lock_guard<std::mutex> lk(mu);
            --sg->running;
            --running;
            if (st == HYPERIM_OK) ++completed; else ++failed;
            latencies.push_back(d.r.latency_seconds);
            last_done = end;
            done[job.ticket] = std::move(d);
        }
        cv_done.notify_all();
        cv_slot.notify_all();
    }
}

extern "C" {

hyperim_status hyperim_server_create(const hyperim_server_args* args, hyperim_server_t* out) {
    using namespace hyperim;
    if (!args || !out) return set_error(HYPERIM_EINVAL, "null argument");
    *out = nullptr;
    if (args->workers < 1 || args->workers > 64) return set_error(HYPERIM_EINVAL, "workers must lie in [1, 64]");
    hyperim_server* s = new (std::nothrow) hyperim_server();
    if (!s) return set_error(HYPERIM_ENOMEM, "host allocation failed");
    s->workers = args->workers;
    s->budget = args->hbm_budget_bytes;
    cudaError_t de = cudaGetDevice(&s->device);
    if (de != cudaSuccess) {
        delete s;
        return cuda_fail(de, "device query");
    }
    s->shares.resize((size_t)s->workers);
    for (int w = 0; w < s->workers; ++w) {
        cudaStream_t st = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return cuda_fail(e, "worker stream");
        }
        s->streams.push_back(st);
    }
    for (int w = 0; w < s->workers; ++w) s->threads.emplace_back([s, w] { s->worker_main(w); });
    *out = s;
    return HYPERIM_OK;
}

hyperim_status hyperim_server_add_graph(hyperim_server_t s, hyperim_graph_t g, int32_t* graph_id) {
    using namespace hyperim;
    if (!s || !g || !graph_id) return set_error(HYPERIM_EINVAL, "null argument");
    if (g->owner) return set_error(HYPERIM_EINVAL, "register the loaded graph, not a share");
    std::lock_guard<std::mutex> lk(s->mu);
    ServerGraph sg;
    sg.g = g;
    s->graphs.push_back(sg);
    *graph_id = (int32_t)s->graphs.size() - 1;
    return HYPERIM_OK;
}

hyperim_status hyperim_server_submit(hyperim_server_t s, const hyperim_query* q, uint64_t* ticket) {
    using namespace hyperim;
    if (!s || !q || !ticket) return set_error(HYPERIM_EINVAL, "null argument");
    if (q->upper_mode != HYPERIM_UPPER_CLOSED && q->upper_mode != HYPERIM_UPPER_PREFIX)
        return set_error(HYPERIM_EINVAL, "unknown upper bound mode");
    if (!(q->eps > 0.0 && q->eps < 1.0) || !(q->ell > 0.0)) return set_error(HYPERIM_EINVAL, "need 0 < eps < 1, ell > 0");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (q->graph_id < 0 || (size_t)q->graph_id >= s->graphs.size())
            return set_error(HYPERIM_EINVAL, "unknown graph id");
        if (q->k < 1 || q->k > s->graphs[(size_t)q->graph_id].g->n)
            return set_error(HYPERIM_EINVAL, "need 1 <= k <= n");
        Job j{s->next_ticket++, *q, clk::now()};
        if (!s->any_submit) {
            s->any_submit = true;
            s->first_submit = j.submit;
        }
        *ticket = j.ticket;
        s->open.insert(j.ticket);
        s->queue.push_back(j);
        ++s->submitted;
    }
    s->cv_job.notify_one();
    return HYPERIM_OK;
}

hyperim_status hyperim_server_wait(hyperim_server_t s, uint64_t ticket, int32_t* seeds_host,
                                   hyperim_query_result* out) {
    using namespace hyperim;
    if (!s || !out) return set_error(HYPERIM_EINVAL, "null argument");
    Done d;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        if (!s->open.count(ticket)) return set_error(HYPERIM_EINVAL, "unknown or already collected ticket");
        s->cv_done.wait(lk, [&] { return s->done.count(ticket) > 0 || s->stop; });
        auto it = s->done.find(ticket);
        if (it == s->done.end()) return set_error(HYPERIM_ESTATE, "server stopped before the query ran");
        d = std::move(it->second);
        s->done.erase(it);
        s->open.erase(ticket);
    }
    *out = d.r;
    if (seeds_host) std::copy(d.seeds.begin(), d.seeds.end(), seeds_host);
    if (d.r.status != HYPERIM_OK) set_error(d.r.status, d.message);  // the query's message, on this thread
    return HYPERIM_OK;
}

hyperim_status hyperim_server_stats(hyperim_server_t s, hyperim_server_stats_t* out) {
    using namespace hyperim;
    if (!s || !out) return set_error(HYPERIM_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = hyperim_server_stats_t{};
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->evictions = s->evictions;
    out->max_running = s->max_running;
    out->device_bytes = s->held_bytes();
    for (const ServerGraph& sg : s->graphs) {
        out->rr_sets_generated += sg.evicted_sets;
        if (sg.r1) out->rr_sets_generated += (uint64_t)sg.r1->count;
        if (sg.r2) out->rr_sets_generated += (uint64_t)sg.r2->count;
    }
    std::vector<double> lat = s->latencies;
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        // nearest-rank percentiles
        auto pct = [&](double q) {
            size_t r = (size_t)std::ceil(q * (double)lat.size());
            return lat[std::min(lat.size(), std::max<size_t>(r, 1)) - 1];
        };
        out->p50_latency_seconds = pct(0.50);
        out->p99_latency_seconds = pct(0.99);
        double sum = 0.0;
        for (double x : lat) sum += x;
        out->mean_latency_seconds = sum / (double)lat.size();
        out->max_latency_seconds = lat.back();
        out->span_seconds = seconds(s->first_submit, s->last_done);
        if (out->span_seconds > 0) out->queries_per_second = (double)lat.size() / out->span_seconds;
    }
    return HYPERIM_OK;
}

void hyperim_server_free(hyperim_server_t s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->queue.clear();
    }
    s->cv_job.notify_all();
    s->cv_slot.notify_all();
    s->cv_done.notify_all();
    for (std::thread& t : s->threads) t.join();
    for (auto& m : s->shares)
        for (auto& kv : m) hyperim_graph_free(kv.second);
    for (ServerGraph& sg : s->graphs) {
        hyperim_pool_free(sg.r1);
        hyperim_pool_free(sg.r2);
    }
    for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
    delete s;
}

}  // extern "C"
