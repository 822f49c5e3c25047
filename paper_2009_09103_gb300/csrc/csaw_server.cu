// csaw_server.cu -- serving sampling and walk requests over one resident graph.
//
// Requests are admitted in arrival order while their device-memory estimate
// fits the budget and a slot is free.  Each slot is a worker thread with its
// own CUDA stream, so admitted requests run concurrently and their kernels
// overlap on the GPU; a request that arrives while others run starts as soon
// as a slot and enough budget are free, without waiting for the running ones
// to finish.  Every request's draws are keyed by its own seed and its own
// instance / walker indices, so its result is the same alone or in the mix.
// The paper has no serving layer; this wraps its selection path (Sec. III-IV)
// for a stream of independent sampling and walk instances (Sec. IV-A).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "csaw_internal.cuh"

namespace csaw {

constexpr uint32_t SERVER_RESULT_TAG = 0x43535256u;   // "CSRV"

static int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket = 0;
    int32_t kind = 0;
    csaw_bias bias{};
    uint64_t rng_seed = 0;
    std::vector<uint32_t> seeds;
    std::vector<uint64_t> io;
    uint32_t n_instances = 0;
    std::vector<uint32_t> fanout;
    std::vector<uint32_t> starts;
    uint32_t length = 0;
    uint64_t estimate = 0;
    enum { PENDING, RUNNING, DONE } state = PENDING;
    csaw_result* result = nullptr;
};

// The sum of the f largest vertex degrees of the graph, from a table of the
// distinct degrees in descending order with running counts and sums: the
// most neighbours that the distinct hubs of an f-vertex frontier can have.
struct DegreeTable {
    std::vector<uint32_t> deg;       // distinct degrees, descending
    std::vector<uint64_t> count;     // vertices with degree >= deg[i]
    std::vector<uint64_t> sum;       // their degrees' sum
    uint64_t top_sum(uint64_t f) const
    {
        if (deg.empty() || f == 0) return 0;
        size_t lo = 0, hi = count.size();
        while (lo < hi) {
            const size_t mid = (lo + hi) / 2;
            if (count[mid] >= f) hi = mid; else lo = mid + 1;
        }
        if (lo == count.size()) return sum.back();
        const uint64_t before_c = lo ? count[lo - 1] : 0, before_s = lo ? sum[lo - 1] : 0;
        return before_s + (f - before_c) * deg[lo];
    }
};

static csaw_status build_degree_table(const csaw_graph* g, DegreeTable* t)
{
    std::vector<uint32_t> d(g->V);
    if (g->V) CSAW_CUDA(cudaMemcpy(d.data(), g->deg, sizeof(uint32_t) * g->V, cudaMemcpyDeviceToHost));
    std::vector<uint64_t> hist((size_t)g->max_degree + 1, 0);
    for (uint32_t x : d) ++hist[x <= g->max_degree ? x : g->max_degree];
    uint64_t c = 0, sm = 0;
    for (uint64_t x = g->max_degree; x >= 1; --x) {
        if (!hist[x]) continue;
        c += hist[x];
        sm += hist[x] * x;
        t->deg.push_back((uint32_t)x);
        t->count.push_back(c);
        t->sum.push_back(sm);
    }
    return CSAW_OK;
}

// Device bytes a request may hold at once (an upper bound of what csaw_walk
// or csaw_sample allocates for it).
static uint64_t estimate_bytes(const csaw_graph* g, const DegreeTable& dt, const Request& r)
{
    if (r.kind == CSAW_REQ_WALK) {
        const uint64_t n = r.starts.size();
        return 4 * n + 4 * n * ((uint64_t)r.length + 1) + 4096;
    }
    const uint64_t S = r.seeds.size();
    const uint32_t depth = (uint32_t)r.fanout.size();
    uint64_t b = 4 * S + 8 * ((uint64_t)r.n_instances + 1) + 64 * 1024;
    b += 16 * (uint64_t)depth * r.n_instances + 8;   // offsets and sizes
    b += 28 * S + 8;                                 // seed keys, sort, compaction
    bool big_k = false;
    for (uint32_t l = 0; l < depth; ++l) big_k |= r.fanout[l] > 256 && r.fanout[l] != CSAW_FANOUT_ALL;
    if (g->max_degree > 8192 && big_k)               // per-CTA slots of long rows
        b += (uint64_t)g->sm_count * 4 * ((uint64_t)g->max_degree * 8 + g->max_degree / 8 + 8);
    uint64_t f = S, hub = 0;
    for (uint32_t l = 0; l < depth; ++l) {
        const uint64_t k = r.fanout[l] < g->max_degree ? r.fanout[l] : g->max_degree;
        const uint64_t e = f * k;
        b += f * 36 + 8 * (uint64_t)(r.n_instances + 1);   // frontier keys, counts, lists, positions
        b += e * 8;                                         // sampled edges
        if (l + 1 < depth) b += e * 28;                     // candidates, sort, compaction
        // hub grouping and shared hub prefix sums, held for one layer at a time
        const uint64_t h = 60 * f + 8 * dt.top_sum(f) + 64;
        if (h > hub) hub = h;
        f = e;
    }
    return b + hub;
}

static csaw_result* new_result(const Request& r)
{
    csaw_result* res = new (std::nothrow) csaw_result();
    if (!res) return nullptr;
    std::memset(res, 0, sizeof(*res));
    res->tag = SERVER_RESULT_TAG;
    res->kind = r.kind;
    res->device_bytes_estimate = r.estimate;
    return res;
}

void free_server_result(void* p)
{
    csaw_result* r = (csaw_result*)p;
    if (!r || r->tag != SERVER_RESULT_TAG) return;
    delete[] r->edge_offsets;
    delete[] r->frontier_sizes;
    delete[] r->src;
    delete[] r->dst;
    delete[] r->path;
    r->tag = 0;
    delete r;
}

// Runs one request on stream s; fills res (status and host arrays).
static void execute(csaw_graph* g, Request& rq, csaw_result* res, cudaStream_t s)
{
    if (rq.kind == CSAW_REQ_WALK) {
        const uint64_t n = rq.starts.size();
        res->n_walkers = n;
        res->length = rq.length;
        res->path = new (std::nothrow) uint32_t[n * ((uint64_t)rq.length + 1) + 1];
        if (!res->path) { res->status = CSAW_ERR_NOMEM; return; }
        res->status = csaw_walk(g, rq.starts.data(), n, rq.length, &rq.bias, rq.rng_seed, res->path,
                                CSAW_MEM_HOST, s);
        return;
    }
    csaw_sample_result* sr = nullptr;
    res->status = csaw_sample(g, rq.seeds.data(), rq.io.data(), rq.n_instances, (uint32_t)rq.fanout.size(),
                              rq.fanout.data(), &rq.bias, rq.rng_seed, CSAW_MEM_HOST, s, &sr);
    if (res->status != CSAW_OK) return;
    csaw_sample_view v;
    csaw_sample_get_view(sr, &v);
    res->depth = v.depth;
    res->n_instances = v.n_instances;
    res->n_edges = v.n_edges;
    const uint64_t ng = (uint64_t)v.depth * v.n_instances;
    res->edge_offsets = new (std::nothrow) uint64_t[ng + 1];
    res->frontier_sizes = new (std::nothrow) uint64_t[ng + 1];
    res->src = new (std::nothrow) uint32_t[v.n_edges + 1];
    res->dst = new (std::nothrow) uint32_t[v.n_edges + 1];
    if (!res->edge_offsets || !res->frontier_sizes || !res->src || !res->dst) {
        res->status = CSAW_ERR_NOMEM;
    } else {
        std::memcpy(res->edge_offsets, v.edge_offsets, sizeof(uint64_t) * (ng + 1));
        std::memcpy(res->frontier_sizes, v.frontier_sizes, sizeof(uint64_t) * (ng ? ng : 1));
        res->status = csaw_sample_copy_edges(sr, res->src, res->dst);
    }
    csaw_result_free(sr);
}

}  // namespace csaw

using namespace csaw;

struct csaw_server {
    csaw_graph* g = nullptr;
    DegreeTable degrees;
    uint64_t budget = 0;
    uint32_t slots = 0;
    std::mutex mu;
    std::condition_variable cv_work;
    std::condition_variable cv_done;
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> reqs;
    uint64_t next_ticket = 1;
    uint64_t in_use = 0;
    uint32_t running = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;

    void worker(uint32_t slot)
    {
        cudaSetDevice(g->device);
        cudaStream_t s = streams[slot];
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            cv_work.wait(lk, [&] {
                return stop || (!pending.empty() && in_use + pending.front()->estimate <= budget);
            });
            if (stop && pending.empty()) break;
            if (stop) {
                // shutting down: pending requests are aborted by destroy
                break;
            }
            Request* rq = pending.front();
            pending.pop_front();
            in_use += rq->estimate;
            ++running;
            rq->state = Request::RUNNING;
            rq->result->t_admit_ns = now_ns();
            lk.unlock();
            rq->result->t_start_ns = now_ns();
            execute(g, *rq, rq->result, s);
            rq->result->t_finish_ns = now_ns();
            lk.lock();
            in_use -= rq->estimate;
            --running;
            rq->state = Request::DONE;
            cv_done.notify_all();
            cv_work.notify_all();
        }
    }
};

extern "C" csaw_status csaw_server_create(csaw_graph* g, const csaw_server_opts* opts, csaw_server** out)
{
    clear_error();
    if (!out) return fail(CSAW_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!g || !opts) return fail(CSAW_ERR_INVALID, "NULL argument");
    if (opts->slots == 0 || opts->slots > 256) return fail(CSAW_ERR_INVALID, "slots must be 1..256");
    if (opts->budget_bytes == 0) return fail(CSAW_ERR_INVALID, "budget must be positive");
    csaw_server* sv = new (std::nothrow) csaw_server();
    if (!sv) return fail(CSAW_ERR_NOMEM, "host allocation failed");
    sv->g = g;
    sv->budget = opts->budget_bytes;
    sv->slots = opts->slots;
    cudaError_t e = cudaSetDevice(g->device);
    if (e == cudaSuccess) {
        const csaw_status st = build_degree_table(g, &sv->degrees);
        if (st != CSAW_OK) { delete sv; return st; }
    }
    for (uint32_t i = 0; e == cudaSuccess && i < opts->slots; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) sv->streams.push_back(st);
    }
    if (e != cudaSuccess) {
        for (auto st : sv->streams) cudaStreamDestroy(st);
        delete sv;
        return cuda_fail(e, "cudaStreamCreate(server)");
    }
    for (uint32_t i = 0; i < opts->slots; ++i) sv->workers.emplace_back([sv, i] { sv->worker(i); });
    *out = sv;
    return CSAW_OK;
}

extern "C" csaw_status csaw_server_destroy(csaw_server* sv)
{
    clear_error();
    if (!sv) return CSAW_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        for (Request* rq : sv->pending) {
            rq->state = Request::DONE;
            rq->result->status = CSAW_ERR_ABORTED;
        }
        sv->pending.clear();
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->workers) t.join();
    for (auto& kv : sv->reqs) {
        free_server_result(kv.second->result);
        delete kv.second;
    }
    for (auto st : sv->streams) cudaStreamDestroy(st);
    delete sv;
    return CSAW_OK;
}

extern "C" csaw_status csaw_submit(csaw_server* sv, const csaw_request* r, uint64_t* ticket)
{
    clear_error();
    if (!sv || !r || !ticket) return fail(CSAW_ERR_INVALID, "NULL argument");
    Request* rq = new (std::nothrow) Request();
    if (!rq) return fail(CSAW_ERR_NOMEM, "host allocation failed");
    rq->kind = r->kind;
    rq->bias = r->bias;
    rq->rng_seed = r->rng_seed;
    int kind;
    csaw_status st = check_bias(sv->g, &r->bias, r->kind == CSAW_REQ_WALK, &kind);
    if (st == CSAW_OK && r->kind == CSAW_REQ_WALK) {
        if (r->n_walkers && !r->starts) st = fail(CSAW_ERR_INVALID, "starts is NULL");
        else rq->starts.assign(r->starts, r->starts + r->n_walkers);
        rq->length = r->length;
        for (uint64_t i = 0; st == CSAW_OK && i < r->n_walkers; ++i)
            if (r->starts[i] >= sv->g->V) st = fail(CSAW_ERR_INVALID, "start %llu out of range", (unsigned long long)i);
    } else if (st == CSAW_OK && r->kind == CSAW_REQ_SAMPLE) {
        if (!r->inst_offsets || !r->fanout) st = fail(CSAW_ERR_INVALID, "inst_offsets/fanout is NULL");
        else if (r->depth < 1 || r->depth > CSAW_MAX_DEPTH) st = fail(CSAW_ERR_INVALID, "depth must be 1..%u", CSAW_MAX_DEPTH);
        else {
            rq->n_instances = r->n_instances;
            rq->io.assign(r->inst_offsets, r->inst_offsets + (size_t)r->n_instances + 1);
            rq->fanout.assign(r->fanout, r->fanout + r->depth);
            const uint64_t ns = rq->io.back();
            if (rq->io[0] != 0) st = fail(CSAW_ERR_INVALID, "inst_offsets must start at 0");
            else if (ns && !r->seeds) st = fail(CSAW_ERR_INVALID, "seeds is NULL");
            else rq->seeds.assign(r->seeds, r->seeds + ns);
        }
    } else if (st == CSAW_OK) {
        st = fail(CSAW_ERR_INVALID, "unknown request kind %d", r->kind);
    }
    if (st != CSAW_OK) { delete rq; return st; }
    rq->estimate = estimate_bytes(sv->g, sv->degrees, *rq);
    if (rq->estimate > sv->budget) {
        const uint64_t est = rq->estimate;
        delete rq;
        return fail(CSAW_ERR_NOMEM, "request needs up to %llu device bytes, the budget is %llu",
                    (unsigned long long)est, (unsigned long long)sv->budget);
    }
    rq->result = new_result(*rq);
    if (!rq->result) { delete rq; return fail(CSAW_ERR_NOMEM, "host allocation failed"); }
    rq->result->t_submit_ns = now_ns();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            free_server_result(rq->result);
            delete rq;
            return fail(CSAW_ERR_ABORTED, "server is shutting down");
        }
        rq->ticket = sv->next_ticket++;
        sv->reqs[rq->ticket] = rq;
        sv->pending.push_back(rq);
        *ticket = rq->ticket;
    }
    sv->cv_work.notify_all();
    return CSAW_OK;
}

extern "C" csaw_status csaw_poll(csaw_server* sv, uint64_t ticket, int64_t timeout_us, csaw_result** out)
{
    clear_error();
    if (!sv || !out) return fail(CSAW_ERR_INVALID, "NULL argument");
    *out = nullptr;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return fail(CSAW_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Request* rq = it->second;
    auto done = [&] { return rq->state == Request::DONE; };
    if (timeout_us < 0) sv->cv_done.wait(lk, done);
    else if (!sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done))
        return fail(CSAW_ERR_TIMEOUT, "request %llu not finished", (unsigned long long)ticket);
    sv->reqs.erase(it);
    *out = rq->result;
    const csaw_status st = rq->result->status;
    delete rq;
    if (st != CSAW_OK) fail(st, "request %llu failed with status %d", (unsigned long long)ticket, (int)st);
    return st;
}

extern "C" csaw_status csaw_cancel(csaw_server* sv, uint64_t ticket)
{
    clear_error();
    if (!sv) return fail(CSAW_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return fail(CSAW_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Request* rq = it->second;
    if (rq->state != Request::PENDING) return fail(CSAW_ERR_INVALID, "request %llu already started", (unsigned long long)ticket);
    for (auto q = sv->pending.begin(); q != sv->pending.end(); ++q)
        if (*q == rq) { sv->pending.erase(q); break; }
    rq->state = Request::DONE;
    rq->result->status = CSAW_ERR_ABORTED;
    rq->result->t_finish_ns = now_ns();
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
    return CSAW_OK;
}

extern "C" csaw_status csaw_server_stats(csaw_server* sv, csaw_server_stats_t* out)
{
    clear_error();
    if (!sv || !out) return fail(CSAW_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    out->pending = (uint32_t)sv->pending.size();
    out->running = sv->running;
    out->bytes_in_use = sv->in_use;
    out->budget_bytes = sv->budget;
    return CSAW_OK;
}
