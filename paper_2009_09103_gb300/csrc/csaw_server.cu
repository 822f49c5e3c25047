// csaw_server.cu -- serving sampling and walk requests over one resident graph.
//
// Requests are admitted in arrival order while their device-memory estimate
// fits the budget and a slot is free.  Each slot is a worker thread with its
// own CUDA stream, so admitted requests run concurrently and their kernels
// overlap on the GPU; a request that arrives while others run starts as soon
// as a slot and enough budget are free, without waiting for the running ones
// to finish.  A slot that frees up takes the oldest waiting request together
// with the other waiting requests of the same kind and bias (continuous
// batching): their instances, or walkers, run as one multi-instance launch --
// the batched multi-instance sampling of Sec. V-B -- with each request's own
// seed and its own instance / walker indices in the draws, so every result
// is the same alone, in a batch or in the mix.  Inputs go in and results come
// out through each slot's pinned staging buffer.  The paper has no serving
// layer; this runs its selection path (Sec. III-IV) for a stream of
// independent sampling and walk instances (Sec. IV-A).
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
    bool large = false;            // more than SMALL_BATCH_EDGES sampled edges possible: low priority
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

// Page-locked host blocks for the arrays of request results, kept for reuse
// for the life of the process in power-of-two classes from 64 KiB and carved
// from slabs of at least 256 MiB (one cudaHostAlloc per slab): a result's
// edges or path are copied from the device straight into one (DMA at the
// link's rate, with no staging copy and no first-touch faults on the host),
// and the block goes back to its class when the result is freed.
struct PinnedPool {
    static constexpr int MIN_CLASS = 16;
    static constexpr size_t SLAB = (size_t)256 << 20;
    std::mutex mu;
    std::vector<std::vector<void*>> free_by_class = std::vector<std::vector<void*>>(64);
    unsigned char* slab = nullptr;
    size_t slab_left = 0;
    // A block of at least `bytes` bytes and its class, or null (class -1)
    // when page-locked memory is refused.
    void* get(size_t bytes, int* cls)
    {
        int c = MIN_CLASS;
        while (c < 62 && ((size_t)1 << c) < bytes) ++c;
        const size_t size = (size_t)1 << c;
        *cls = -1;
        std::lock_guard<std::mutex> lk(mu);
        auto& f = free_by_class[c];
        if (!f.empty()) {
            void* p = f.back();
            f.pop_back();
            *cls = c;
            return p;
        }
        if (slab_left < size) {
            void* p = nullptr;
            const size_t n = size > SLAB ? size : SLAB;
            if (cudaHostAlloc(&p, n, cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            slab = (unsigned char*)p;   // the rest of the previous slab stays unused
            slab_left = n;
        }
        void* p = slab;
        slab += size;
        slab_left -= size;
        *cls = c;
        return p;
    }
    void put(void* p, int cls)
    {
        std::lock_guard<std::mutex> lk(mu);
        free_by_class[cls].push_back(p);
    }
};

static PinnedPool* result_pool()
{
    static PinnedPool* pool = new PinnedPool();   // never freed: results may outlive every server
    return pool;
}

// A server result: the caller's view first, then where its arrays came from.
struct ServerResult {
    csaw_result pub;
    int cls[5] = {-1, -1, -1, -1, -1};   // edge_offsets, frontier_sizes, src, dst, path (-1: new[])
};

// An array of n elements of T for result slot k: from the pool, or new[].
template <class T>
static T* result_array(ServerResult* r, int k, uint64_t n)
{
    int cls = -1;
    void* p = result_pool()->get(sizeof(T) * (size_t)n, &cls);
    r->cls[k] = cls;
    if (p) return (T*)p;
    return new (std::nothrow) T[n];
}

static csaw_result* new_result(const Request& r)
{
    ServerResult* res = new (std::nothrow) ServerResult();
    if (!res) return nullptr;
    std::memset(&res->pub, 0, sizeof(res->pub));
    res->pub.tag = SERVER_RESULT_TAG;
    res->pub.kind = r.kind;
    res->pub.device_bytes_estimate = r.estimate;
    return &res->pub;
}

void free_server_result(void* p)
{
    csaw_result* r = (csaw_result*)p;
    if (!r || r->tag != SERVER_RESULT_TAG) return;
    ServerResult* sr = reinterpret_cast<ServerResult*>(r);
    void* arrays[5] = {r->edge_offsets, r->frontier_sizes, r->src, r->dst, r->path};
    for (int k = 0; k < 5; ++k) {
        if (!arrays[k]) continue;
        if (sr->cls[k] >= 0) result_pool()->put(arrays[k], sr->cls[k]);
        else if (k < 2) delete[] (uint64_t*)arrays[k];
        else delete[] (uint32_t*)arrays[k];
    }
    r->tag = 0;
    delete sr;
}

// One slot: two streams and a pinned staging buffer (grown on demand).
// Small batches run on the high-priority stream, so that their blocks are
// scheduled ahead of the waiting blocks of large batches in other slots;
// the batched walk kernels keep their blocks short for the same reason.
struct Lane {
    cudaStream_t lo = nullptr, hi = nullptr;
    cudaStream_t s = nullptr;          // the stream of the current batch
    unsigned char* pin = nullptr;
    size_t pin_cap = 0;
};

constexpr uint64_t SMALL_BATCH_EDGES = 1ull << 18;   // at most this many sampled edges: high priority

static csaw_status lane_pinned(Lane& L, size_t bytes)
{
    if (bytes <= L.pin_cap) return CSAW_OK;
    if (L.pin) {
        CSAW_CUDA(cudaStreamSynchronize(L.s));
        cudaFreeHost(L.pin);
        L.pin = nullptr;
        L.pin_cap = 0;
    }
    size_t cap = bytes < (1u << 20) ? (1u << 20) : bytes;
    cap += cap / 4;
    void* p = nullptr;
    CSAW_CUDA(cudaHostAlloc(&p, cap, cudaHostAllocDefault));
    L.pin = (unsigned char*)p;
    L.pin_cap = cap;
    return CSAW_OK;
}

static inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Walk requests of one bias in one launch.  Inputs are packed in the staging
// buffer as [segment starts u64 (R+1) | row offsets u64 (R) | lengths u32 (R)
// | keys u32 (2R) | start vertices u32 (n)], copied in once; each request's
// path matrix is copied straight into its result.  A batch of one runs the
// walk kernels of csaw_walk; larger batches run their batched forms, with
// persistent grids (short-lived blocks were measured slower: a block holds
// its SM until its slowest walker is done).
static csaw_status execute_walks(csaw_graph* g, Lane& L, std::vector<Request*>& batch)
{
    const size_t R = batch.size();
    uint64_t n = 0, rows = 0;
    uint32_t max_len = 0;
    for (Request* rq : batch) {
        n += rq->starts.size();
        rows += (uint64_t)rq->starts.size() * ((uint64_t)rq->length + 1);
        max_len = rq->length > max_len ? rq->length : max_len;
    }
    const size_t o_start = 0, o_row0 = align16(o_start + 8 * (R + 1)), o_len = align16(o_row0 + 8 * R);
    const size_t o_key = align16(o_len + 4 * R), o_starts = align16(o_key + 8 * R);
    const size_t in_bytes = align16(o_starts + 4 * n);
    const size_t out_bytes = 4 * rows;
    CSAW_TRY(lane_pinned(L, in_bytes));
    uint64_t* h_start = (uint64_t*)(L.pin + o_start);
    uint64_t* h_row0 = (uint64_t*)(L.pin + o_row0);
    uint32_t* h_len = (uint32_t*)(L.pin + o_len);
    uint32_t* h_key = (uint32_t*)(L.pin + o_key);
    uint32_t* h_starts = (uint32_t*)(L.pin + o_starts);
    uint64_t w = 0, row = 0;
    for (size_t r = 0; r < R; ++r) {
        const Request* rq = batch[r];
        h_start[r] = w;
        h_row0[r] = row;
        h_len[r] = rq->length;
        h_key[2 * r] = (uint32_t)rq->rng_seed;
        h_key[2 * r + 1] = (uint32_t)(rq->rng_seed >> 32);
        if (!rq->starts.empty()) std::memcpy(h_starts + w, rq->starts.data(), 4 * rq->starts.size());
        w += rq->starts.size();
        row += (uint64_t)rq->starts.size() * ((uint64_t)rq->length + 1);
    }
    h_start[R] = w;
    void* d_in = nullptr;
    void* d_path = nullptr;
    CSAW_TRY(dalloc(&d_in, in_bytes, L.s));
    csaw_status st = dalloc(&d_path, out_bytes ? out_bytes : 4, L.s);
    if (st == CSAW_OK) {
        cudaError_t e = cudaMemcpyAsync(d_in, L.pin, in_bytes, cudaMemcpyHostToDevice, L.s);
        if (e != cudaSuccess) st = cuda_fail(e, "copy walk batch in");
    }
    if (st == CSAW_OK) {
        unsigned char* d = (unsigned char*)d_in;
        WalkSegments seg;
        seg.start = (const uint64_t*)(d + o_start);
        seg.row0 = (const uint64_t*)(d + o_row0);
        seg.len = (const uint32_t*)(d + o_len);
        seg.key = (const uint32_t*)(d + o_key);
        seg.n = (uint32_t)R;
        seg.warp_budget = 0;
        if (R == 1) {
            const Request* rq = batch[0];
            st = csaw_walk(g, (const uint32_t*)(d + o_starts), n, rq->length, &rq->bias, rq->rng_seed,
                           (uint32_t*)d_path, CSAW_MEM_DEVICE, L.s);
        } else {
            st = walk_batch(g, &batch[0]->bias, (const uint32_t*)(d + o_starts), n, seg, max_len,
                            (uint32_t*)d_path, L.s);
        }
    }
    row = 0;
    for (size_t r = 0; st == CSAW_OK && r < R; ++r) {
        Request* rq = batch[r];
        csaw_result* res = rq->result;
        const uint64_t cnt = (uint64_t)rq->starts.size() * ((uint64_t)rq->length + 1);
        res->n_walkers = rq->starts.size();
        res->length = rq->length;
        res->path = result_array<uint32_t>(reinterpret_cast<ServerResult*>(res), 4, cnt + 1);
        if (!res->path) {
            res->status = CSAW_ERR_NOMEM;
        } else {
            res->status = CSAW_OK;
            if (cnt) {
                cudaError_t e = cudaMemcpyAsync(res->path, (const uint32_t*)d_path + row, 4 * cnt,
                                                cudaMemcpyDeviceToHost, L.s);
                if (e != cudaSuccess) st = cuda_fail(e, "copy paths out");
            }
        }
        row += cnt;
    }
    dfree(d_in, L.s);
    dfree(d_path, L.s);
    if (st == CSAW_OK) {
        cudaError_t e = cudaStreamSynchronize(L.s);
        if (e != cudaSuccess) st = cuda_fail(e, "walk batch");
    }
    (void)out_bytes;
    return st;
}

// Sampling requests of one bias in one multi-instance run.  The batch's
// instances are the requests' instances in order; the tables give each one
// its request's key, its own index and its request's fanout per layer (0
// past the request's depth).  Inputs are packed as [instance offsets u64
// (N+1) | keys u32 (2N) | indices u32 (N) | fanouts u32 (depth N) | seeds u32
// (S)]; each request's edges are copied straight into its result, one copy
// per layer for src and one for dst.
static csaw_status execute_samples(csaw_graph* g, Lane& L, std::vector<Request*>& batch)
{
    uint64_t N = 0, S = 0;
    uint32_t depth = 0;
    for (Request* rq : batch) {
        N += rq->n_instances;
        S += rq->seeds.size();
        depth = (uint32_t)rq->fanout.size() > depth ? (uint32_t)rq->fanout.size() : depth;
    }
    if (N >= 0xFFFFFFFFull || S >= 0xFFFFFFFFull) return fail(CSAW_ERR_INVALID, "batch too large");
    const size_t o_io = 0, o_key = align16(8 * (N + 1)), o_id = align16(o_key + 8 * N);
    const size_t o_fan = align16(o_id + 4 * N), o_seeds = align16(o_fan + 4 * (size_t)depth * N);
    const size_t in_bytes = align16(o_seeds + 4 * S);
    CSAW_TRY(lane_pinned(L, in_bytes));
    uint64_t* h_io = (uint64_t*)(L.pin + o_io);
    uint32_t* h_key = (uint32_t*)(L.pin + o_key);
    uint32_t* h_id = (uint32_t*)(L.pin + o_id);
    uint32_t* h_fan = (uint32_t*)(L.pin + o_fan);
    uint32_t* h_seeds = (uint32_t*)(L.pin + o_seeds);
    std::vector<uint32_t> fan_max(depth, 0);
    uint64_t i0 = 0, s0 = 0;
    for (Request* rq : batch) {
        for (uint32_t i = 0; i < rq->n_instances; ++i) {
            h_io[i0 + i] = s0 + rq->io[i];
            h_key[2 * (i0 + i)] = (uint32_t)rq->rng_seed;
            h_key[2 * (i0 + i) + 1] = (uint32_t)(rq->rng_seed >> 32);
            h_id[i0 + i] = i;
            for (uint32_t l = 0; l < depth; ++l)
                h_fan[(uint64_t)l * N + i0 + i] = l < rq->fanout.size() ? rq->fanout[l] : 0u;
        }
        for (uint32_t l = 0; l < rq->fanout.size(); ++l)
            fan_max[l] = rq->fanout[l] > fan_max[l] ? rq->fanout[l] : fan_max[l];
        if (!rq->seeds.empty()) std::memcpy(h_seeds + s0, rq->seeds.data(), 4 * rq->seeds.size());
        i0 += rq->n_instances;
        s0 += rq->seeds.size();
    }
    h_io[N] = S;
    int kind;
    CSAW_TRY(check_bias(g, &batch[0]->bias, false, &kind));
    void* d_in = nullptr;
    CSAW_TRY(dalloc(&d_in, in_bytes, L.s));
    csaw_sample_result* R = nullptr;
    csaw_status st = CSAW_OK;
    cudaError_t e = cudaMemcpyAsync(d_in, L.pin, in_bytes, cudaMemcpyHostToDevice, L.s);
    if (e != cudaSuccess) st = cuda_fail(e, "copy sample batch in");
    if (st == CSAW_OK) {
        unsigned char* d = (unsigned char*)d_in;
        SampleTables t;
        t.inst_key = (const uint32_t*)(d + o_key);
        t.inst_id = (const uint32_t*)(d + o_id);
        t.inst_fan = (const uint32_t*)(d + o_fan);
        st = sample_batch(g, (const uint32_t*)(d + o_seeds), (const uint64_t*)(d + o_io), (uint32_t)N, S, depth,
                          fan_max.data(), t, kind, L.s, &R);
    }
    dfree(d_in, L.s);
    if (st != CSAW_OK) return st;
    csaw_sample_view v;
    csaw_sample_get_view(R, &v);
    // each request: its instances' edges of its own layers, in csaw_sample's layout
    i0 = 0;
    for (Request* rq : batch) {
        csaw_result* res = rq->result;
        const uint32_t n = rq->n_instances, dep = (uint32_t)rq->fanout.size();
        const uint64_t ng = (uint64_t)dep * n;
        uint64_t total = 0;
        for (uint32_t l = 0; l < dep; ++l)
            total += v.edge_offsets[(uint64_t)l * N + i0 + n] - v.edge_offsets[(uint64_t)l * N + i0];
        res->depth = dep;
        res->n_instances = n;
        res->n_edges = total;
        ServerResult* sr = reinterpret_cast<ServerResult*>(res);
        res->edge_offsets = result_array<uint64_t>(sr, 0, ng + 1);
        res->frontier_sizes = result_array<uint64_t>(sr, 1, ng + 1);
        res->src = result_array<uint32_t>(sr, 2, total + 1);
        res->dst = result_array<uint32_t>(sr, 3, total + 1);
        if (!res->edge_offsets || !res->frontier_sizes || !res->src || !res->dst) {
            res->status = CSAW_ERR_NOMEM;
        } else {
            res->status = CSAW_OK;
            uint64_t at = 0;
            for (uint32_t l = 0; st == CSAW_OK && l < dep; ++l) {
                const uint64_t* eo = v.edge_offsets + (uint64_t)l * N + i0;
                const uint64_t layer0 = v.edge_offsets[(uint64_t)l * N];
                for (uint32_t i = 0; i < n; ++i) {
                    res->edge_offsets[(uint64_t)l * n + i] = at + (eo[i] - eo[0]);
                    res->frontier_sizes[(uint64_t)l * n + i] = v.frontier_sizes[(uint64_t)l * N + i0 + i];
                }
                const uint64_t cnt = eo[n] - eo[0];
                if (cnt) {
                    e = cudaMemcpyAsync(res->src + at, v.src[l] + (eo[0] - layer0), 4 * cnt,
                                        cudaMemcpyDeviceToHost, L.s);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(res->dst + at, v.dst[l] + (eo[0] - layer0), 4 * cnt,
                                            cudaMemcpyDeviceToHost, L.s);
                    if (e != cudaSuccess) st = cuda_fail(e, "copy edges out");
                }
                at += cnt;
            }
            res->edge_offsets[ng] = total;
        }
        i0 += n;
    }
    if (st == CSAW_OK) {
        e = cudaStreamSynchronize(L.s);
        if (e != cudaSuccess) st = cuda_fail(e, "sample batch");
    }
    free_sample_result_on(R, L.s);   // csaw_result_free would wait for every slot's kernels
    return st;
}


// Sampled edges a request produces at most: walk steps; for sampling, per
// layer the smaller of frontier x fanout and the degrees of the frontier's
// largest possible rows (the visited filter is not counted).
static uint64_t edge_bound(const csaw_graph* g, const DegreeTable& dt, const Request* rq)
{
    if (rq->kind == CSAW_REQ_WALK) return (uint64_t)rq->starts.size() * rq->length;
    const uint64_t f_max = (uint64_t)g->V * (rq->n_instances ? rq->n_instances : 1);
    uint64_t f = rq->seeds.size(), total = 0;
    for (uint32_t k : rq->fanout) {
        uint64_t e = f > (1ull << 40) / (k ? k : 1) ? (1ull << 40) : f * k;
        const uint64_t rows = dt.top_sum(f < g->V ? f : g->V) * (f / (g->V ? g->V : 1) + 1);
        e = e < rows ? e : rows;
        total += e;
        f = e < f_max ? e : f_max;
    }
    return total;
}

// Runs a batch (one kind, one bias) on the slot; fills every request's result.
static void execute(csaw_graph* g, Lane& L, std::vector<Request*>& batch)
{
    L.s = batch[0]->large ? L.lo : L.hi;
    const csaw_status st = batch[0]->kind == CSAW_REQ_WALK ? execute_walks(g, L, batch)
                                                            : execute_samples(g, L, batch);
    if (st != CSAW_OK)
        for (Request* rq : batch) rq->result->status = st;
}

static bool same_bias(const csaw_bias& a, const csaw_bias& b)
{
    return a.kind == b.kind && (a.kind != CSAW_BIAS_NODE2VEC ||
                                (a.n2v_mult[0] == b.n2v_mult[0] && a.n2v_mult[1] == b.n2v_mult[1] &&
                                 a.n2v_mult[2] == b.n2v_mult[2]));
}

}  // namespace csaw

using namespace csaw;

struct csaw_server {
    csaw_graph* g = nullptr;
    DegreeTable degrees;
    uint64_t budget = 0;
    uint32_t slots = 0;
    uint32_t max_batch = 32;
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
    std::vector<Lane> lanes;

    // The oldest waiting request whose estimate fits the budget.  Called
    // with mu held.
    std::deque<Request*>::iterator startable()
    {
        for (auto it = pending.begin(); it != pending.end(); ++it)
            if (in_use + (*it)->estimate <= budget) return it;
        return pending.end();
    }

    // That request, then (up to max_batch in all) every other waiting request
    // of the same kind, bias and class whose estimate still fits the budget,
    // in arrival order.  Called with mu held.
    void take_batch(std::vector<Request*>& batch)
    {
        batch.clear();
        auto first = startable();
        Request* head = *first;
        pending.erase(first);
        batch.push_back(head);
        uint64_t est = head->estimate;
        uint64_t items = head->kind == CSAW_REQ_WALK ? head->starts.size() : head->n_instances;
        uint64_t seeds = head->seeds.size();
        for (auto it = pending.begin(); it != pending.end() && batch.size() < max_batch;) {
            Request* rq = *it;
            const uint64_t more = rq->kind == CSAW_REQ_WALK ? rq->starts.size() : rq->n_instances;
            if (rq->kind == head->kind && same_bias(rq->bias, head->bias) && rq->large == head->large &&
                in_use + est + rq->estimate <= budget && items + more < 0x7FFFFFFFull &&
                seeds + rq->seeds.size() < 0x7FFFFFFFull) {
                batch.push_back(rq);
                est += rq->estimate;
                items += more;
                seeds += rq->seeds.size();
                it = pending.erase(it);
            } else {
                ++it;
            }
        }
    }

    void worker(uint32_t slot)
    {
        cudaSetDevice(g->device);
        AllocScope alloc_scope(g);   // request buffers through the graph's allocator, if set
        Lane& L = lanes[slot];
        std::vector<Request*> batch;
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            cv_work.wait(lk, [&] { return stop || startable() != pending.end(); });
            if (stop) break;   // pending requests are aborted by destroy
            take_batch(batch);
            const int64_t t_admit = now_ns();
            for (Request* rq : batch) {
                in_use += rq->estimate;
                ++running;
                rq->state = Request::RUNNING;
                rq->result->t_admit_ns = t_admit;
            }
            lk.unlock();
            const int64_t t_start = now_ns();
            for (Request* rq : batch) rq->result->t_start_ns = t_start;
            execute(g, L, batch);
            const int64_t t_finish = now_ns();
            lk.lock();
            for (Request* rq : batch) {
                rq->result->t_finish_ns = t_finish;
                in_use -= rq->estimate;
                --running;
                rq->state = Request::DONE;
            }
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
    sv->max_batch = opts->max_batch ? opts->max_batch : 32;
    cudaError_t e = cudaSetDevice(g->device);
    if (e == cudaSuccess) {
        const csaw_status st = build_degree_table(g, &sv->degrees);
        if (st != CSAW_OK) { delete sv; return st; }
    }
    sv->lanes.resize(opts->slots);
    int prio_lo = 0, prio_hi = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    for (uint32_t i = 0; e == cudaSuccess && i < opts->slots; ++i) {
        e = cudaStreamCreateWithPriority(&sv->lanes[i].lo, cudaStreamNonBlocking, prio_lo);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sv->lanes[i].hi, cudaStreamNonBlocking, prio_hi);
        sv->lanes[i].s = sv->lanes[i].lo;
    }
    if (e != cudaSuccess) {
        for (auto& L : sv->lanes) {
            if (L.lo) cudaStreamDestroy(L.lo);
            if (L.hi) cudaStreamDestroy(L.hi);
        }
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
    for (auto& L : sv->lanes) {
        cudaStreamSynchronize(L.lo);
        cudaStreamSynchronize(L.hi);
        cudaStreamDestroy(L.lo);
        cudaStreamDestroy(L.hi);
        if (L.pin) cudaFreeHost(L.pin);
    }
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
        else if (r->n_walkers >= 0x7FFFFFFFull) st = fail(CSAW_ERR_INVALID, "too many walkers");
        else if (r->length == 0xFFFFFFFFu) st = fail(CSAW_ERR_INVALID, "length too large");
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
            for (uint32_t i = 0; st == CSAW_OK && i < rq->n_instances; ++i)
                if (rq->io[i + 1] < rq->io[i]) st = fail(CSAW_ERR_INVALID, "inst_offsets must be non-decreasing");
            for (uint32_t l = 0; st == CSAW_OK && l < r->depth; ++l)
                if (rq->fanout[l] == 0) st = fail(CSAW_ERR_INVALID, "fanout[%u] is 0", l);
            if (st == CSAW_OK && ns && !r->seeds) st = fail(CSAW_ERR_INVALID, "seeds is NULL");
            if (st == CSAW_OK && ns >= 0x7FFFFFFFull) st = fail(CSAW_ERR_INVALID, "too many seeds");
            if (st == CSAW_OK) rq->seeds.assign(r->seeds, r->seeds + ns);
            for (uint64_t j = 0; st == CSAW_OK && j < ns; ++j)
                if (rq->seeds[j] >= sv->g->V) st = fail(CSAW_ERR_INVALID, "seed %llu out of range", (unsigned long long)j);
        }
    } else if (st == CSAW_OK) {
        st = fail(CSAW_ERR_INVALID, "unknown request kind %d", r->kind);
    }
    if (st != CSAW_OK) { delete rq; return st; }
    rq->estimate = estimate_bytes(sv->g, sv->degrees, *rq);
    rq->large = edge_bound(sv->g, sv->degrees, rq) > SMALL_BATCH_EDGES;
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
    sv->cv_work.notify_one();   // one idle slot takes it (and whatever else waits)
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
