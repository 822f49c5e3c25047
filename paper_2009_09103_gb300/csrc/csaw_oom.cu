// csaw_oom.cu -- random walks over a graph that stays in host memory
// (out-of-memory sampling, Sec. V-A: graph partitions and workload-aware
// partition scheduling).
//
// The CSR lives in host memory and is cut into vertex ranges whose rows fit a
// device slot of the given budget.  Walkers keep their state (current vertex,
// step) on the device.  Each round counts the active walkers per partition,
// loads the partition with the most of them (the workload-aware schedule of
// Sec. V-A: partitions with more active instances go first), builds its
// edge-weight prefix sums on the device and advances every walker that stands
// in it until the walker leaves the partition, finishes or meets a dead end.
// A walk step draws from the counter {0, vertex, step, walker} exactly as
// csaw_walk does, and picks by the same prefix sums, so the paths equal
// csaw_walk's whatever the partitioning and the order of rounds.
#include <algorithm>
#include <vector>

#include "csaw_internal.cuh"

namespace csaw {

struct OomWalkParams {
    const uint64_t* __restrict__ off;   // slot: rebased offsets of [v0, v1], off[0] = 0
    const uint32_t* __restrict__ col;   // slot: columns of the partition's rows
    const uint64_t* __restrict__ cdf;   // slot: inclusive row prefix sums (null: uniform)
    uint32_t v0, v1;
    uint64_t n;
    uint32_t L;
    PhiloxKeys keys;
    uint32_t* cur;                      // [n] current vertex
    uint32_t* step;                     // [n] steps taken
    uint32_t* __restrict__ path;        // [n][L+1]
};

// One thread per walker: steps while the walker stands in [v0, v1).
__global__ void __launch_bounds__(256) oom_walk_kernel(OomWalkParams p)
{
    const uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= p.n) return;
    uint32_t s = p.step[w];
    uint32_t cur = p.cur[w];
    if (s >= p.L || cur < p.v0 || cur >= p.v1) return;
    uint32_t* row = p.path + w * ((uint64_t)p.L + 1);
    while (s < p.L && cur >= p.v0 && cur < p.v1) {
        const uint64_t beg = __ldg(p.off + (cur - p.v0));
        const uint32_t d = (uint32_t)(__ldg(p.off + (cur - p.v0) + 1) - beg);
        const uint64_t T = p.cdf ? (d ? __ldg(p.cdf + beg + d - 1) : 0ull) : d;
        if (T == 0) {   // dead end: the rest of the row stays CSAW_NONE
            s = p.L;
            break;
        }
        const uint64_t x = scale_draw(philox_draw(p.keys, 0u, cur, s, (uint32_t)w), T);
        uint32_t j;
        if (p.cdf) {
            uint32_t lo = 0, hi = d;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (__ldg(p.cdf + beg + mid) > x) hi = mid; else lo = mid + 1;
            }
            j = lo;
        } else {
            j = (uint32_t)x;   // uniform: S[i] = i + 1
        }
        cur = __ldg(p.col + beg + j);
        ++s;
        row[s] = cur;
    }
    p.cur[w] = cur;
    p.step[w] = s;
}

// Inclusive prefix sums of each row's weights in a loaded partition (warp per row).
__global__ void __launch_bounds__(256) oom_cdf_kernel(const uint64_t* __restrict__ off,
                                                     const uint32_t* __restrict__ w, uint32_t rows,
                                                     uint64_t* __restrict__ cdf)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t r = gw; r < rows; r += nw) {
        const uint64_t beg = off[r], end = off[r + 1];
        uint64_t carry = 0;
        for (uint64_t base = beg; base < end; base += 32) {
            const uint64_t i = base + lane;
            const uint64_t incl = carry + warp_inclusive_scan_u64(i < end ? (uint64_t)__ldg(w + i) : 0ull, lane);
            if (i < end) cdf[i] = incl;
            carry = __shfl_sync(CSAW_FULL_MASK, incl, 31);
        }
    }
}

// Start state: path rows [start, NONE, ...], walkers at their starts.
__global__ void oom_init_kernel(const uint32_t* __restrict__ starts, uint64_t n, uint32_t L, uint32_t V,
                                uint32_t* cur, uint32_t* step, uint32_t* path)
{
    const uint64_t row_len = (uint64_t)L + 1;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * row_len;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t w = t / row_len, k = t % row_len;
        const uint32_t s0 = __ldg(starts + w);
        path[t] = k == 0 ? s0 : CSAW_NONE;
        if (k == 0) {
            cur[w] = s0;
            step[w] = s0 < V ? 0u : L;   // an invalid start never moves
        }
    }
}

// Active walkers per partition (partition bounds in vb[0..np]).
__global__ void oom_count_kernel(const uint32_t* __restrict__ cur, const uint32_t* __restrict__ step, uint64_t n,
                                 uint32_t L, const uint32_t* __restrict__ vb, uint32_t np,
                                 unsigned long long* counts)
{
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n;
         w += (uint64_t)gridDim.x * blockDim.x) {
        if (step[w] >= L) continue;
        const uint32_t v = cur[w];
        uint32_t lo = 0, hi = np;   // last q with vb[q] <= v
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (vb[mid] <= v) lo = mid; else hi = mid;
        }
        atomicAdd(counts + lo, 1ull);
    }
}

__global__ void partition_check_kernel(uint32_t* __restrict__ col, uint32_t* __restrict__ w, uint64_t ne,
                                       uint32_t V, const uint32_t* __restrict__ deg, uint32_t* __restrict__ err)
{
    uint32_t flags = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t c = col[i];
        if (c >= V) {
            flags |= 1u;
            col[i] = 0;
            c = 0;
        }
        if (w && w[i] == 0) {
            flags |= 2u;
            w[i] = 1;
        }
        if (deg && deg[c] == 0) flags |= 4u;
    }
    flags = __reduce_or_sync(CSAW_FULL_MASK, flags);
    if ((threadIdx.x & 31) == 0 && flags) atomicOr(err, flags);
}

bool host_register(void* p, size_t bytes)
{
    if (cudaHostRegister(p, bytes, cudaHostRegisterReadOnly) == cudaSuccess) return true;
    cudaGetLastError();
    if (cudaHostRegister(p, bytes, cudaHostRegisterDefault) == cudaSuccess) return true;
    cudaGetLastError();
    return false;
}

// Columns of a host CSR read in place: err |= 1 where one is not a vertex.
__global__ void direct_check_kernel(const uint32_t* col, uint64_t ne, uint32_t V, uint32_t* err)
{
    uint32_t bad = 0;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (uint64_t)gridDim.x * blockDim.x)
        bad |= col[e] >= V;
    if (__any_sync(CSAW_FULL_MASK, bad) && (threadIdx.x & 31) == 0) atomicOr(err, 1u);
}

// Direct mode of csaw_walk_oom_ex: the GPU reads the host CSR in place
// (coherent access to pageable host memory).  The device holds the walkers,
// the path and, for edge weights, the summaries and vertex records of the
// weights' prefix sums (built from the host weights by the segmented scan);
// every step reads one record, bisects the summaries and then reads one
// 32-byte group of weights and the picked column over the host link.
static csaw_status walk_oom_direct(const uint64_t* off, const uint32_t* cols, const uint32_t* weights,
                                   uint32_t V, uint64_t E, int sm_count, const uint32_t* starts, uint64_t n,
                                   uint32_t length, uint64_t rng_seed, uint32_t* path, cudaStream_t s)
{
    const uint64_t row_len = (uint64_t)length + 1;
    void *d_starts = nullptr, *d_path = nullptr, *d_err = nullptr, *d_sum = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(s);
        for (void* p : {d_starts, d_path, d_err, d_sum}) dfree(p, s);
    };
    csaw_status st = dalloc(&d_starts, sizeof(uint32_t) * n, s);
    if (st == CSAW_OK) st = dalloc(&d_path, sizeof(uint32_t) * n * row_len, s);
    if (st == CSAW_OK) st = dalloc(&d_err, sizeof(uint32_t), s);
    if (st == CSAW_OK && weights) st = dalloc(&d_sum, sizeof(uint64_t) * wsum_layout(E, V).words, s);
    if (st != CSAW_OK) { cleanup(); return st; }
    cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_starts, starts, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "copy starts"); }
    if (E) direct_check_kernel<<<(unsigned)sm_count * 8, 256, 0, s>>>(cols, E, V, (uint32_t*)d_err);
    const CdfView c = wsum_view((const uint64_t*)d_sum, E, V);
    if (weights)
        st = enqueue_cdf_build_raw(off, cols, weights, nullptr, V, E, sm_count, CSAW_BIAS_EDGE_WEIGHT, nullptr,
                                   (uint64_t*)c.s1, (uint64_t*)c.s2, (uint64_t*)c.rec, s);
    uint32_t err = 0;
    e = cudaMemcpyAsync(&err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess && st == CSAW_OK) st = cuda_fail(e, "column check");
    if (st == CSAW_OK && err) st = fail(CSAW_ERR_INVALID, "a column is not a vertex");
    if (st == CSAW_OK)
        st = launch_walk_host(c, off, cols, weights, V, E, sm_count, (const uint32_t*)d_starts, n, length, rng_seed,
                              (uint32_t*)d_path, s);
    if (st == CSAW_OK) {
        e = cudaMemcpyAsync(path, d_path, sizeof(uint32_t) * n * row_len, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "copy path");
    }
    cleanup();
    return st;
}

void launch_partition_check(uint32_t* col, uint32_t* w, uint64_t ne, uint32_t V, const uint32_t* deg,
                            uint32_t* err, cudaStream_t s)
{
    if (ne == 0) return;
    uint64_t blocks = (ne + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    partition_check_kernel<<<(unsigned)blocks, 256, 0, s>>>(col, w, ne, V, deg, err);
}

}  // namespace csaw

using namespace csaw;

extern "C" csaw_status csaw_oom_plan(const uint64_t* row_offsets, uint32_t n_vertices, int weighted,
                                     uint64_t device_budget_bytes, uint32_t* bounds, uint32_t bounds_cap,
                                     uint32_t* n_partitions)
{
    clear_error();
    if (!row_offsets || !n_partitions) return fail(CSAW_ERR_INVALID, "row_offsets/n_partitions is NULL");
    if (n_vertices == 0) return fail(CSAW_ERR_INVALID, "no vertices");
    // a partition [first, v) needs 8 bytes per offset (rows + 1) and, per
    // edge, its column (4) and for edge weight its weight (4) and prefix sum (8)
    const uint64_t per_edge = weighted ? 16 : 4, per_vertex = 8;
    uint32_t np = 0, first = 0, v = 0;
    uint64_t edges = 0;
    if (bounds && bounds_cap > 0) bounds[0] = 0;
    while (v < n_vertices) {
        if (row_offsets[v + 1] < row_offsets[v]) return fail(CSAW_ERR_INVALID, "row_offsets must not decrease");
        const uint64_t d = row_offsets[v + 1] - row_offsets[v];
        const uint64_t need = (edges + d) * per_edge + ((uint64_t)(v - first) + 2) * per_vertex;
        if (need > device_budget_bytes) {
            if (v == first)
                return fail(CSAW_ERR_NOMEM, "the row of vertex %u (%llu edges) exceeds the device budget", v,
                            (unsigned long long)d);
            ++np;
            if (bounds && np < bounds_cap) bounds[np] = v;
            first = v;
            edges = 0;
            continue;
        }
        edges += d;
        ++v;
    }
    ++np;
    if (bounds) {
        if (np + 1 > bounds_cap) return fail(CSAW_ERR_INVALID, "bounds holds %u entries, %u needed", bounds_cap, np + 1);
        bounds[np] = n_vertices;
    }
    *n_partitions = np;
    return CSAW_OK;
}

extern "C" csaw_status csaw_walk_oom_ex(const uint64_t* row_offsets, const uint32_t* cols, const uint32_t* weights,
                                        uint32_t n_vertices, uint64_t n_edges, uint64_t device_budget_bytes,
                                        const uint32_t* starts, uint64_t n_walkers, uint32_t length,
                                        const csaw_bias* bias, uint64_t rng_seed, uint32_t* path,
                                        csaw_oom_stats* stats, void* stream, const csaw_oom_opts* opts)
{
    clear_error();
    if (stats) *stats = csaw_oom_stats{};
    if (!row_offsets || (n_edges && !cols)) return fail(CSAW_ERR_INVALID, "row_offsets/cols is NULL");
    if (!bias) return fail(CSAW_ERR_INVALID, "bias is NULL");
    const int kind = bias->kind;
    if (kind != CSAW_BIAS_UNIFORM && kind != CSAW_BIAS_EDGE_WEIGHT)
        return fail(CSAW_ERR_INVALID, "out-of-memory walks take uniform or edge-weight bias");
    const bool weighted = kind == CSAW_BIAS_EDGE_WEIGHT && weights != nullptr;
    const uint32_t n_slots = opts && opts->slots ? opts->slots : 2;
    if (n_slots > 8) return fail(CSAW_ERR_INVALID, "at most 8 slots");
    if (n_walkers == 0) return CSAW_OK;
    if (!starts || !path) return fail(CSAW_ERR_INVALID, "starts/path is NULL");
    if (n_walkers > 0xFFFFFFFFull) return fail(CSAW_ERR_INVALID, "at most 2^32-1 walkers per call");
    if (length == 0xFFFFFFFFu) return fail(CSAW_ERR_INVALID, "length too large");
    for (uint64_t i = 0; i < n_walkers; ++i)
        if (starts[i] >= n_vertices)
            return fail(CSAW_ERR_INVALID, "start %u of walker %llu out of range", starts[i], (unsigned long long)i);
    if (n_vertices == 0 || row_offsets[0] != 0 || row_offsets[n_vertices] != n_edges)
        return fail(CSAW_ERR_INVALID, "row_offsets must run from 0 to n_edges");
    for (uint32_t v = 0; v < n_vertices; ++v)
        if (row_offsets[v + 1] < row_offsets[v]) return fail(CSAW_ERR_INVALID, "row_offsets must not decrease");
    // Columns are checked on the device as each partition arrives (a column
    // that is not a vertex is replaced, so that no walker leaves every
    // partition, and the call fails).
    cudaStream_t s = (cudaStream_t)stream;

    // Direct mode, where the device reads host memory in place and the
    // summaries and records fit the budget.
    if (opts && opts->direct) {
        int dev = 0, pageable = 0, sm_count = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "device query");
        const uint64_t need = weighted ? sizeof(uint64_t) * wsum_layout(n_edges, n_vertices).words : 0;
        const bool aligned = ((uintptr_t)cols % 16 == 0) && (!weighted || (uintptr_t)weights % 16 == 0);
        if (pageable && aligned && need <= device_budget_bytes * n_slots) {
            if (stats) {
                stats->partitions = 1;
                stats->direct = 1;
            }
            return walk_oom_direct(row_offsets, cols, weighted ? weights : nullptr, n_vertices, n_edges, sm_count,
                                   starts, n_walkers, length, rng_seed, path, s);
        }
    }

    // Partitions: vertex ranges whose slot fits the budget.
    uint32_t np = 0;
    CSAW_TRY(csaw_oom_plan(row_offsets, n_vertices, weighted ? 1 : 0, device_budget_bytes, nullptr, 0, &np));
    std::vector<uint32_t> vb((size_t)np + 1);
    CSAW_TRY(csaw_oom_plan(row_offsets, n_vertices, weighted ? 1 : 0, device_budget_bytes, vb.data(), np + 1, &np));
    uint64_t max_edges = 0, max_rows = 0;
    for (uint32_t q = 0; q < np; ++q) {
        max_edges = std::max(max_edges, row_offsets[vb[q + 1]] - row_offsets[vb[q]]);
        max_rows = std::max<uint64_t>(max_rows, vb[q + 1] - vb[q]);
    }

    // One slot per partition held on the device; the copies of a partition
    // (and its prefix sums) run on their own stream, so the load of the
    // second-busiest partition overlaps the current round.
    struct Slot {
        void *off = nullptr, *col = nullptr, *w = nullptr, *cdf = nullptr;
        std::vector<uint64_t> rebased;   // host staging of its rebased offsets
        int64_t part = -1;
        uint64_t stamp = 0;              // last round that loaded or used it
        cudaEvent_t loaded = nullptr, freed = nullptr;
    };
    std::vector<Slot> slot(n_slots);
    const uint64_t row_len = (uint64_t)length + 1;
    void *d_starts = nullptr, *d_path = nullptr, *d_cur = nullptr, *d_step = nullptr, *d_vb = nullptr;
    void* d_cnt = nullptr;
    void* d_chk = nullptr;   // partition check flags
    cudaStream_t cs = nullptr;
    bool registered_col = false, registered_w = false;
    auto cleanup = [&]() {
        cudaStreamSynchronize(s);
        if (cs) {
            cudaStreamSynchronize(cs);
            cudaStreamDestroy(cs);
        }
        for (void* p : {d_starts, d_path, d_cur, d_step, d_vb, d_cnt, d_chk}) dfree(p, s);
        for (auto& sl : slot) {
            for (void* p : {sl.off, sl.col, sl.w, sl.cdf}) dfree(p, s);
            if (sl.loaded) cudaEventDestroy(sl.loaded);
            if (sl.freed) cudaEventDestroy(sl.freed);
        }
        if (registered_col) cudaHostUnregister((void*)cols);
        if (registered_w) cudaHostUnregister((void*)weights);
    };
    if (opts && opts->pin_host && n_edges) {
        registered_col = host_register((void*)cols, sizeof(uint32_t) * n_edges);
        if (weighted)
            registered_w = host_register((void*)weights, sizeof(uint32_t) * n_edges);
        cudaGetLastError();   // a refused registration leaves ordinary (pageable) copies
    }
    csaw_status st = dalloc(&d_starts, sizeof(uint32_t) * n_walkers, s);
    if (st == CSAW_OK) st = dalloc(&d_path, sizeof(uint32_t) * n_walkers * row_len, s);
    if (st == CSAW_OK) st = dalloc(&d_cur, sizeof(uint32_t) * n_walkers, s);
    if (st == CSAW_OK) st = dalloc(&d_step, sizeof(uint32_t) * n_walkers, s);
    if (st == CSAW_OK) st = dalloc(&d_vb, sizeof(uint32_t) * (np + 1), s);
    if (st == CSAW_OK) st = dalloc(&d_cnt, sizeof(unsigned long long) * np, s);
    if (st == CSAW_OK) st = dalloc(&d_chk, sizeof(uint32_t), s);
    if (st == CSAW_OK) {
        cudaError_t e0 = cudaMemsetAsync(d_chk, 0, sizeof(uint32_t), s);
        if (e0 == cudaSuccess) e0 = cudaStreamSynchronize(s);   // before the copy stream uses it
        if (e0 != cudaSuccess) st = cuda_fail(e0, "memset");
    }
    for (auto& sl : slot) {
        if (st == CSAW_OK) st = dalloc(&sl.off, sizeof(uint64_t) * (max_rows + 1), s);
        if (st == CSAW_OK) st = dalloc(&sl.col, sizeof(uint32_t) * (max_edges ? max_edges : 1), s);
        if (st == CSAW_OK && weighted) st = dalloc(&sl.w, sizeof(uint32_t) * (max_edges ? max_edges : 1), s);
        if (st == CSAW_OK && weighted) st = dalloc(&sl.cdf, sizeof(uint64_t) * (max_edges ? max_edges : 1), s);
        if (st == CSAW_OK) {
            cudaError_t e = cudaEventCreateWithFlags(&sl.loaded, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.freed, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(sl.freed, s);
            if (e != cudaSuccess) st = cuda_fail(e, "cudaEvent");
        }
    }
    if (st == CSAW_OK) {
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamCreate");
    }
    if (st != CSAW_OK) { cleanup(); return st; }
    cudaError_t e = cudaMemcpyAsync(d_starts, starts, sizeof(uint32_t) * n_walkers, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_vb, vb.data(), sizeof(uint32_t) * (np + 1), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "copy starts"); }
    oom_init_kernel<<<1024, 256, 0, s>>>((const uint32_t*)d_starts, n_walkers, length, n_vertices,
                                         (uint32_t*)d_cur, (uint32_t*)d_step, (uint32_t*)d_path);

    OomWalkParams p;
    p.keys = philox_round_keys(rng_seed);
    p.n = n_walkers;
    p.L = length;
    p.cur = (uint32_t*)d_cur;
    p.step = (uint32_t*)d_step;
    p.path = (uint32_t*)d_path;
    std::vector<unsigned long long> counts(np);
    csaw_oom_stats acc{};
    acc.partitions = np;
    uint64_t round = 0;
    // Loads partition q into a slot other than `avoid` (unless it is resident
    // already): an empty slot, else the least recently used one.
    auto load = [&](uint32_t q, int avoid, int* out_slot) -> cudaError_t {
        ++round;
        for (uint32_t k = 0; k < n_slots; ++k)
            if (slot[k].part == (int64_t)q) {
                slot[k].stamp = round;
                *out_slot = (int)k;
                return cudaSuccess;
            }
        int k = -1;
        for (uint32_t j = 0; j < n_slots; ++j) {
            if ((int)j == avoid && n_slots > 1) continue;
            if (k < 0 || slot[j].part < 0 || (slot[k].part >= 0 && slot[j].stamp < slot[k].stamp)) k = (int)j;
            if (slot[j].part < 0) break;
        }
        Slot& sl = slot[k];
        sl.stamp = round;
        const uint32_t v0 = vb[q], v1 = vb[q + 1];
        const uint64_t e0 = row_offsets[v0], ne = row_offsets[v1] - e0;
        cudaError_t ce = cudaStreamWaitEvent(cs, sl.freed, 0);
        if (ce != cudaSuccess) return ce;
        ce = cudaStreamSynchronize(cs);   // the slot's host staging may be rewritten
        if (ce != cudaSuccess) return ce;
        sl.rebased.resize((size_t)(v1 - v0) + 1);
        for (uint32_t v = v0; v <= v1; ++v) sl.rebased[v - v0] = row_offsets[v] - e0;
        ce = cudaMemcpyAsync(sl.off, sl.rebased.data(), sizeof(uint64_t) * sl.rebased.size(),
                             cudaMemcpyHostToDevice, cs);
        if (ce == cudaSuccess && ne)
            ce = cudaMemcpyAsync(sl.col, cols + e0, sizeof(uint32_t) * ne, cudaMemcpyHostToDevice, cs);
        if (ce == cudaSuccess && weighted && ne)
            ce = cudaMemcpyAsync(sl.w, weights + e0, sizeof(uint32_t) * ne, cudaMemcpyHostToDevice, cs);
        if (ce == cudaSuccess) {
            launch_partition_check((uint32_t*)sl.col, nullptr, ne, n_vertices, nullptr, (uint32_t*)d_chk, cs);
            ce = cudaGetLastError();
        }
        if (ce == cudaSuccess && weighted) {
            const uint64_t blocks = std::min<uint64_t>(((uint64_t)(v1 - v0) + 7) / 8, 4096);
            oom_cdf_kernel<<<(unsigned)(blocks ? blocks : 1), 256, 0, cs>>>((const uint64_t*)sl.off,
                                                                         (const uint32_t*)sl.w, v1 - v0,
                                                                         (uint64_t*)sl.cdf);
            ce = cudaGetLastError();
        }
        if (ce == cudaSuccess) ce = cudaEventRecord(sl.loaded, cs);
        if (ce != cudaSuccess) return ce;
        sl.part = q;
        acc.loads += 1;
        acc.bytes_loaded += sizeof(uint64_t) * sl.rebased.size() + ne * (weighted ? 8 : 4);
        *out_slot = k;
        return cudaSuccess;
    };
    const unsigned walk_blocks = (unsigned)((n_walkers + 255) / 256);
    while (true) {
        e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * np, s);
        if (e != cudaSuccess) break;
        oom_count_kernel<<<1024, 256, 0, s>>>((const uint32_t*)d_cur, (const uint32_t*)d_step, n_walkers, length,
                                              (const uint32_t*)d_vb, np, (unsigned long long*)d_cnt);
        e = cudaMemcpyAsync(counts.data(), d_cnt, sizeof(unsigned long long) * np, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        // workload-aware schedule: the partition with the most active walkers,
        // and the next busiest to load while this round runs
        uint32_t q = 0;
        for (uint32_t k = 1; k < np; ++k)
            if (counts[k] > counts[q]) q = k;
        if (counts[q] == 0) break;   // every walker finished
        int q2 = -1;
        for (uint32_t k = 0; k < np; ++k)
            if (k != q && counts[k] && (q2 < 0 || counts[k] > counts[q2])) q2 = (int)k;
        const bool resident = [&] {
            for (auto& sl : slot) if (sl.part == (int64_t)q) return true;
            return false;
        }();
        if (resident) ++acc.reuses;
        int k = -1;
        e = load(q, -1, &k);
        if (e != cudaSuccess) break;
        Slot& sl = slot[k];
        e = cudaStreamWaitEvent(s, sl.loaded, 0);
        if (e != cudaSuccess) break;
        p.off = (const uint64_t*)sl.off;
        p.col = (const uint32_t*)sl.col;
        p.cdf = weighted ? (const uint64_t*)sl.cdf : nullptr;
        p.v0 = vb[q];
        p.v1 = vb[q + 1];
        oom_walk_kernel<<<walk_blocks, 256, 0, s>>>(p);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(sl.freed, s);
        if (e != cudaSuccess) break;
        if (q2 >= 0 && n_slots > 1) {
            int k2 = -1;
            e = load((uint32_t)q2, k, &k2);
            if (e != cudaSuccess) break;
        }
    }
    uint32_t chk = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(path, d_path, sizeof(uint32_t) * n_walkers * row_len, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&chk, d_chk, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    acc.pinned_bytes = (registered_col ? sizeof(uint32_t) * n_edges : 0) + (registered_w ? sizeof(uint32_t) * n_edges : 0);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "out-of-memory walk");
    if (chk & 1u) return fail(CSAW_ERR_INVALID, "a column is not a vertex of the graph");
    if (stats) *stats = acc;
    return CSAW_OK;
}

extern "C" csaw_status csaw_walk_oom(const uint64_t* row_offsets, const uint32_t* cols, const uint32_t* weights,
                                     uint32_t n_vertices, uint64_t n_edges, uint64_t device_budget_bytes,
                                     const uint32_t* starts, uint64_t n_walkers, uint32_t length,
                                     const csaw_bias* bias, uint64_t rng_seed, uint32_t* path,
                                     csaw_oom_stats* stats, void* stream)
{
    const csaw_oom_opts one = {1, 0};
    return csaw_walk_oom_ex(row_offsets, cols, weights, n_vertices, n_edges, device_budget_bytes, starts, n_walkers,
                            length, bias, rng_seed, path, stats, stream, &one);
}
