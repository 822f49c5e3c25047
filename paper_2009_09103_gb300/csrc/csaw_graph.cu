// csaw_graph.cu -- errors, allocation, and the device-resident CSR graph.
//
// The graph is the input every selection reads (Sec. II-A; all neighbours of
// a vertex must be present to form its biases, Sec. V-A).  It is copied once
// into HBM and validated there: offsets monotone and ending at E, columns in
// range, rows strictly ascending.  The degree array and the maximum degree and
// weight are derived in the same pass.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "csaw_internal.cuh"

namespace csaw {

static thread_local char g_last_error[512] = "";

csaw_status fail(csaw_status st, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

csaw_status cuda_fail(cudaError_t err, const char* what)
{
    if (err == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(CSAW_ERR_NOMEM, "%s: %s", what, cudaGetErrorString(err));
    }
    return fail(CSAW_ERR_CUDA, "%s: %s", what, cudaGetErrorString(err));
}

void clear_error() { g_last_error[0] = '\0'; }

static thread_local const DevAllocator* t_alloc = nullptr;

const DevAllocator* current_allocator() { return t_alloc; }

AllocScope::AllocScope(const csaw_graph* g) : prev(t_alloc)
{
    t_alloc = (g && g->allocator.alloc) ? &g->allocator : nullptr;
}

AllocScope::~AllocScope() { t_alloc = prev; }

csaw_status alloc_with(const DevAllocator* a, void** p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (a && a->alloc) {
        *p = a->alloc((uint64_t)bytes, (void*)s, a->ctx);
        if (!*p) return fail(CSAW_ERR_NOMEM, "the caller's allocator returned no memory for %zu bytes", bytes);
        return CSAW_OK;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? CSAW_ERR_NOMEM : CSAW_ERR_CUDA,
                    "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    return CSAW_OK;
}

void free_with(const DevAllocator& a, void* p, cudaStream_t s)
{
    if (!p) return;
    if (a.free) a.free(p, (void*)s, a.ctx);
    else cudaFree(p);
}

csaw_status dalloc(void** p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (t_alloc) return alloc_with(t_alloc, p, bytes, s);
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? CSAW_ERR_NOMEM : CSAW_ERR_CUDA,
                    "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    return CSAW_OK;
}

void dfree(void* p, cudaStream_t s)
{
    if (!p) return;
    if (t_alloc) t_alloc->free(p, (void*)s, t_alloc->ctx);
    else cudaFreeAsync(p, s);
}

csaw_status check_bias(const csaw_graph* g, const csaw_bias* bias, bool allow_node2vec, int* kind_out)
{
    if (!bias) return fail(CSAW_ERR_INVALID, "bias is NULL");
    int kind = bias->kind;
    switch (kind) {
    case CSAW_BIAS_UNIFORM:
    case CSAW_BIAS_NEIGHBOR_DEGREE:
        break;
    case CSAW_BIAS_EDGE_WEIGHT:
        if (!g->w) kind = CSAW_BIAS_UNIFORM;   // all weights one: same picks as uniform
        break;
    case CSAW_BIAS_NODE2VEC: {
        if (!allow_node2vec)
            return fail(CSAW_ERR_INVALID, "node2vec bias needs a walk's previous vertex");
        uint64_t m = 0;
        for (int i = 0; i < 3; ++i) m = bias->n2v_mult[i] > m ? bias->n2v_mult[i] : m;
        if ((uint64_t)g->max_weight * m > 0xFFFFFFFFull)
            return fail(CSAW_ERR_OVERFLOW,
                        "node2vec bias max_weight (%u) * max multiplier (%llu) does not fit in 32 bits",
                        g->max_weight, (unsigned long long)m);
        break;
    }
    default:
        return fail(CSAW_ERR_INVALID, "unknown bias kind %d", kind);
    }
    *kind_out = kind;
    return CSAW_OK;
}

// ---------------------------------------------------------------------------
// Validation and derived arrays.  One warp per row; flags collect violations.
enum : uint32_t {
    BAD_OFFSET_ORDER = 1u,
    BAD_COLUMN_RANGE = 2u,
    BAD_ROW_ORDER = 4u,
    BAD_ROW_LENGTH = 8u,
    BAD_ENDS = 16u,
};

__global__ void validate_kernel(const uint64_t* __restrict__ off, const uint32_t* __restrict__ col,
                                const uint32_t* __restrict__ w, uint32_t V, uint64_t E,
                                uint32_t* __restrict__ deg, uint32_t* __restrict__ flags,
                                uint32_t* __restrict__ max_deg, uint32_t* __restrict__ max_w,
                                uint32_t* __restrict__ min_w)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t local_flags = 0, local_maxw = 0, local_maxd = 0, local_minw = 0xFFFFFFFFu;
    if (warp == 0 && lane == 0) {
        if (off[0] != 0 || off[V] != E) local_flags |= BAD_ENDS;
    }
    for (uint64_t v = warp; v < V; v += nwarps) {
        const uint64_t beg = off[v], end = off[v + 1];
        if (end < beg || end > E) {
            local_flags |= BAD_OFFSET_ORDER;
            if (lane == 0) deg[v] = 0;
            continue;
        }
        const uint64_t d = end - beg;
        if (d > 0xFFFFFFFFull) local_flags |= BAD_ROW_LENGTH;
        if (lane == 0) deg[v] = (uint32_t)(d > 0xFFFFFFFFull ? 0xFFFFFFFFull : d);
        if (d > local_maxd) local_maxd = (uint32_t)(d > 0xFFFFFFFFull ? 0xFFFFFFFFull : d);
        for (uint64_t e = beg + lane; e < end; e += 32) {
            const uint32_t c = col[e];
            if (c >= V) local_flags |= BAD_COLUMN_RANGE;
            if (e + 1 < end && col[e + 1] <= c) local_flags |= BAD_ROW_ORDER;
            if (w) {
                local_maxw = max(local_maxw, w[e]);
                local_minw = min(local_minw, w[e]);
            }
        }
    }
    local_flags = __reduce_or_sync(CSAW_FULL_MASK, local_flags);
    local_maxw = __reduce_max_sync(CSAW_FULL_MASK, local_maxw);
    local_maxd = __reduce_max_sync(CSAW_FULL_MASK, local_maxd);
    local_minw = __reduce_min_sync(CSAW_FULL_MASK, local_minw);
    if (lane == 0) {
        if (local_flags) atomicOr(flags, local_flags);
        atomicMax(max_w, local_maxw);
        atomicMax(max_deg, local_maxd);
        atomicMin(min_w, local_minw);
    }
}

// Whether some edge points at a vertex with no neighbours (a zero
// neighbour-degree bias).  Runs after validation has filled deg.
__global__ void zero_target_kernel(const uint32_t* __restrict__ col, const uint32_t* __restrict__ deg,
                                   uint64_t E, uint32_t* __restrict__ flag)
{
    uint32_t found = 0;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (uint64_t)gridDim.x * blockDim.x)
        found |= deg[col[e]] == 0;
    found = __reduce_or_sync(CSAW_FULL_MASK, found);
    if ((threadIdx.x & 31) == 0 && found) atomicOr(flag, 1u);
}

}  // namespace csaw

using namespace csaw;

extern "C" const char* csaw_last_error(void) { return g_last_error; }

extern "C" uint32_t csaw_version(void) { return 10100u; }

extern "C" csaw_status csaw_graph_destroy(csaw_graph* g)
{
    clear_error();
    if (!g) return CSAW_OK;
    for (int k = 0; k < 4; ++k) free_with(g->cdf_alloc[k], g->cdf[k], nullptr);
    cudaFree(g->off);
    cudaFree(g->col);
    cudaFree(g->w);
    cudaFree(g->deg);
    delete g;
    return CSAW_OK;
}

extern "C" csaw_status csaw_graph_create(const uint64_t* row_offsets, uint32_t n_vertices,
                                         const uint32_t* cols, const uint32_t* weights,
                                         uint64_t n_edges, int mem_kind, void* stream,
                                         csaw_graph** out)
{
    clear_error();
    if (!out) return fail(CSAW_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!row_offsets || (n_edges > 0 && !cols))
        return fail(CSAW_ERR_INVALID, "row_offsets/cols is NULL");
    if (n_vertices == 0) return fail(CSAW_ERR_INVALID, "graph has no vertices");
    if (n_vertices == 0xFFFFFFFFu) return fail(CSAW_ERR_INVALID, "vertex id 0xFFFFFFFF is reserved");
    if (mem_kind != CSAW_MEM_HOST && mem_kind != CSAW_MEM_DEVICE)
        return fail(CSAW_ERR_INVALID, "bad mem_kind %d", mem_kind);
    if (mem_kind == CSAW_MEM_HOST) {
        if (row_offsets[0] != 0 || row_offsets[n_vertices] != n_edges)
            return fail(CSAW_ERR_INVALID, "row_offsets must start at 0 and end at n_edges");
    }
    cudaStream_t s = (cudaStream_t)stream;
    csaw_graph* g = new (std::nothrow) csaw_graph();
    if (!g) return fail(CSAW_ERR_NOMEM, "host allocation failed");
    {
        cudaError_t e0 = cudaGetDevice(&g->device);
        if (e0 == cudaSuccess)
            e0 = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device);
        if (e0 != cudaSuccess) {
            delete g;
            return cuda_fail(e0, "device query");
        }
    }
    {
        // Keep freed stream-ordered allocations in the device's pool instead of
        // returning them at every synchronisation: calls reuse their buffers.
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, g->device) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    g->V = n_vertices;
    g->E = n_edges;
    const size_t off_b = sizeof(uint64_t) * ((size_t)n_vertices + 1);
    const size_t col_b = sizeof(uint32_t) * (size_t)n_edges;
    const size_t deg_b = sizeof(uint32_t) * (size_t)n_vertices;
    // Column and weight arrays carry CSAW_EDGE_PAD zeroed entries past the end so
    // that 16-byte vector loads of the last row's final group stay inside them.
    const size_t pad_b = sizeof(uint32_t) * CSAW_EDGE_PAD;
    cudaError_t e = cudaMalloc(&g->off, off_b);
    if (e == cudaSuccess) e = cudaMalloc(&g->col, col_b + pad_b);
    if (e == cudaSuccess && weights) e = cudaMalloc(&g->w, col_b + pad_b);
    if (e == cudaSuccess) e = cudaMalloc(&g->deg, deg_b);
    if (e == cudaSuccess) e = cudaMemsetAsync((char*)g->col + col_b, 0, pad_b, s);
    if (e == cudaSuccess && weights) e = cudaMemsetAsync((char*)g->w + col_b, 0, pad_b, s);
    if (e != cudaSuccess) {
        csaw_graph_destroy(g);
        return cuda_fail(e, "cudaMalloc(graph)");
    }
    g->device_bytes = off_b + col_b + (weights ? col_b : 0) + deg_b;
    const cudaMemcpyKind kind = mem_kind == CSAW_MEM_HOST ? cudaMemcpyHostToDevice
                                                          : cudaMemcpyDeviceToDevice;
    e = cudaMemcpyAsync(g->off, row_offsets, off_b, kind, s);
    if (e == cudaSuccess && col_b) e = cudaMemcpyAsync(g->col, cols, col_b, kind, s);
    if (e == cudaSuccess && weights && col_b) e = cudaMemcpyAsync(g->w, weights, col_b, kind, s);
    uint32_t* d_stat = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d_stat, 8 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_stat, 0, 8 * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_stat + 3, 0xFF, sizeof(uint32_t), s);
    if (e == cudaSuccess) {
        const int threads = 256;
        const uint64_t warps_needed = n_vertices;
        uint64_t blocks = (warps_needed * 32 + threads - 1) / threads;
        const uint64_t cap = (uint64_t)g->sm_count * 16;
        if (blocks > cap) blocks = cap;
        validate_kernel<<<(unsigned)blocks, threads, 0, s>>>(g->off, g->col, g->w, n_vertices, n_edges,
                                                             g->deg, d_stat, d_stat + 1, d_stat + 2,
                                                             d_stat + 3);
        e = cudaGetLastError();
    }
    uint32_t h_flags = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_flags, d_stat, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && h_flags == 0 && n_edges > 0) {
        // columns are known to be in range now
        uint64_t blocks = (n_edges + 255) / 256;
        const uint64_t cap = (uint64_t)g->sm_count * 16;
        if (blocks > cap) blocks = cap;
        zero_target_kernel<<<(unsigned)blocks, 256, 0, s>>>(g->col, g->deg, n_edges, d_stat + 4);
        e = cudaGetLastError();
    }
    uint32_t h_stat[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_stat, d_stat, sizeof(h_stat), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_stat);
    if (e != cudaSuccess) {
        csaw_graph_destroy(g);
        return cuda_fail(e, "graph upload/validation");
    }
    if (h_stat[0]) {
        csaw_graph_destroy(g);
        return fail(CSAW_ERR_INVALID, "invalid CSR (flags 0x%x: 1 offsets, 2 column range, "
                    "4 row order/duplicates, 8 row length, 16 ends)", h_stat[0]);
    }
    g->max_degree = h_stat[1];
    g->max_weight = weights ? h_stat[2] : 1u;
    g->min_weight = (weights && n_edges > 0) ? h_stat[3] : 1u;
    g->zero_degree_target = h_stat[4] != 0;
    *out = g;
    return CSAW_OK;
}

extern "C" csaw_status csaw_graph_get_info(const csaw_graph* g, csaw_graph_info* out)
{
    clear_error();
    if (!g || !out) return fail(CSAW_ERR_INVALID, "NULL argument");
    out->n_vertices = g->V;
    out->n_edges = g->E;
    out->max_degree = g->max_degree;
    out->max_weight = g->max_weight;
    out->device_bytes = g->device_bytes;
    return CSAW_OK;
}

// ---------------------------------------------------------------------------
// Cached cumulative bias arrays (the CTPS of Sec. II-B kept per edge for a
// static bias).  One warp per row in rounds of 512 neighbours: each lane takes
// four aligned groups of four, forms their inclusive sums, and a warp scan of
// the lane totals gives every lane its offset; groups are written as two
// 16-byte stores (partial groups at the row ends element by element).

namespace csaw {

bool cached_cdf_usable(const csaw_graph* g, int kind)
{
    if (kind == CSAW_BIAS_UNIFORM) return true;
    if (kind == CSAW_BIAS_EDGE_WEIGHT) return g->cdf[kind] != nullptr && g->min_weight > 0;
    if (kind == CSAW_BIAS_NEIGHBOR_DEGREE) return g->cdf[kind] != nullptr && !g->zero_degree_target;
    return false;
}

template <int KIND>
__global__ void build_cdf_kernel(const uint64_t* __restrict__ off, const uint32_t* __restrict__ col,
                                 const uint32_t* __restrict__ w, const uint32_t* __restrict__ deg,
                                 uint32_t V, uint64_t* __restrict__ cdf, unsigned long long* next_row)
{
    const int lane = threadIdx.x & 31;
    while (true) {
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(next_row, 1ull);
        v = __shfl_sync(CSAW_FULL_MASK, v, 0);
        if (v >= V) break;
        const uint64_t beg = off[v], end = off[v + 1];
        if (beg == end) continue;
        const uint64_t abeg = beg & ~3ull;
        uint64_t carry = 0;
        for (uint64_t base = abeg; base < end; base += 512) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint64_t g0 = base + 128ull * u + 4ull * lane;
                uint32_t b[4] = {0u, 0u, 0u, 0u};
                if (g0 < end) {
                    if constexpr (KIND == CSAW_BIAS_EDGE_WEIGHT) {
                        const uint4 q = __ldg(reinterpret_cast<const uint4*>(w + g0));
                        b[0] = q.x; b[1] = q.y; b[2] = q.z; b[3] = q.w;
                    } else {
                        const uint4 q = __ldg(reinterpret_cast<const uint4*>(col + g0));
                        b[0] = __ldg(deg + q.x);
                        b[1] = q.y < V ? __ldg(deg + q.y) : 0u;
                        b[2] = q.z < V ? __ldg(deg + q.z) : 0u;
                        b[3] = q.w < V ? __ldg(deg + q.w) : 0u;
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (g0 + j < beg || g0 + j >= end) b[j] = 0u;
                }
                const uint64_t i0 = b[0], i1 = i0 + b[1], i2 = i1 + b[2], i3 = i2 + b[3];
                const uint64_t incl = warp_inclusive_scan_u64(i3, lane);
                const uint64_t off0 = carry + incl - i3;
                if (g0 < end) {
                    const uint64_t e[4] = {off0 + i0, off0 + i1, off0 + i2, off0 + i3};
                    if (g0 >= beg && g0 + 4 <= end) {
                        ulonglong2* dst = reinterpret_cast<ulonglong2*>(cdf + g0);
                        dst[0] = make_ulonglong2(e[0], e[1]);
                        dst[1] = make_ulonglong2(e[2], e[3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (g0 + j >= beg && g0 + j < end) cdf[g0 + j] = e[j];
                    }
                }
                carry += __shfl_sync(CSAW_FULL_MASK, incl, 31);
            }
        }
    }
}

}  // namespace csaw

extern "C" csaw_status csaw_graph_build_cdf(csaw_graph* g, int32_t bias_kind, void* stream)
{
    clear_error();
    if (!g) return fail(CSAW_ERR_INVALID, "graph is NULL");
    if (bias_kind != CSAW_BIAS_EDGE_WEIGHT && bias_kind != CSAW_BIAS_NEIGHBOR_DEGREE)
        return fail(CSAW_ERR_INVALID, "only edge-weight and neighbour-degree biases are static");
    if (bias_kind == CSAW_BIAS_EDGE_WEIGHT && !g->w)
        return fail(CSAW_ERR_INVALID, "the graph has no weights (edge-weight bias is uniform)");
    if (g->cdf[bias_kind]) return CSAW_OK;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t* cdf = nullptr;
    // padded like col/w so that 16-byte stores of a row's last group stay inside
    CSAW_TRY(alloc_with(&g->allocator, (void**)&cdf, sizeof(uint64_t) * (g->E + CSAW_EDGE_PAD), s));
    unsigned long long* ctr = nullptr;
    cudaError_t e = cudaMalloc(&ctr, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
        const unsigned blocks = (unsigned)g->sm_count * 8;
        if (bias_kind == CSAW_BIAS_EDGE_WEIGHT)
            build_cdf_kernel<CSAW_BIAS_EDGE_WEIGHT><<<blocks, 256, 0, s>>>(g->off, g->col, g->w, g->deg, g->V, cdf, ctr);
        else
            build_cdf_kernel<CSAW_BIAS_NEIGHBOR_DEGREE><<<blocks, 256, 0, s>>>(g->off, g->col, g->w, g->deg, g->V, cdf, ctr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(ctr);
    if (e != cudaSuccess) {
        free_with(g->allocator, cdf, s);
        return cuda_fail(e, "build cumulative array");
    }
    g->cdf[bias_kind] = cdf;
    g->cdf_alloc[bias_kind] = g->allocator;
    g->device_bytes += sizeof(uint64_t) * (g->E + CSAW_EDGE_PAD);
    return CSAW_OK;
}

extern "C" csaw_status csaw_graph_set_allocator(csaw_graph* g, csaw_alloc_fn alloc, csaw_free_fn free,
                                                void* ctx)
{
    clear_error();
    if (!g) return fail(CSAW_ERR_INVALID, "graph is NULL");
    if ((alloc == nullptr) != (free == nullptr))
        return fail(CSAW_ERR_INVALID, "give both alloc and free, or neither");
    g->allocator.alloc = alloc;
    g->allocator.free = free;
    g->allocator.ctx = alloc ? ctx : nullptr;
    return CSAW_OK;
}

extern "C" csaw_status csaw_graph_drop_cdf(csaw_graph* g, int32_t bias_kind)
{
    clear_error();
    if (!g) return fail(CSAW_ERR_INVALID, "graph is NULL");
    if (bias_kind < 0 || bias_kind > 3) return fail(CSAW_ERR_INVALID, "bad bias kind");
    if (g->cdf[bias_kind]) {
        cudaDeviceSynchronize();   // no call may be running on the graph; its frees may still be queued
        free_with(g->cdf_alloc[bias_kind], g->cdf[bias_kind], nullptr);
        g->cdf[bias_kind] = nullptr;
        g->device_bytes -= sizeof(uint64_t) * (g->E + CSAW_EDGE_PAD);
    }
    return CSAW_OK;
}
