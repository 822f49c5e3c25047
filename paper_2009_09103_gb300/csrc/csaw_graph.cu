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
#include <mutex>
#include <new>
#include <vector>

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

// The library's own stream-ordered pool, one per device.  Freed blocks stay
// in it (they are not returned at every synchronisation), and a block freed
// on one stream is reused on another only once that free has completed: the
// pool never makes an allocation wait for work queued on another stream, so
// one server slot's buffers never wait for another slot's kernels.
static cudaError_t lib_pool(cudaMemPool_t* out)
{
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if ((size_t)dev < pools.size() && pools[dev]) {
        *out = pools[dev];
        return cudaSuccess;
    }
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    int no = 0;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    if (pools.size() <= (size_t)dev) pools.resize(dev + 1, nullptr);
    pools[dev] = pool;
    *out = pool;
    return cudaSuccess;
}

csaw_status dalloc(void** p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (t_alloc) return alloc_with(t_alloc, p, bytes, s);
    cudaMemPool_t pool;
    cudaError_t e = lib_pool(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, pool, s);
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
// static bias).  The array over all rows is one segmented inclusive scan of
// the edge biases, segments being the rows, so the work is split by edges,
// not rows: tiles of CB_TILE consecutive edges, CB_ITEMS per thread, each
// thread reading its biases as two 16-byte loads.  Three launches, none of
// which waits on another block:
//   cdf_tile_sum_kernel   each tile's segmented total (whether a row starts
//                         in it; the sum since its last row start)
//   cdf_tile_carry_kernel one block: the running row sum entering each tile
//   cdf_tile_scan_kernel  the tile's scan with that carry, written as 16-byte
//                         stores, and the summary entries of its groups.
// Row starts inside a tile come from the row offsets: cdf_tile_rows_kernel
// first records, for every tile, the row holding its first edge (one pass
// over the rows), and a tile sets one shared-memory bit per row start
// between its own row and the next tile's.  The scan also writes the
// summaries s1 (every 8th sum) and s2 (every 64th), and cdf_records_kernel
// the per-vertex records {row start, row end, row total}: a walk step reads
// one record sector, bisects s2, then reads one or two sectors of s1 and of
// the array.

namespace csaw {

bool cached_cdf_usable(const csaw_graph* g, int kind)
{
    if (kind == CSAW_BIAS_UNIFORM) return true;
    if (kind == CSAW_BIAS_EDGE_WEIGHT) return g->cdf[kind] != nullptr && g->min_weight > 0;
    if (kind == CSAW_BIAS_NEIGHBOR_DEGREE) return g->cdf[kind] != nullptr && !g->zero_degree_target;
    return false;
}

bool cdf_kind_positive(const csaw_graph* g, int kind)
{
    if (kind == CSAW_BIAS_EDGE_WEIGHT) return g->w != nullptr && g->min_weight > 0;
    if (kind == CSAW_BIAS_NEIGHBOR_DEGREE) return !g->zero_degree_target;
    return false;
}

uint64_t cdf_words(uint64_t E, uint64_t V) { return cdf_layout(E, V).words; }

constexpr int CB_THREADS = 256;
constexpr int CB_ITEMS = 8;
constexpr uint32_t CB_TILE = CB_THREADS * CB_ITEMS;   // 2048 edges per tile
constexpr int CB_CARRY_THREADS = 1024;

// A segmented sum: f = some row starts in the span, s = the sum of the
// biases after its last row start (the whole span's if none starts in it).
struct SegSum {
    uint32_t f;
    uint64_t s;
};

__device__ __forceinline__ SegSum seg_join(SegSum a, SegSum b)
{
    return SegSum{a.f | b.f, b.f ? b.s : a.s + b.s};
}

__device__ __forceinline__ SegSum warp_inclusive_seg(SegSum x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t yf = __shfl_up_sync(CSAW_FULL_MASK, x.f, o);
        const uint64_t ys = __shfl_up_sync(CSAW_FULL_MASK, x.s, o);
        if (lane >= o) {
            if (!x.f) x.s += ys;
            x.f |= yf;
        }
    }
    return x;
}

// tile_row[t] = the row holding edge t * CB_TILE (each tile start lies in
// exactly one row with edges).
__global__ void cdf_tile_rows_kernel(const uint64_t* __restrict__ off, uint32_t V, uint32_t* __restrict__ tile_row)
{
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t beg = __ldg(off + v), end = __ldg(off + v + 1);
        for (uint64_t t = (beg + CB_TILE - 1) / CB_TILE; t * CB_TILE < end; ++t) tile_row[t] = (uint32_t)v;
    }
}

// Per-thread state of one tile: the thread's biases, its row-start bits and
// its own segmented sums.
template <int KIND>
struct CdfTile {
    uint32_t b[CB_ITEMS];
    uint32_t starts;   // bit j: a row starts at the thread's j-th edge
    uint64_t pb;       // the thread's first edge

    __device__ void load(const uint64_t* __restrict__ off, const uint32_t* __restrict__ col,
                         const uint32_t* __restrict__ w, const uint32_t* __restrict__ deg, uint32_t V,
                         uint64_t E, const uint32_t* __restrict__ tile_row, uint64_t n_tiles, uint64_t t,
                         uint32_t* s_bits)
    {
        const int tid = threadIdx.x;
        const uint64_t p0 = t * CB_TILE;
        const uint32_t span = (uint32_t)((p0 + CB_TILE < E ? p0 + CB_TILE : E) - p0);
        for (int i = tid; i < (int)(CB_TILE / 32); i += CB_THREADS) s_bits[i] = 0;
        // r0 holds the tile's first edge, r1 the next tile's (the last row
        // for the last tile); the rows between start inside (p0, p0 + span]
        // (empty rows share the start of the next row with edges)
        const uint32_t r0 = __ldg(tile_row + t);
        const uint32_t r1 = t + 1 < n_tiles ? __ldg(tile_row + t + 1) : V - 1;
        __syncthreads();
        if (tid == 0 && __ldg(off + r0) == p0) atomicOr(s_bits, 1u);
        for (uint64_t r = (uint64_t)r0 + 1 + tid; r <= r1; r += CB_THREADS) {
            const uint64_t q = __ldg(off + r) - p0;
            if (q < span) atomicOr(s_bits + (q >> 5), 1u << (q & 31));
        }
        pb = p0 + (uint64_t)CB_ITEMS * tid;
        if (pb + CB_ITEMS <= E) {
            if constexpr (KIND == CSAW_BIAS_EDGE_WEIGHT) {
                const uint4 u0 = __ldg(reinterpret_cast<const uint4*>(w + pb));
                const uint4 u1 = __ldg(reinterpret_cast<const uint4*>(w + pb) + 1);
                b[0] = u0.x; b[1] = u0.y; b[2] = u0.z; b[3] = u0.w;
                b[4] = u1.x; b[5] = u1.y; b[6] = u1.z; b[7] = u1.w;
            } else {
                const uint4 u0 = __ldg(reinterpret_cast<const uint4*>(col + pb));
                const uint4 u1 = __ldg(reinterpret_cast<const uint4*>(col + pb) + 1);
                const uint32_t c[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
                for (int j = 0; j < CB_ITEMS; ++j) b[j] = __ldg(deg + c[j]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < CB_ITEMS; ++j) {
                b[j] = 0u;
                if (pb + j < E) {
                    if constexpr (KIND == CSAW_BIAS_EDGE_WEIGHT) b[j] = __ldg(w + pb + j);
                    else b[j] = __ldg(deg + __ldg(col + pb + j));
                }
            }
        }
        __syncthreads();
        starts = (s_bits[(CB_ITEMS * tid) >> 5] >> ((CB_ITEMS * tid) & 31)) & 0xFFu;
    }

    // The thread's own segmented total.
    __device__ SegSum total() const
    {
        uint64_t run = 0;
#pragma unroll
        for (int j = 0; j < CB_ITEMS; ++j) {
            if ((starts >> j) & 1u) run = 0;
            run += b[j];
        }
        return SegSum{starts != 0u, run};
    }
};

// Block-wide exclusive segmented scan of the threads' totals (thread order);
// the tile's total goes to *tile_total (every thread gets it).
__device__ __forceinline__ SegSum block_exclusive_seg(SegSum mine, SegSum* s_warp, SegSum* tile_total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const SegSum incl = warp_inclusive_seg(mine, lane);
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    SegSum before{0u, 0ull};
    for (int k = 0; k < wid; ++k) before = seg_join(before, s_warp[k]);
    SegSum all = before;
    for (int k = wid; k < CB_THREADS / 32; ++k) all = seg_join(all, s_warp[k]);
    *tile_total = all;
    SegSum prev{__shfl_up_sync(CSAW_FULL_MASK, incl.f, 1), __shfl_up_sync(CSAW_FULL_MASK, incl.s, 1)};
    if (lane == 0) prev = SegSum{0u, 0ull};
    return seg_join(before, prev);
}

template <int KIND>
__global__ void __launch_bounds__(CB_THREADS) cdf_tile_sum_kernel(const uint64_t* __restrict__ off,
                                                                   const uint32_t* __restrict__ col,
                                                                   const uint32_t* __restrict__ w,
                                                                   const uint32_t* __restrict__ deg, uint32_t V,
                                                                   uint64_t E, const uint32_t* __restrict__ tile_row,
                                                                   uint64_t n_tiles, uint32_t* __restrict__ tile_f,
                                                                   uint64_t* __restrict__ tile_s)
{
    __shared__ uint32_t s_bits[CB_TILE / 32];
    __shared__ SegSum s_warp[CB_THREADS / 32];
    const uint64_t t = blockIdx.x;
    CdfTile<KIND> tl;
    tl.load(off, col, w, deg, V, E, tile_row, n_tiles, t, s_bits);
    SegSum tot;
    block_exclusive_seg(tl.total(), s_warp, &tot);
    if (threadIdx.x == 0) {
        tile_f[t] = tot.f;
        tile_s[t] = tot.s;
    }
}

// One block.  tile_s becomes the running row sum entering each tile (the
// segmented sum of all earlier tiles; edge 0 always starts a row).
__global__ void __launch_bounds__(CB_CARRY_THREADS) cdf_tile_carry_kernel(const uint32_t* __restrict__ tile_f,
                                                                          uint64_t* __restrict__ tile_s,
                                                                          uint64_t n_tiles)
{
    __shared__ SegSum s_warp[CB_CARRY_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint64_t per = (n_tiles + CB_CARRY_THREADS - 1) / CB_CARRY_THREADS;
    const uint64_t t0 = per * tid < n_tiles ? per * tid : n_tiles;
    const uint64_t t1 = t0 + per < n_tiles ? t0 + per : n_tiles;
    SegSum mine{0u, 0ull};
    for (uint64_t t = t0; t < t1; ++t) mine = seg_join(mine, SegSum{tile_f[t], tile_s[t]});
    const SegSum incl = warp_inclusive_seg(mine, lane);
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    SegSum acc{0u, 0ull};
    for (int k = 0; k < wid; ++k) acc = seg_join(acc, s_warp[k]);
    SegSum prev{__shfl_up_sync(CSAW_FULL_MASK, incl.f, 1), __shfl_up_sync(CSAW_FULL_MASK, incl.s, 1)};
    if (lane == 0) prev = SegSum{0u, 0ull};
    acc = seg_join(acc, prev);
    for (uint64_t t = t0; t < t1; ++t) {
        const SegSum here{tile_f[t], tile_s[t]};
        tile_s[t] = acc.s;
        acc = seg_join(acc, here);
    }
}

template <int KIND>
__global__ void __launch_bounds__(CB_THREADS) cdf_tile_scan_kernel(const uint64_t* __restrict__ off,
                                                                    const uint32_t* __restrict__ col,
                                                                    const uint32_t* __restrict__ w,
                                                                    const uint32_t* __restrict__ deg, uint32_t V,
                                                                    uint64_t E, const uint32_t* __restrict__ tile_row,
                                                                    uint64_t n_tiles, const uint64_t* __restrict__ carry,
                                                                    uint64_t* __restrict__ cdf, uint64_t* __restrict__ s1,
                                                                    uint64_t* __restrict__ s2)
{
    __shared__ uint32_t s_bits[CB_TILE / 32];
    __shared__ SegSum s_warp[CB_THREADS / 32];
    const uint64_t t = blockIdx.x;
    CdfTile<KIND> tl;
    tl.load(off, col, w, deg, V, E, tile_row, n_tiles, t, s_bits);
    SegSum tot;
    const SegSum ex = seg_join(SegSum{0u, __ldg(carry + t)}, block_exclusive_seg(tl.total(), s_warp, &tot));
    uint64_t out[CB_ITEMS];
    uint64_t run = ex.s;
#pragma unroll
    for (int j = 0; j < CB_ITEMS; ++j) {
        if ((tl.starts >> j) & 1u) run = 0;
        run += tl.b[j];
        out[j] = run;
    }
    const uint64_t pb = tl.pb;
    if (pb + CB_ITEMS <= E) {
        if (cdf) {
            ulonglong2* dst = reinterpret_cast<ulonglong2*>(cdf + pb);
#pragma unroll
            for (int j = 0; j < CB_ITEMS / 2; ++j) dst[j] = make_ulonglong2(out[2 * j], out[2 * j + 1]);
        }
        s1[pb >> 3] = out[CB_ITEMS - 1];
        if (((pb >> 3) & 7) == 7) s2[pb >> 6] = out[CB_ITEMS - 1];   // edge 64h + 63
    } else if (cdf) {
#pragma unroll
        for (int j = 0; j < CB_ITEMS; ++j)
            if (pb + j < E) cdf[pb + j] = out[j];
    }
}

// rec[v] = {off[v], off[v+1], row total, 0}, two 16-byte stores per vertex.
// The total is cdf[end - 1], or without a leaf level the last summary entry
// inside the row plus the weights after it (edge weights).
__global__ void cdf_records_kernel(const uint64_t* __restrict__ off, uint32_t V, const uint64_t* __restrict__ cdf,
                                   const uint64_t* __restrict__ s1, const uint32_t* __restrict__ w,
                                   uint64_t* __restrict__ rec)
{
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t beg = off[v], end = off[v + 1];
        uint64_t T = 0;
        if (end > beg && cdf) {
            T = cdf[end - 1];
        } else if (end > beg) {
            const uint64_t gb = ((end - 1) >> 3) << 3;
            T = gb > beg ? s1[(gb >> 3) - 1] : 0ull;
            for (uint64_t q = gb > beg ? gb : beg; q < end; ++q) T += w[q];
        }
        ulonglong2* r = reinterpret_cast<ulonglong2*>(rec + 4 * v);
        r[0] = make_ulonglong2(beg, end);
        r[1] = make_ulonglong2(T, 0ull);
    }
}

csaw_status enqueue_cdf_build_raw(const uint64_t* off, const uint32_t* col, const uint32_t* w, const uint32_t* deg,
                                  uint32_t V, uint64_t E, int sm_count, int kind, uint64_t* leaf, uint64_t* s1,
                                  uint64_t* s2, uint64_t* rec, cudaStream_t s)
{
    uint64_t vb = ((uint64_t)V + 255) / 256;
    if (vb > (uint64_t)sm_count * 8) vb = (uint64_t)sm_count * 8;
    const unsigned vgrid = (unsigned)(vb ? vb : 1);
    if (E == 0) {
        if (V) cdf_records_kernel<<<vgrid, 256, 0, s>>>(off, V, leaf, s1, w, rec);
        const cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? CSAW_OK : cuda_fail(e, "cumulative array launch");
    }
    const uint64_t n_tiles = (E + CB_TILE - 1) / CB_TILE;
    if (n_tiles > 0x7FFFFFFFull) return fail(CSAW_ERR_INVALID, "too many edges for the cumulative array");
    void* tf = nullptr;
    void* ts = nullptr;
    void* tr = nullptr;
    CSAW_TRY(dalloc(&tf, sizeof(uint32_t) * n_tiles, s));
    csaw_status st = dalloc(&ts, sizeof(uint64_t) * n_tiles, s);
    if (st == CSAW_OK) st = dalloc(&tr, sizeof(uint32_t) * n_tiles, s);
    if (st != CSAW_OK) { dfree(tf, s); dfree(ts, s); return st; }
    const unsigned grid = (unsigned)n_tiles;
    uint32_t* tile_row = (uint32_t*)tr;
    cdf_tile_rows_kernel<<<vgrid, 256, 0, s>>>(off, V, tile_row);
    if (kind == CSAW_BIAS_EDGE_WEIGHT) {
        cdf_tile_sum_kernel<CSAW_BIAS_EDGE_WEIGHT><<<grid, CB_THREADS, 0, s>>>(
            off, col, w, deg, V, E, tile_row, n_tiles, (uint32_t*)tf, (uint64_t*)ts);
        cdf_tile_carry_kernel<<<1, CB_CARRY_THREADS, 0, s>>>((const uint32_t*)tf, (uint64_t*)ts, n_tiles);
        cdf_tile_scan_kernel<CSAW_BIAS_EDGE_WEIGHT><<<grid, CB_THREADS, 0, s>>>(
            off, col, w, deg, V, E, tile_row, n_tiles, (const uint64_t*)ts, leaf, s1, s2);
    } else {
        cdf_tile_sum_kernel<CSAW_BIAS_NEIGHBOR_DEGREE><<<grid, CB_THREADS, 0, s>>>(
            off, col, w, deg, V, E, tile_row, n_tiles, (uint32_t*)tf, (uint64_t*)ts);
        cdf_tile_carry_kernel<<<1, CB_CARRY_THREADS, 0, s>>>((const uint32_t*)tf, (uint64_t*)ts, n_tiles);
        cdf_tile_scan_kernel<CSAW_BIAS_NEIGHBOR_DEGREE><<<grid, CB_THREADS, 0, s>>>(
            off, col, w, deg, V, E, tile_row, n_tiles, (const uint64_t*)ts, leaf, s1, s2);
    }
    cdf_records_kernel<<<vgrid, 256, 0, s>>>(off, V, leaf, s1, w, rec);
    cudaError_t e = cudaGetLastError();
    dfree(tf, s);
    dfree(ts, s);
    dfree(tr, s);
    if (e != cudaSuccess) return cuda_fail(e, "cumulative array launch");
    return CSAW_OK;
}

csaw_status enqueue_cdf_build(const csaw_graph* g, int kind, uint64_t* cdf, cudaStream_t s)
{
    const CdfLayout L = cdf_layout(g->E, g->V);
    return enqueue_cdf_build_raw(g->off, g->col, g->w, g->deg, g->V, g->E, g->sm_count, kind, cdf, cdf + L.s1,
                                 cdf + L.s2, cdf + L.rec, s);
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
    // padded like col/w so that a group's 16-byte loads and stores stay
    // inside; the summary follows the padding
    const size_t bytes = sizeof(uint64_t) * cdf_words(g->E, g->V);
    CSAW_TRY(alloc_with(&g->allocator, (void**)&cdf, bytes, s));
    csaw_status st = enqueue_cdf_build(g, bias_kind, cdf, s);
    if (st == CSAW_OK) {
        const cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "build cumulative array");
    }
    if (st != CSAW_OK) {
        cudaStreamSynchronize(s);
        free_with(g->allocator, cdf, s);
        return st;
    }
    g->cdf[bias_kind] = cdf;
    g->cdf_alloc[bias_kind] = g->allocator;
    g->device_bytes += bytes;
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
        g->device_bytes -= sizeof(uint64_t) * cdf_words(g->E, g->V);
    }
    return CSAW_OK;
}
