// csaw_walk_cdf.cu -- random walks over a static bias's cumulative array
// (Sec. II-A, II-B: the CTPS of every row built once, then searched).
#include <atomic>
#include <vector>

#include "csaw_internal.cuh"

namespace csaw {

// ---------------------------------------------------------------------------
// Walks over a cached cumulative array (static biases): one thread per
// walker.  A step reads the vertex's record {row start, row end, row total}
// (one 32-byte sector), maps the draw to x and searches the row's prefix
// sums through their summaries (cdf_search; uniform bias: the pick is x),
// so its cost is a few dependent loads instead of a stream over the row;
// 32 walkers per warp keep many searches in flight.  The picks are those of
// the streaming kernel: the same prefix sums and the same draws.
//
// Path stores: a warp's 32 walkers (consecutive rows) stage their next 16
// path entries in a shared-memory tile, one tile row per walker; when the
// tile is full (or the walk ends) the warp writes it out two walkers at a
// time, each walker's entries as 64 consecutive bytes of its row.  Stores
// from one thread per walker would put 32 different rows behind every warp
// store, each sector written a few bytes at a time.
//
// L2 residency: the records and summaries (about 9 bytes per edge / 8 + 32
// per vertex) are what walkers at the same hubs re-read; the array's own
// sectors, the picked columns and the path rows are touched once.  Those are
// read and written evict-first (ld/st .cs) so that they pass through L2
// without pushing the summaries out.
constexpr int WC_THREADS = 256;
constexpr int WC_WARPS = WC_THREADS / 32;
constexpr int WC_TILE = 16;                  // path entries staged per walker

// How a step finds its pick: uniform (x itself), the array's leaf level, or
// the summaries and the weights (w_search, no leaf level).
constexpr int WC_UNIFORM = 0, WC_LEAF = 1, WC_WEIGHTS = 2;

struct WalkCdfParams {
    const uint64_t* __restrict__ off;
    const uint32_t* __restrict__ col;
    const uint32_t* __restrict__ w;      // weights (WC_WEIGHTS)
    uint64_t E;
    CdfView c;                           // the cumulative array (cdf null for uniform bias)
    uint32_t V;
    const uint32_t* __restrict__ starts;
    uint64_t n;
    uint32_t L;
    uint32_t* __restrict__ path;
    uint32_t w0;                         // the call's index of walker 0 of this launch (its draws)
    PhiloxKeys keys;
    WalkSegments seg;                    // batched kernel: several requests in one launch
};

// Writes the staged entries t in [t0, t_end) of the warp's walkers base ..
// base + 31 (those below n): per iteration, lanes 0-15 store 16 consecutive
// entries of one walker's row and lanes 16-31 those of the next walker.
__device__ __forceinline__ void walk_tile_flush(const WalkCdfParams& p, uint32_t (*tile)[WC_TILE + 1],
                                                uint64_t base, uint64_t row_len, uint64_t t0, uint64_t t_end,
                                                int lane)
{
    __syncwarp();
    const int half = lane >> 4, c = lane & 15;
    const uint64_t t = t0 + (uint64_t)c;
    uint64_t wk = base + (uint64_t)half;
    uint32_t* out = p.path + wk * row_len + t;
    const uint64_t step = 2 * row_len;
#pragma unroll 2
    for (int i = half; i < 32; i += 2) {
        if (wk < p.n && t < t_end) __stcs(out, tile[i][c]);
        wk += 2;
        out += step;
    }
    __syncwarp();
}

// The same for a batch, where each walker has its own row start (row0,
// relative to path) and row length (rl, 0 for lanes without a walker).
__device__ __forceinline__ void walk_tile_flush_rows(const WalkCdfParams& p, uint32_t (*tile)[WC_TILE + 1],
                                                     uint64_t row0, uint64_t rl, uint64_t t0, int lane)
{
    __syncwarp();
    const int half = lane >> 4, c = lane & 15;
    const uint64_t t = t0 + (uint64_t)c;
#pragma unroll 2
    for (int i0 = 0; i0 < 32; i0 += 2) {
        const int i = i0 + half;
        const uint64_t r0 = __shfl_sync(CSAW_FULL_MASK, row0, i);
        const uint64_t n = __shfl_sync(CSAW_FULL_MASK, rl, i);
        if (t < n) p.path[r0 + t] = tile[i][c];
    }
    __syncwarp();
}

// Loads of the CSR arrays: read-only cache for graph arrays, plain loads for
// arrays in host memory (HOST: read in place over the host link).
template <bool HOST, class T>
__device__ __forceinline__ T ld_graph(const T* p)
{
    if constexpr (HOST) return *p;
    else return __ldg(p);
}

// HOST: off, col and w are host arrays (unpadded), read in place.
template <int MODE, bool BATCH = false, bool HOST = false>
__global__ void __launch_bounds__(WC_THREADS, 6) walk_cached_kernel(WalkCdfParams p)
{
    __shared__ uint32_t s_tile[WC_WARPS][32][WC_TILE + 1];   // +1: conflict-free column writes
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t (*tile)[WC_TILE + 1] = s_tile[wid];
    const uint64_t row_len = (uint64_t)p.L + 1;
    const uint64_t n_warps = (uint64_t)gridDim.x * WC_WARPS;
    for (uint64_t base = ((uint64_t)blockIdx.x * WC_WARPS + wid) * 32; base < p.n; base += n_warps * 32) {
        const uint64_t wk = base + (uint64_t)lane;
        // batch: this lane's request (key, index, length) and row; the warp
        // runs to the longest length among its lanes
        WalkerSlot ws{};
        uint32_t L = p.L;
        uint64_t rl = 0;
        if constexpr (BATCH) {
            if (wk < p.n) {
                ws = walker_slot(p.seg, wk);
                rl = (uint64_t)ws.L + 1;
            }
            L = __reduce_max_sync(CSAW_FULL_MASK, ws.L);
        }
        // alive: still walking; cur = CSAW_NONE once stopped (or never started)
        uint32_t cur = wk < p.n ? __ldg(p.starts + wk) : CSAW_NONE;
        if (cur >= p.V) cur = CSAW_NONE;
        bool alive = cur != CSAW_NONE;
        tile[lane][0] = cur;
        uint64_t t0 = 0;                   // path position of tile column 0
        for (uint32_t s = 0; s < L; ++s) {
            if constexpr (BATCH) alive = alive && s < ws.L;
            if (alive) {
                // the row: offsets (uniform) or the vertex's record {start, end, total}
                uint64_t beg, end, T = 0;
                if constexpr (MODE == WC_UNIFORM) {
                    beg = ld_graph<HOST>(p.off + cur);
                    end = ld_graph<HOST>(p.off + cur + 1);
                } else {
                    const ulonglong2* rc = reinterpret_cast<const ulonglong2*>(p.c.rec + 4ull * cur);
                    const ulonglong2 r0 = __ldg(rc), r1 = __ldg(rc + 1);
                    beg = r0.x;
                    end = r0.y;
                    T = r1.x;
                }
                bool stop = beg == end;
                uint64_t i = 0;
                if (!stop) {
                    uint64_t r;
                    if constexpr (BATCH) r = philox_draw(ws.k0, ws.k1, 0u, cur, s, ws.id);
                    else r = philox_draw(p.keys, 0u, cur, s, p.w0 + (uint32_t)wk);
                    if constexpr (MODE == WC_UNIFORM) {
                        i = scale_draw(r, end - beg);
                    } else {
                        stop = T == 0;
                        if (!stop) {
                            const uint64_t x = scale_draw(r, T);
                            if constexpr (MODE == WC_LEAF) i = cdf_search<true>(p.c, beg, end, x) - beg;
                            else i = w_search<!HOST>(p.c, p.w, p.E, beg, end, x) - beg;
                        }
                    }
                }
                if (stop) { alive = false; cur = CSAW_NONE; }
                else if constexpr (HOST) cur = p.col[beg + i];
                else cur = __ldcs(p.col + beg + i);
            }
            const uint64_t t = (uint64_t)s + 1;      // path position of this step's vertex
            tile[lane][t - t0] = cur;
            if (t - t0 == WC_TILE - 1 || t == L) {
                if constexpr (BATCH) walk_tile_flush_rows(p, tile, ws.row0, rl, t0, lane);
                else walk_tile_flush(p, tile, base, row_len, t0, t + 1, lane);
                t0 = t + 1;
            }
        }
        if (L == 0) {
            if constexpr (BATCH) walk_tile_flush_rows(p, tile, ws.row0, rl, 0, lane);
            else walk_tile_flush(p, tile, base, row_len, 0, 1, lane);
        }
    }
}

// Resident blocks per SM of one instantiation (queried once).
template <int MODE, bool BATCH, bool HOST>
static csaw_status walk_cached_occupancy(int* per_sm_out)
{
    static std::atomic<int> cached{0};
    int per_sm = cached.load(std::memory_order_acquire);
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_cached_kernel<MODE, BATCH, HOST>,
                                                                      WC_THREADS, 0);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy(walk_cached)");
        if (per_sm < 1) per_sm = 1;
        cached.store(per_sm, std::memory_order_release);
    }
    *per_sm_out = per_sm;
    return CSAW_OK;
}

template <int MODE, bool BATCH, bool HOST = false>
static csaw_status launch_walk_cached_k(const WalkCdfParams& p, int sm_count, cudaStream_t s)
{
    int per_sm = 0;
    CSAW_TRY((walk_cached_occupancy<MODE, BATCH, HOST>(&per_sm)));
    uint64_t blocks = (p.n + WC_THREADS - 1) / WC_THREADS;
    uint64_t cap = (uint64_t)sm_count * per_sm;
    if (BATCH && p.seg.warp_budget) {
        // each warp walks at most warp_budget groups of 32 walkers
        const uint64_t per_block = (uint64_t)WC_THREADS * p.seg.warp_budget;
        cap = (p.n + per_block - 1) / per_block;
    }
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    walk_cached_kernel<MODE, BATCH, HOST><<<(unsigned)blocks, WC_THREADS, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "walk_cached_kernel launch");
    return CSAW_OK;
}

csaw_status launch_walk_cached(const csaw_graph* g, int kind, const uint64_t* cdf, bool leaf,
                               const uint32_t* starts, uint64_t w0, uint64_t n, uint32_t length, uint64_t rng_seed,
                               uint32_t* path, cudaStream_t s)
{
    WalkCdfParams p;
    p.off = g->off; p.col = g->col; p.w = g->w; p.E = g->E;
    const uint64_t* base = kind == CSAW_BIAS_UNIFORM ? nullptr : cdf;
    p.c = leaf ? cdf_view(base, g->E, g->V) : wsum_view(base, g->E, g->V);
    p.V = g->V; p.starts = starts; p.n = n; p.L = length; p.path = path;
    p.w0 = (uint32_t)w0;
    p.keys = philox_round_keys(rng_seed);
    p.seg = WalkSegments{};
    if (kind == CSAW_BIAS_UNIFORM) return launch_walk_cached_k<WC_UNIFORM, false>(p, g->sm_count, s);
    if (!leaf) return launch_walk_cached_k<WC_WEIGHTS, false>(p, g->sm_count, s);
    return launch_walk_cached_k<WC_LEAF, false>(p, g->sm_count, s);
}

csaw_status launch_walk_host(const CdfView& c, const uint64_t* off, const uint32_t* col, const uint32_t* w,
                             uint32_t V, uint64_t E, int sm_count, const uint32_t* starts, uint64_t n,
                             uint32_t length, uint64_t rng_seed, uint32_t* path, cudaStream_t s)
{
    WalkCdfParams p;
    p.off = off; p.col = col; p.w = w; p.E = E;
    p.c = c;
    p.V = V; p.starts = starts; p.n = n; p.L = length; p.path = path;
    p.w0 = 0;
    p.keys = philox_round_keys(rng_seed);
    p.seg = WalkSegments{};
    if (!w) return launch_walk_cached_k<WC_UNIFORM, false, true>(p, sm_count, s);
    return launch_walk_cached_k<WC_WEIGHTS, false, true>(p, sm_count, s);
}

// With host outputs the walkers run in chunks of whole resident waves (the
// walkers the persistent grid holds at once: a thread walks one walker's
// whole path, so a launch takes as many path-lengths as it has waves, the
// last one partial), at most WC_MAX_CHUNKS of them: each chunk's rows are
// copied out while the next chunk walks, and only the last, partial wave's
// copy is left after the walk.
constexpr uint64_t WC_MAX_CHUNKS = 64;

csaw_status walk_cached_to_host(const csaw_graph* g, int kind, const uint64_t* cdf, bool leaf,
                                const uint32_t* h_starts, const uint32_t* d_starts, uint64_t n, uint32_t length,
                                uint64_t rng_seed, uint32_t* d_path, uint32_t* h_path, cudaStream_t s,
                                cudaEvent_t walked)
{
    const uint64_t row_len = (uint64_t)length + 1;
    int per_sm = 0;
    if (kind == CSAW_BIAS_UNIFORM) CSAW_TRY((walk_cached_occupancy<WC_UNIFORM, false, false>(&per_sm)));
    else if (!leaf) CSAW_TRY((walk_cached_occupancy<WC_WEIGHTS, false, false>(&per_sm)));
    else CSAW_TRY((walk_cached_occupancy<WC_LEAF, false, false>(&per_sm)));
    const uint64_t wave = (uint64_t)g->sm_count * (uint64_t)per_sm * WC_THREADS;
    const uint64_t waves = (n + wave - 1) / wave;
    const uint64_t per_chunk = (waves + WC_MAX_CHUNKS - 1) / WC_MAX_CHUNKS;
    const uint64_t chunk = wave * per_chunk;
    const uint64_t k = (n + chunk - 1) / chunk;
    cudaStream_t cs = nullptr;
    std::vector<cudaEvent_t> ev(k > 1 ? k : 0, nullptr);
    csaw_status st = CSAW_OK;
    cudaError_t e = cudaSuccess;
    if (k > 1) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (uint64_t c = 0; e == cudaSuccess && c < ev.size(); ++c) e = cudaEventCreateWithFlags(&ev[c], cudaEventDisableTiming);
    if (e != cudaSuccess) st = cuda_fail(e, "copy stream");
    // every chunk's walk first (the copies of pageable memory block the host)
    for (uint64_t c = 0, w0 = 0; st == CSAW_OK && w0 < n; w0 += chunk, ++c) {
        const uint64_t m = n - w0 < chunk ? n - w0 : chunk;
        st = launch_walk_cached(g, kind, cdf, leaf, d_starts + w0, w0, m, length, rng_seed, d_path + w0 * row_len, s);
        if (st == CSAW_OK && k > 1) {
            e = cudaEventRecord(ev[c], s);
            if (e != cudaSuccess) st = cuda_fail(e, "chunk event");
        }
    }
    if (st == CSAW_OK && walked) {
        e = cudaEventRecord(walked, s);
        if (e != cudaSuccess) st = cuda_fail(e, "walk event");
    }
    // the host starts are checked while the walks run
    for (uint64_t i = 0; st == CSAW_OK && i < n; ++i)
        if (h_starts[i] >= g->V)
            st = fail(CSAW_ERR_INVALID, "start %llu of walker %llu out of range", (unsigned long long)h_starts[i],
                      (unsigned long long)i);
    // then each chunk's rows, on the copy stream once the chunk is done
    for (uint64_t c = 0, w0 = 0; st == CSAW_OK && w0 < n; w0 += chunk, ++c) {
        const uint64_t m = n - w0 < chunk ? n - w0 : chunk;
        cudaStream_t q = k > 1 ? cs : s;
        if (k > 1) e = cudaStreamWaitEvent(cs, ev[c], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_path + w0 * row_len, d_path + w0 * row_len, sizeof(uint32_t) * m * row_len,
                                cudaMemcpyDeviceToHost, q);
        if (e != cudaSuccess) st = cuda_fail(e, "copy path");
    }
    if (k > 1) {
        e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess && st == CSAW_OK) st = cuda_fail(e, "copy path");
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess && st == CSAW_OK) st = cuda_fail(e, "walk");
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (cs) cudaStreamDestroy(cs);
    return st;
}

csaw_status walk_batch_cached(const csaw_graph* g, int kind, const uint32_t* d_starts, uint64_t n,
                              const WalkSegments& seg, uint32_t max_len, uint32_t* d_path, cudaStream_t s)
{
    WalkCdfParams p;
    p.off = g->off; p.col = g->col; p.w = g->w; p.E = g->E;
    p.c = cdf_view(kind == CSAW_BIAS_UNIFORM ? nullptr : g->cdf[kind], g->E, g->V);
    p.V = g->V; p.starts = d_starts; p.n = n; p.L = max_len; p.path = d_path;
    p.w0 = 0;
    p.keys = philox_round_keys(0);
    p.seg = seg;
    return kind == CSAW_BIAS_UNIFORM ? launch_walk_cached_k<WC_UNIFORM, true>(p, g->sm_count, s)
                                     : launch_walk_cached_k<WC_LEAF, true>(p, g->sm_count, s);
}

}  // namespace csaw
