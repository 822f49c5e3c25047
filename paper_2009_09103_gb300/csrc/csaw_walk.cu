// csaw_walk.cu -- biased random walks (Sec. II-A), one warp per walker.
//
// A walk step at vertex v with degree d is inverse transform sampling over
// v's neighbour list (Sec. II-B, Eq. 1) with a single draw, so the cumulative
// bias array never has to be stored: the warp streams the biases once to get
// the total T (keeping one running prefix per chunk in shared memory), maps
// the draw to x in [0, T), then rescans only the chunk that holds x with a
// warp scan to find the first neighbour whose inclusive prefix exceeds x.
// Rows of at most 256 neighbours stay in registers and need one pass.
//
// Work distribution: a persistent grid; each warp takes the next walker from
// a global counter and runs all its steps.  The path row is buffered one
// 32-entry block per warp (lane j holds entry 32*blk + j) and written with
// one coalesced store per block.
#include "csaw_internal.cuh"

namespace csaw {

constexpr int WALK_THREADS = 256;
constexpr int WALK_WARPS = WALK_THREADS / 32;
constexpr int ELEMS = 8;                 // neighbours per lane per round
constexpr uint32_t ROUND = 32 * ELEMS;   // neighbours per warp per round
constexpr uint32_t CHUNK_SLOTS = 256;    // chunk prefixes per warp (shared memory)

struct WalkParams {
    const uint64_t* __restrict__ off;
    const uint32_t* __restrict__ col;
    const uint32_t* __restrict__ w;
    const uint32_t* __restrict__ deg;
    uint32_t V;
    const uint32_t* __restrict__ starts;
    uint64_t n;
    uint32_t L;
    uint32_t* __restrict__ path;
    uint32_t k0, k1;
    uint32_t m0, m1, m2;
    unsigned long long* next_walker;
};

struct PrevCtx {
    uint32_t prev;       // previous vertex (node2vec), CSAW_NONE on the first step
    uint64_t pbeg, pend; // its neighbour range
};

// EdgeBias (Eq. 3) of the neighbour at edge index e.
template <int KIND>
__device__ __forceinline__ uint32_t edge_bias(const WalkParams& p, uint64_t e, const PrevCtx& c)
{
    if constexpr (KIND == CSAW_BIAS_UNIFORM) {
        return 1u;
    } else if constexpr (KIND == CSAW_BIAS_EDGE_WEIGHT) {
        return __ldg(p.w + e);
    } else if constexpr (KIND == CSAW_BIAS_NEIGHBOR_DEGREE) {
        return __ldg(p.deg + __ldg(p.col + e));
    } else {
        const uint32_t wt = p.w ? __ldg(p.w + e) : 1u;
        if (c.prev == CSAW_NONE) return wt;
        const uint32_t u = __ldg(p.col + e);
        if (u == c.prev) return wt * p.m0;
        return sorted_contains(p.col, c.pbeg, c.pend, u) ? wt * p.m1 : wt * p.m2;
    }
}

// Biases of one round: lane holds neighbours j = base + 32*u + lane.
template <int KIND>
__device__ __forceinline__ void load_round(const WalkParams& p, uint64_t beg, uint32_t d,
                                           uint32_t base, const PrevCtx& c, int lane,
                                           uint32_t (&b)[ELEMS])
{
#pragma unroll
    for (int u = 0; u < ELEMS; ++u) {
        const uint32_t j = base + 32u * u + lane;
        b[u] = j < d ? edge_bias<KIND>(p, beg + j, c) : 0u;
    }
}

// Find, in one round whose biases are b and whose elements start at prefix
// `before`, the neighbour whose interval holds x.  Returns true and sets
// *idx (round-relative) if the round holds x.
__device__ __forceinline__ bool locate_in_round(const uint32_t (&b)[ELEMS], uint64_t& before,
                                                uint64_t x, int lane, uint32_t* idx)
{
#pragma unroll
    for (int u = 0; u < ELEMS; ++u) {
        const uint64_t incl = warp_inclusive_scan_u64(b[u], lane);
        const uint64_t tile = __shfl_sync(CSAW_FULL_MASK, incl, 31);
        if (before + tile > x) {
            const uint32_t hit = __ballot_sync(CSAW_FULL_MASK, before + incl > x);
            *idx = 32u * u + (__ffs(hit) - 1);
            return true;
        }
        before += tile;
    }
    return false;
}

// One walk step at a vertex with neighbours [beg, beg + d): the inverse
// transform pick for draw r.  Returns false at a dead end (T == 0).
template <int KIND>
__device__ __forceinline__ bool walk_pick(const WalkParams& p, uint64_t beg, uint32_t d,
                                          const PrevCtx& c, uint64_t r, uint64_t* s_chunk,
                                          int lane, uint32_t* idx)
{
    if (d == 0) return false;
    if constexpr (KIND == CSAW_BIAS_UNIFORM) {
        *idx = (uint32_t)scale_draw(r, d);   // b = 1: S[i] = i + 1, so the pick is x itself
        return true;
    }
    if (d <= ROUND) {
        uint32_t b[ELEMS];
        load_round<KIND>(p, beg, d, 0, c, lane, b);
        uint64_t s = 0;
#pragma unroll
        for (int u = 0; u < ELEMS; ++u) s += b[u];
        const uint64_t T = warp_sum_u64(s);
        if (T == 0) return false;
        const uint64_t x = scale_draw(r, T);
        uint64_t before = 0;
        locate_in_round(b, before, x, lane, idx);
        return true;
    }
    // Pass 1: total, with the running prefix stored after every chunk of G rounds.
    const uint32_t nrounds = (d + ROUND - 1) / ROUND;
    const uint32_t G = (nrounds + CHUNK_SLOTS - 1) / CHUNK_SLOTS;
    const uint32_t nchunks = (nrounds + G - 1) / G;
    uint64_t running = 0;
    for (uint32_t ch = 0; ch < nchunks; ++ch) {
        const uint32_t r_end = min(nrounds, (ch + 1) * G);
        for (uint32_t rr = ch * G; rr < r_end; ++rr) {
            uint32_t b[ELEMS];
            load_round<KIND>(p, beg, d, rr * ROUND, c, lane, b);
            uint64_t s = 0;
#pragma unroll
            for (int u = 0; u < ELEMS; ++u) s += b[u];
            running += warp_sum_u64(s);
        }
        if (lane == 0) s_chunk[ch] = running;
    }
    __syncwarp();
    const uint64_t T = running;
    if (T == 0) return false;
    const uint64_t x = scale_draw(r, T);
    // Chunk holding x: the first whose inclusive prefix exceeds x.
    uint32_t ch = 0;
    for (uint32_t base = 0; base < nchunks; base += 32) {
        const uint32_t i = base + lane;
        const uint64_t v = i < nchunks ? s_chunk[i] : ~0ull;
        const uint32_t hit = __ballot_sync(CSAW_FULL_MASK, v > x);
        if (hit) { ch = base + __ffs(hit) - 1; break; }
    }
    uint64_t before = ch > 0 ? s_chunk[ch - 1] : 0;
    __syncwarp();
    // Pass 2: rescan that chunk's rounds.
    const uint32_t r_end = min(nrounds, (ch + 1) * G);
    for (uint32_t rr = ch * G; rr < r_end; ++rr) {
        uint32_t b[ELEMS];
        load_round<KIND>(p, beg, d, rr * ROUND, c, lane, b);
        uint32_t in_round;
        if (locate_in_round(b, before, x, lane, &in_round)) {
            *idx = rr * ROUND + in_round;
            return true;
        }
    }
    *idx = d - 1;   // not reached: x < T lies in some chunk
    return true;
}

template <int KIND>
__global__ void __launch_bounds__(WALK_THREADS) walk_kernel(WalkParams p)
{
    __shared__ uint64_t s_chunk_all[WALK_WARPS][CHUNK_SLOTS];
    const int lane = threadIdx.x & 31;
    uint64_t* s_chunk = s_chunk_all[threadIdx.x >> 5];
    const uint64_t row_len = (uint64_t)p.L + 1;

    while (true) {
        unsigned long long wk = 0;
        if (lane == 0) wk = atomicAdd(p.next_walker, 1ull);
        wk = __shfl_sync(CSAW_FULL_MASK, wk, 0);
        if (wk >= p.n) break;
        uint32_t* row = p.path + wk * row_len;
        uint32_t cur = __ldg(p.starts + wk);
        if (cur >= p.V) {
            for (uint64_t t = lane; t < row_len; t += 32) row[t] = CSAW_NONE;
            continue;
        }
        PrevCtx c;
        c.prev = CSAW_NONE;
        c.pbeg = c.pend = 0;
        uint32_t buf = lane == 0 ? cur : CSAW_NONE;   // entries of the current 32-block
        uint64_t flushed = 0;                         // entries [0, flushed) are in memory
        for (uint32_t s = 0; s < p.L; ++s) {
            const uint64_t beg = __ldg(p.off + cur);
            const uint64_t end = __ldg(p.off + cur + 1);
            const uint32_t d = (uint32_t)(end - beg);
            const uint64_t r = philox_draw(p.k0, p.k1, 0u, cur, s, (uint32_t)wk);
            uint32_t idx;
            if (!walk_pick<KIND>(p, beg, d, c, r, s_chunk, lane, &idx)) break;
            const uint32_t nxt = __ldg(p.col + beg + idx);
            if constexpr (KIND == CSAW_BIAS_NODE2VEC) {
                c.prev = cur;
                c.pbeg = beg;
                c.pend = end;
            }
            cur = nxt;
            const uint64_t t = (uint64_t)s + 1;
            if ((uint32_t)(t & 31) == (uint32_t)lane) buf = cur;
            if ((t & 31) == 31) {
                row[t - 31 + lane] = buf;
                buf = CSAW_NONE;
                flushed = t + 1;
            }
        }
        // Remaining entries: the buffered block, then CSAW_NONE to the end of the row.
        for (uint64_t t = flushed + lane; t < row_len; t += 32)
            row[t] = (t < flushed + 32) ? buf : CSAW_NONE;
    }
}

static csaw_status launch_walk(int kind, const WalkParams& p, int sm_count, cudaStream_t s)
{
    int per_sm = 1;
    cudaError_t e = cudaSuccess;
    switch (kind) {
#define CSAW_WALK_CASE(K)                                                                      \
    case K:                                                                                    \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_kernel<K>, WALK_THREADS, 0); \
        if (e != cudaSuccess) return cuda_fail(e, "occupancy(walk)");                          \
        walk_kernel<K><<<sm_count * (per_sm > 0 ? per_sm : 1), WALK_THREADS, 0, s>>>(p);       \
        break;
        CSAW_WALK_CASE(CSAW_BIAS_UNIFORM)
        CSAW_WALK_CASE(CSAW_BIAS_EDGE_WEIGHT)
        CSAW_WALK_CASE(CSAW_BIAS_NEIGHBOR_DEGREE)
        CSAW_WALK_CASE(CSAW_BIAS_NODE2VEC)
#undef CSAW_WALK_CASE
    default:
        return fail(CSAW_ERR_INVALID, "unknown bias kind %d", kind);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "walk_kernel launch");
    return CSAW_OK;
}

}  // namespace csaw

using namespace csaw;

extern "C" csaw_status csaw_walk(csaw_graph* g, const uint32_t* starts, uint64_t n_walkers,
                                 uint32_t length, const csaw_bias* bias, uint64_t rng_seed,
                                 uint32_t* path, int mem_kind, void* stream)
{
    clear_error();
    if (!g) return fail(CSAW_ERR_INVALID, "graph is NULL");
    int kind;
    CSAW_TRY(check_bias(g, bias, true, &kind));
    if (mem_kind != CSAW_MEM_HOST && mem_kind != CSAW_MEM_DEVICE)
        return fail(CSAW_ERR_INVALID, "bad mem_kind %d", mem_kind);
    if (n_walkers == 0) return CSAW_OK;
    if (!starts || !path) return fail(CSAW_ERR_INVALID, "starts/path is NULL");
    if (n_walkers > 0xFFFFFFFFull) return fail(CSAW_ERR_INVALID, "at most 2^32-1 walkers per call");
    if (length == 0xFFFFFFFFu) return fail(CSAW_ERR_INVALID, "length too large");
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t row_len = (uint64_t)length + 1;
    const size_t path_bytes = sizeof(uint32_t) * row_len * n_walkers;

    const uint32_t* d_starts = starts;
    uint32_t* d_path = path;
    if (mem_kind == CSAW_MEM_HOST) {
        for (uint64_t i = 0; i < n_walkers; ++i)
            if (starts[i] >= g->V)
                return fail(CSAW_ERR_INVALID, "start %llu of walker %llu out of range",
                            (unsigned long long)starts[i], (unsigned long long)i);
        void* a = nullptr;
        void* b = nullptr;
        CSAW_TRY(dalloc(&a, sizeof(uint32_t) * n_walkers, s));
        csaw_status st = dalloc(&b, path_bytes, s);
        if (st != CSAW_OK) { dfree(a, s); return st; }
        d_starts = (const uint32_t*)a;
        d_path = (uint32_t*)b;
        cudaError_t e = cudaMemcpyAsync(a, starts, sizeof(uint32_t) * n_walkers,
                                        cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) { dfree(a, s); dfree(b, s); return cuda_fail(e, "copy starts"); }
    }
    void* counter = nullptr;
    csaw_status st = dalloc(&counter, sizeof(unsigned long long), s);
    if (st == CSAW_OK) {
        cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) st = cuda_fail(e, "memset counter");
    }
    if (st == CSAW_OK) {
        WalkParams p;
        p.off = g->off; p.col = g->col; p.w = g->w; p.deg = g->deg; p.V = g->V;
        p.starts = d_starts; p.n = n_walkers; p.L = length; p.path = d_path;
        p.k0 = (uint32_t)rng_seed; p.k1 = (uint32_t)(rng_seed >> 32);
        p.m0 = bias->n2v_mult[0]; p.m1 = bias->n2v_mult[1]; p.m2 = bias->n2v_mult[2];
        p.next_walker = (unsigned long long*)counter;
        st = launch_walk(kind, p, g->sm_count, s);
    }
    dfree(counter, s);
    if (mem_kind == CSAW_MEM_HOST) {
        if (st == CSAW_OK) {
            cudaError_t e = cudaMemcpyAsync(path, d_path, path_bytes, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = cuda_fail(e, "copy path");
        }
        dfree((void*)d_starts, s);
        dfree(d_path, s);
    }
    return st;
}
