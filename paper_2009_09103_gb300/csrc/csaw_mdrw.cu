// csaw_mdrw.cu -- multi-dimensional random walk (frontier sampling, Sec. II-A),
// the sampler of the case study of Sec. III-D (Figs. 3-4): VertexBias = degree
// picks one slot of an instance's pool (Eq. 2), EdgeBias = 1 picks one
// neighbour of its vertex, and Update puts that neighbour in the slot (Eq. 4).
//
// One warp per instance, persistent over instances (global counter).  A step
// is inverse transform sampling over the pool in slot order in two levels: the
// warp scans the degree sums of the pool's 32-slot blocks (lane l holds a
// contiguous run of blocks) to find the block holding the draw, then scans
// that block's 32 degrees to find the slot.  The neighbour pick with EdgeBias
// = 1 is the draw itself (S[t] = t + 1).  Then the slot takes the new vertex
// and its degree, and the block its new sum.  A pool of at most
// MDRW_SMALL_POOL slots keeps its block sums in registers (two per lane) and
// its degrees in shared memory, so a step touches global memory only for the
// picked block's vertex ids and the graph; larger pools keep all three in a
// global scratch row.  Sampled edges are buffered one 32-step block per warp
// and written with coalesced stores.
#include <atomic>

#include "csaw_internal.cuh"

namespace csaw {

constexpr int MDRW_THREADS = 128;
constexpr uint32_t MDRW_SMALL_POOL = 2048;   // 64 blocks: two block sums per lane

struct MdrwParams {
    const uint64_t* __restrict__ off;
    const uint32_t* __restrict__ col;
    const uint32_t* __restrict__ deg;
    uint32_t V;
    const uint32_t* __restrict__ pools;   // [n][m] initial pools
    uint64_t n;
    uint32_t m;          // pool size
    uint32_t steps;
    uint32_t nblk;       // 32-slot blocks per pool
    uint32_t per_lane;   // blocks per lane in the top-level scan (large pools)
    uint32_t* ids;       // [n][m] scratch: the pool's vertices
    uint32_t* dg;        // [n][m] scratch: their degrees (large pools)
    uint64_t* bs;        // [n][nblk] scratch: degree sum of each block (large pools)
    PhiloxKeys keys;
    uint32_t* __restrict__ src;   // [n][steps]
    uint32_t* __restrict__ dst;
    unsigned long long* next;
};

template <bool SMALL>
__global__ void __launch_bounds__(MDRW_THREADS) mdrw_kernel(MdrwParams p)
{
    __shared__ uint32_t s_dg_all[SMALL ? MDRW_THREADS / 32 : 1][SMALL ? MDRW_SMALL_POOL : 1];
    const int lane = threadIdx.x & 31;
    uint32_t* s_dg = s_dg_all[SMALL ? threadIdx.x >> 5 : 0];
    while (true) {
        unsigned long long wk = 0;
        if (lane == 0) wk = atomicAdd(p.next, 1ull);
        wk = __shfl_sync(CSAW_FULL_MASK, wk, 0);
        if (wk >= p.n) break;
        const uint32_t inst = (uint32_t)wk;
        uint32_t* ids = p.ids + wk * p.m;
        uint32_t* dg = SMALL ? s_dg : p.dg + wk * p.m;
        uint64_t* bs = SMALL ? nullptr : p.bs + wk * p.nblk;
        uint64_t r0 = 0, r1 = 0;   // small pools: sums of blocks 2*lane and 2*lane + 1
        // the pool, its degrees (VertexBias) and the block sums
        for (uint32_t b = 0; b < p.nblk; ++b) {
            const uint32_t j = b * 32u + (uint32_t)lane;
            uint32_t dv = 0;
            if (j < p.m) {
                const uint32_t v = __ldg(p.pools + wk * p.m + j);
                dv = v < p.V ? __ldg(p.deg + v) : 0u;
                ids[j] = v;
                dg[j] = dv;
            }
            const uint64_t sum = warp_sum_u64(dv);
            if constexpr (SMALL) {
                if (b == 2u * lane) r0 = sum;
                if (b == 2u * lane + 1u) r1 = sum;
            } else if (lane == 0) {
                bs[b] = sum;
            }
        }
        __syncwarp();
        uint32_t* srow = p.src + wk * p.steps;
        uint32_t* drow = p.dst + wk * p.steps;
        uint32_t bsrc = CSAW_NONE, bdst = CSAW_NONE;   // step 32*blk + lane of the current block
        uint64_t flushed = 0;                          // steps [0, flushed) are in memory
        // the pool draw depends on the step alone: the next one is computed
        // while this step waits for the graph
        uint64_t r_pool = philox_draw(p.keys, 0u, CSAW_NONE, 0u, inst);
        for (uint32_t s = 0; s < p.steps; ++s) {
            // top level: this lane's run of blocks
            const uint32_t b0 = (uint32_t)lane * (SMALL ? 2u : p.per_lane);
            uint64_t tl = 0;
            if constexpr (SMALL) {
                tl = r0 + r1;
            } else {
                for (uint32_t k = 0; k < p.per_lane; ++k)
                    if (b0 + k < p.nblk) tl += bs[b0 + k];
            }
            const uint64_t incl = warp_inclusive_scan_u64(tl, lane);
            const uint64_t T = __shfl_sync(CSAW_FULL_MASK, incl, 31);
            if (T == 0) break;   // no vertex of the pool has an edge
            const uint64_t x = scale_draw(r_pool, T);
            const int L = __ffs(__ballot_sync(CSAW_FULL_MASK, incl > x)) - 1;
            uint32_t B = 0;
            uint64_t before = 0;
            if (lane == L) {
                uint64_t acc = incl - tl;
                if constexpr (SMALL) {
                    if (acc + r0 > x) {
                        B = b0;
                    } else {
                        B = b0 + 1u;
                        acc += r0;
                    }
                } else {
                    for (uint32_t k = 0; k < p.per_lane; ++k) {
                        const uint64_t nb = acc + (b0 + k < p.nblk ? bs[b0 + k] : 0ull);
                        if (nb > x) { B = b0 + k; break; }
                        acc = nb;
                    }
                }
                before = acc;
            }
            B = __shfl_sync(CSAW_FULL_MASK, B, L);
            before = __shfl_sync(CSAW_FULL_MASK, before, L);
            // the slot inside block B: first whose inclusive prefix exceeds x
            const uint32_t j = B * 32u + (uint32_t)lane;
            const uint32_t dj = j < p.m ? dg[j] : 0u;
            const uint32_t vj = j < p.m ? ids[j] : 0u;
            const uint64_t inc2 = before + warp_inclusive_scan_u64(dj, lane);
            const int L2 = __ffs(__ballot_sync(CSAW_FULL_MASK, inc2 > x)) - 1;
            const uint32_t v = __shfl_sync(CSAW_FULL_MASK, vj, L2);
            const uint32_t dv = __shfl_sync(CSAW_FULL_MASK, dj, L2);
            // EdgeBias = 1: the neighbour is the draw itself
            const uint32_t t = (uint32_t)scale_draw(philox_draw(p.keys, 0u, v, s, inst), dv);
            const uint32_t u = __ldg(p.col + __ldg(p.off + v) + t);
            r_pool = philox_draw(p.keys, 0u, CSAW_NONE, s + 1u, inst);
            const uint32_t du = __ldg(p.deg + u);
            __syncwarp();   // every lane has read this step's pool
            if constexpr (SMALL) {
                if ((uint32_t)lane == (B >> 1)) {
                    if (B & 1u) r1 = r1 - dv + du;
                    else r0 = r0 - dv + du;
                }
            }
            if (lane == 0) {
                const uint32_t slot = B * 32u + (uint32_t)L2;
                ids[slot] = u;
                dg[slot] = du;
                if constexpr (!SMALL) bs[B] = bs[B] - dv + du;
            }
            __syncwarp();   // the update is visible to the next step
            if ((s & 31u) == (uint32_t)lane) { bsrc = v; bdst = u; }
            if ((s & 31u) == 31u) {
                srow[s - 31u + lane] = bsrc;
                drow[s - 31u + lane] = bdst;
                bsrc = bdst = CSAW_NONE;
                flushed = (uint64_t)s + 1;
            }
        }
        // the buffered block, then CSAW_NONE to the end of the rows
        for (uint64_t t = flushed + lane; t < p.steps; t += 32) {
            const bool in_block = t < flushed + 32;
            srow[t] = in_block ? bsrc : CSAW_NONE;
            drow[t] = in_block ? bdst : CSAW_NONE;
        }
        __syncwarp();   // this instance's reads of the shared degrees are done
    }
}

template <bool SMALL>
static csaw_status launch_mdrw(const MdrwParams& p, int sm_count, cudaStream_t s)
{
    // resident blocks per SM, looked up once (calls may come from several threads)
    static std::atomic<int> cached{0};
    int per_sm = cached.load(std::memory_order_acquire);
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mdrw_kernel<SMALL>,
                                                                      MDRW_THREADS, 0);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy(mdrw)");
        if (per_sm < 1) per_sm = 1;
        cached.store(per_sm, std::memory_order_release);
    }
    uint64_t blocks = (p.n + MDRW_THREADS / 32 - 1) / (MDRW_THREADS / 32);
    const uint64_t cap = (uint64_t)sm_count * per_sm;
    if (blocks > cap) blocks = cap;
    mdrw_kernel<SMALL><<<(unsigned)blocks, MDRW_THREADS, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mdrw_kernel launch");
    return CSAW_OK;
}

}  // namespace csaw

using namespace csaw;

extern "C" csaw_status csaw_mdrw(csaw_graph* g, const uint32_t* pools, uint64_t n_instances,
                                 uint32_t pool_size, uint32_t steps, uint64_t rng_seed, uint32_t* src,
                                 uint32_t* dst, int mem_kind, void* stream)
{
    clear_error();
    if (!g) return fail(CSAW_ERR_INVALID, "graph is NULL");
    AllocScope alloc_scope(g);
    if (mem_kind != CSAW_MEM_HOST && mem_kind != CSAW_MEM_DEVICE)
        return fail(CSAW_ERR_INVALID, "bad mem_kind %d", mem_kind);
    if (pool_size == 0 || pool_size > CSAW_MDRW_MAX_POOL)
        return fail(CSAW_ERR_INVALID, "pool_size %u outside 1..%u", pool_size, CSAW_MDRW_MAX_POOL);
    if (n_instances > 0xFFFFFFFFull) return fail(CSAW_ERR_INVALID, "at most 2^32-1 instances per call");
    if (n_instances == 0) return CSAW_OK;
    if (!pools) return fail(CSAW_ERR_INVALID, "pools is NULL");
    if (steps > 0 && (!src || !dst)) return fail(CSAW_ERR_INVALID, "src/dst is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t pool_elems = n_instances * (uint64_t)pool_size;
    const uint64_t out_elems = n_instances * (uint64_t)steps;
    const uint32_t nblk = (pool_size + 31) / 32;

    void* d_pools = (void*)pools;
    void* d_src = src;
    void* d_dst = dst;
    void* ids = nullptr;
    void* dgs = nullptr;
    void* bsum = nullptr;
    void* counter = nullptr;
    csaw_status st = CSAW_OK;
    auto cleanup = [&]() {
        if (mem_kind == CSAW_MEM_HOST) { dfree(d_pools, s); dfree(d_src, s); dfree(d_dst, s); }
        dfree(ids, s); dfree(dgs, s); dfree(bsum, s); dfree(counter, s);
    };
    if (mem_kind == CSAW_MEM_HOST) {
        d_pools = d_src = d_dst = nullptr;
        st = dalloc(&d_pools, sizeof(uint32_t) * pool_elems, s);
        if (st == CSAW_OK) st = dalloc(&d_src, sizeof(uint32_t) * out_elems, s);
        if (st == CSAW_OK) st = dalloc(&d_dst, sizeof(uint32_t) * out_elems, s);
        if (st == CSAW_OK) {
            cudaError_t e = cudaMemcpyAsync(d_pools, pools, sizeof(uint32_t) * pool_elems,
                                            cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) st = cuda_fail(e, "copy pools");
        }
    }
    if (st == CSAW_OK) st = dalloc(&ids, sizeof(uint32_t) * pool_elems, s);
    const bool small = pool_size <= MDRW_SMALL_POOL;   // degrees and block sums kept on chip
    if (st == CSAW_OK) st = dalloc(&dgs, small ? 16 : sizeof(uint32_t) * pool_elems, s);
    if (st == CSAW_OK) st = dalloc(&bsum, small ? 16 : sizeof(uint64_t) * n_instances * nblk, s);
    if (st == CSAW_OK) st = dalloc(&counter, sizeof(unsigned long long), s);
    if (st == CSAW_OK) {
        cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) st = cuda_fail(e, "memset counter");
    }
    if (st == CSAW_OK) {
        MdrwParams p;
        p.off = g->off; p.col = g->col; p.deg = g->deg; p.V = g->V;
        p.pools = (const uint32_t*)d_pools;
        p.n = n_instances; p.m = pool_size; p.steps = steps;
        p.nblk = nblk; p.per_lane = (nblk + 31) / 32;
        p.ids = (uint32_t*)ids; p.dg = (uint32_t*)dgs; p.bs = (uint64_t*)bsum;
        p.keys = philox_round_keys(rng_seed);
        p.src = (uint32_t*)d_src; p.dst = (uint32_t*)d_dst;
        p.next = (unsigned long long*)counter;
        st = small ? launch_mdrw<true>(p, g->sm_count, s) : launch_mdrw<false>(p, g->sm_count, s);
    }
    if (st == CSAW_OK && mem_kind == CSAW_MEM_HOST && out_elems > 0) {
        cudaError_t e = cudaMemcpyAsync(src, d_src, sizeof(uint32_t) * out_elems, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dst, d_dst, sizeof(uint32_t) * out_elems, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) st = cuda_fail(e, "copy src/dst");
    }
    cleanup();
    if (st == CSAW_OK && mem_kind == CSAW_MEM_HOST) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "mdrw");
    }
    return st;
}
