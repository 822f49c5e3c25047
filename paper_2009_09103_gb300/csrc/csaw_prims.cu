// csaw_prims.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// Both read their element count from device memory (so a pipeline of calls
// needs no host round trip and can be captured in a CUDA graph) and use a
// fixed grid whose blocks each own a contiguous range of tiles.  Frontier
// compaction (Update, Eq. 4: the next frontier is the sorted set of picks
// minus the visited set) is built from these two.
#include "csaw_internal.cuh"

namespace csaw {

// ---------------------------------------------------------------- scan
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr uint64_t SCAN_TILE = (uint64_t)SCAN_THREADS * SCAN_ITEMS;
constexpr int SCAN_MAX_BLOCKS = 1024;

static int scan_blocks(uint64_t n_max)
{
    uint64_t tiles = (n_max + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles < 1) tiles = 1;
    return (int)(tiles < (uint64_t)SCAN_MAX_BLOCKS ? tiles : SCAN_MAX_BLOCKS);
}

size_t scan_scratch_bytes(uint64_t) { return sizeof(uint64_t) * (SCAN_MAX_BLOCKS + 1); }

__device__ __forceinline__ void block_range(uint64_t n, uint64_t tile, uint64_t* lo, uint64_t* hi)
{
    const uint64_t tiles = (n + tile - 1) / tile;
    const uint64_t per = (tiles + gridDim.x - 1) / gridDim.x;
    uint64_t b = (uint64_t)blockIdx.x * per * tile;
    uint64_t e = b + per * tile;
    *lo = b < n ? b : n;
    *hi = e < n ? e : n;
}

// Block-wide exclusive scan of one uint64 per thread; returns the block total.
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* excl, uint64_t* s_warp)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t incl = warp_inclusive_scan_u64(v, lane);
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        uint64_t t = lane < nw ? s_warp[lane] : 0;
        const uint64_t ti = warp_inclusive_scan_u64(t, lane);
        if (lane < nw) s_warp[lane] = ti - t;
        if (lane == nw - 1) s_warp[32] = ti;
    }
    __syncthreads();
    *excl = s_warp[wid] + incl - v;
    const uint64_t total = s_warp[32];
    __syncthreads();
    return total;
}

__global__ void scan_reduce_kernel(const uint32_t* __restrict__ in, const uint64_t* __restrict__ n_dev,
                                   uint64_t* __restrict__ bsum)
{
    __shared__ uint64_t s_warp[33];
    uint64_t lo, hi;
    block_range(*n_dev, SCAN_TILE, &lo, &hi);
    uint64_t s = 0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += SCAN_THREADS) s += in[i];
    uint64_t excl;
    const uint64_t total = block_exclusive_scan(s, &excl, s_warp);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void scan_top_kernel(uint64_t* __restrict__ bsum, int nblocks, uint64_t* __restrict__ total_out)
{
    __shared__ uint64_t s_warp[33];
    // nblocks <= 1024 = blockDim: one value per thread
    const uint64_t v = (int)threadIdx.x < nblocks ? bsum[threadIdx.x] : 0;
    uint64_t excl;
    const uint64_t total = block_exclusive_scan(v, &excl, s_warp);
    if ((int)threadIdx.x < nblocks) bsum[threadIdx.x] = excl;
    if (threadIdx.x == 0 && total_out) *total_out = total;
}

__global__ void scan_down_kernel(const uint32_t* __restrict__ in, const uint64_t* __restrict__ n_dev,
                                 const uint64_t* __restrict__ boff, uint64_t* __restrict__ out)
{
    __shared__ uint64_t s_warp[33];
    const uint64_t n = *n_dev;
    uint64_t lo, hi;
    block_range(n, SCAN_TILE, &lo, &hi);
    uint64_t base = boff[blockIdx.x];
    for (uint64_t t0 = lo; t0 < hi; t0 += SCAN_TILE) {
        const uint64_t my = t0 + (uint64_t)threadIdx.x * SCAN_ITEMS;
        uint32_t v[SCAN_ITEMS];
        uint64_t s = 0;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; ++j) {
            v[j] = (my + j < hi) ? in[my + j] : 0u;
            s += v[j];
        }
        uint64_t excl;
        const uint64_t total = block_exclusive_scan(s, &excl, s_warp);
        uint64_t run = base + excl;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; ++j) {
            if (my + j < hi) out[my + j] = run;
            run += v[j];
        }
        base += total;
    }
    // the last block writes out[n] = grand total
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = base;
}

// out[i] = sum of in[0..i) for i <= n; *total_out (optional, device) = out[n].
csaw_status scan_u32(const uint32_t* in, uint64_t* out, const uint64_t* n_dev, uint64_t n_max,
                     void* scratch, uint64_t* total_out, cudaStream_t s)
{
    const int nb = scan_blocks(n_max);
    uint64_t* bsum = (uint64_t*)scratch;
    scan_reduce_kernel<<<nb, SCAN_THREADS, 0, s>>>(in, n_dev, bsum);
    scan_top_kernel<<<1, SCAN_MAX_BLOCKS, 0, s>>>(bsum, nb, total_out);
    scan_down_kernel<<<nb, SCAN_THREADS, 0, s>>>(in, n_dev, bsum, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "scan kernels");
    return CSAW_OK;
}

// ---------------------------------------------------------------- radix sort
// Stable LSD sort of uint64 keys, 8 bits per pass.  Pass = per-block digit
// histograms, one scan over (digit, block), and a scatter in which every
// block walks its tiles in order; inside a tile each warp ranks its 32-key
// rounds with __match_any_sync, and warps are combined in order, so equal
// digits keep their input order.
constexpr int SORT_THREADS = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_ROUNDS = 8;                                       // 32-key rounds per warp per tile
constexpr uint64_t SORT_TILE = (uint64_t)SORT_THREADS * SORT_ROUNDS; // 2048 keys
constexpr int SORT_MAX_BLOCKS = 1024;
constexpr int RADIX = 256;

static int sort_blocks(uint64_t n_max, int sm_count)
{
    uint64_t tiles = (n_max + SORT_TILE - 1) / SORT_TILE;
    if (tiles < 1) tiles = 1;
    uint64_t cap = (uint64_t)sm_count * 4;
    if (cap > SORT_MAX_BLOCKS) cap = SORT_MAX_BLOCKS;
    return (int)(tiles < cap ? tiles : cap);
}

size_t sort_scratch_bytes(uint64_t) { return sizeof(uint32_t) * ((size_t)RADIX * SORT_MAX_BLOCKS + RADIX) + 64; }

__global__ void __launch_bounds__(SORT_THREADS) sort_hist_kernel(const uint64_t* __restrict__ keys,
                                                                 const uint64_t* __restrict__ n_dev,
                                                                 int shift, uint32_t* __restrict__ hist)
{
    __shared__ uint32_t s_h[RADIX];
    for (int i = threadIdx.x; i < RADIX; i += SORT_THREADS) s_h[i] = 0;
    __syncthreads();
    uint64_t lo, hi;
    block_range(*n_dev, SORT_TILE, &lo, &hi);
    for (uint64_t i = lo + threadIdx.x; i < hi; i += SORT_THREADS)
        atomicAdd(&s_h[(keys[i] >> shift) & (RADIX - 1)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += SORT_THREADS) hist[(size_t)d * gridDim.x + blockIdx.x] = s_h[d];
}

// Exclusive scan of each digit's per-block counts, in place (one CTA per
// digit, its counts are contiguous in the digit-major layout); the digit's
// total goes to dtot[digit].
__global__ void sort_scan_kernel(uint32_t* __restrict__ hist, int nblocks, uint32_t* __restrict__ dtot)
{
    __shared__ uint64_t s_warp[33];
    uint32_t* h = hist + (size_t)blockIdx.x * nblocks;
    uint64_t carry = 0;
    for (int base = 0; base < nblocks; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nblocks ? h[i] : 0u;
        uint64_t excl;
        const uint64_t tot = block_exclusive_scan(v, &excl, s_warp);
        if (i < nblocks) h[i] = (uint32_t)(carry + excl);
        carry += tot;
    }
    if (threadIdx.x == 0) dtot[blockIdx.x] = (uint32_t)carry;
}

__global__ void __launch_bounds__(SORT_THREADS) sort_scatter_kernel(const uint64_t* __restrict__ keys,
                                                                    uint64_t* __restrict__ out,
                                                                    const uint64_t* __restrict__ n_dev,
                                                                    int shift,
                                                                    const uint32_t* __restrict__ hist,
                                                                    const uint32_t* __restrict__ dtot)
{
    __shared__ uint32_t s_base[RADIX];             // next output slot of each digit for this block
    __shared__ uint32_t s_cnt[SORT_WARPS][RADIX];  // per-warp digit counts, then warp offsets
    __shared__ uint64_t s_warp[33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    {
        // start of each digit = earlier digits' totals + earlier blocks' counts
        static_assert(SORT_THREADS == RADIX, "one digit per thread");
        uint64_t digit_base;
        block_exclusive_scan(dtot[threadIdx.x], &digit_base, s_warp);
        s_base[threadIdx.x] = (uint32_t)digit_base + hist[(size_t)threadIdx.x * gridDim.x + blockIdx.x];
    }
    uint64_t lo, hi;
    block_range(*n_dev, SORT_TILE, &lo, &hi);
    const uint32_t lt = lanemask_lt();
    for (uint64_t t0 = lo; t0 < hi; t0 += SORT_TILE) {
        for (int i = threadIdx.x; i < SORT_WARPS * RADIX; i += SORT_THREADS) (&s_cnt[0][0])[i] = 0;
        __syncthreads();
        uint64_t k[SORT_ROUNDS];
        uint32_t dig[SORT_ROUNDS], loc[SORT_ROUNDS];
        const uint64_t wbase = t0 + (uint64_t)wid * 32 * SORT_ROUNDS;
#pragma unroll
        for (int r = 0; r < SORT_ROUNDS; ++r) {
            const uint64_t i = wbase + (uint64_t)r * 32 + lane;
            const bool valid = i < hi;
            k[r] = valid ? keys[i] : 0;
            dig[r] = valid ? (uint32_t)((k[r] >> shift) & (RADIX - 1)) : (uint32_t)RADIX;
        }
#pragma unroll
        for (int r = 0; r < SORT_ROUNDS; ++r) {
            const uint32_t peers = __match_any_sync(CSAW_FULL_MASK, dig[r]);
            const int leader = __ffs(peers) - 1;
            uint32_t before = 0;
            if (lane == leader && dig[r] < RADIX) {
                before = s_cnt[wid][dig[r]];
                s_cnt[wid][dig[r]] = before + __popc(peers);
            }
            before = __shfl_sync(CSAW_FULL_MASK, before, leader);
            loc[r] = before + __popc(peers & lt);
            __syncwarp();
        }
        __syncthreads();
        // warp offsets per digit, in warp order, starting at the block's base
        for (int d = threadIdx.x; d < RADIX; d += SORT_THREADS) {
            uint32_t run = s_base[d];
#pragma unroll
            for (int w = 0; w < SORT_WARPS; ++w) {
                const uint32_t c = s_cnt[w][d];
                s_cnt[w][d] = run;
                run += c;
            }
            s_base[d] = run;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < SORT_ROUNDS; ++r)
            if (dig[r] < RADIX) out[s_cnt[wid][dig[r]] + loc[r]] = k[r];
        __syncthreads();
    }
}

// Sort n keys (n at *n_dev, at most n_max < 2^32) on their low `bits` bits.
// keys and alt are both n_max long; *result points at whichever holds the
// sorted keys.
csaw_status radix_sort_u64(uint64_t* keys, uint64_t* alt, const uint64_t* n_dev, uint64_t n_max,
                           int bits, int sm_count, void* scratch, cudaStream_t s, uint64_t** result)
{
    if (n_max >= 0xFFFFFFFFull) return fail(CSAW_ERR_INVALID, "radix sort limited to 2^32-1 keys");
    const int nb = sort_blocks(n_max, sm_count);
    uint32_t* hist = (uint32_t*)scratch;
    uint32_t* dtot = hist + (size_t)RADIX * SORT_MAX_BLOCKS;
    uint64_t* src = keys;
    uint64_t* dst = alt;
    for (int shift = 0; shift < bits; shift += 8) {
        sort_hist_kernel<<<nb, SORT_THREADS, 0, s>>>(src, n_dev, shift, hist);
        sort_scan_kernel<<<RADIX, 256, 0, s>>>(hist, nb, dtot);
        sort_scatter_kernel<<<nb, SORT_THREADS, 0, s>>>(src, dst, n_dev, shift, hist, dtot);
        uint64_t* t = src; src = dst; dst = t;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "radix sort kernels");
    *result = src;
    return CSAW_OK;
}

}  // namespace csaw
