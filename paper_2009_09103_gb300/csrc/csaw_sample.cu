// csaw_sample.cu -- layered biased neighbour sampling over many instances.
//
// The framework loop of C-SAW (Sec. III-B, Fig. 2(b)) for traversal-based
// sampling: every vertex of the frontier selects up to fanout[l] neighbours
// by inverse transform sampling (Sec. II-B, Eq. 1) without replacement
// (Sec. IV-B), each pick is a sampled edge, and Update (Eq. 4) forms the next
// frontier from the picks that the instance has not visited.
//
// Device layout per layer l:
//   frontier   sorted uint64 keys (instance << vbits | vertex), with per
//              instance ranges foff[i] .. foff[i+1]
//   counts     picks per frontier entry, min(k, #positive biases), and their
//              exclusive scan pos[] (edge position of each entry)
//   edges      src/dst (uint32) at pos[e] .. pos[e+1]; for all but the last
//              layer also candidate keys (instance << vbits | dst)
// Work split: entries whose neighbours are all taken, or with degree <= 256,
// are warp items (cumulative bias array in shared memory); the rest are CTA
// items: the CTA builds the cumulative array (shared memory up to 8192
// neighbours, a per-CTA global scratch slot above that) and one warp draws.
// A persistent grid takes CTA items first, then warp items, from two
// atomic counters.
//
// Draws: attempt a of frontier vertex v in instance i at layer l uses the
// Philox counter (a, v, l, i).  A warp evaluates attempts 32j .. 32j+31 at
// once; a lane's pick is new if no earlier lane of the round and no earlier
// round chose it (__match_any_sync plus a bitmap), and new picks are kept in
// lane order while fewer than k are held.  After CSAW_ATTEMPT_CAP attempts the
// remaining picks use updated sampling (Sec. IV-B, Fig. 5(b)): the draw is
// scaled to the unpicked total and mapped past the picked intervals, which is
// the same choice as searching a recomputed prefix sum.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "csaw_internal.cuh"

namespace csaw {

constexpr int SEL_THREADS = 256;
constexpr int SEL_WARPS = SEL_THREADS / 32;
constexpr uint32_t WARP_MAX_DEG = 256;     // warp items: degree <= this
constexpr uint32_t CTA_SMEM_DEG = 8192;    // CTA items keep S in shared memory up to this
constexpr uint32_t WARP_SLOT = WARP_MAX_DEG * 8 + (WARP_MAX_DEG / 32) * 4;   // bytes per warp
constexpr size_t SEL_DYN_SMEM = (size_t)CTA_SMEM_DEG * 8 + (CTA_SMEM_DEG / 32) * 4;

static_assert(SEL_WARPS * WARP_SLOT <= SEL_DYN_SMEM, "warp slots reuse the CTA region");

struct SelParams {
    const uint64_t* __restrict__ off;
    const uint32_t* __restrict__ col;
    const uint32_t* __restrict__ w;
    const uint32_t* __restrict__ deg;
    const uint64_t* __restrict__ fkeys;
    uint32_t vbits;
    uint64_t vmask;
    uint32_t k;
    uint32_t layer;
    uint32_t k0, k1;
    bool zero_bias;                       // some bias of this kind may be zero
    const uint64_t* __restrict__ pos;     // [n+1]
    const uint32_t* __restrict__ warp_list;
    const uint32_t* __restrict__ cta_list;
    const unsigned long long* n_items;    // [0] warp items, [1] CTA items
    unsigned long long* next;             // [0] warp counter, [1] CTA counter
    uint32_t* __restrict__ out_src;
    uint32_t* __restrict__ out_dst;
    uint64_t* __restrict__ out_cand;      // nullptr on the last layer
    uint64_t* __restrict__ scratch_S;     // per-CTA slots for CTA items above CTA_SMEM_DEG
    uint32_t* __restrict__ scratch_bits;
    uint64_t scratch_stride;              // entries per slot (max degree)
};

template <int KIND>
__device__ __forceinline__ uint32_t sel_bias(const SelParams& p, uint64_t e)
{
    if constexpr (KIND == CSAW_BIAS_UNIFORM) return 1u;
    else if constexpr (KIND == CSAW_BIAS_EDGE_WEIGHT) return __ldg(p.w + e);
    else return __ldg(p.deg + __ldg(p.col + e));
}

__device__ __forceinline__ void emit(const SelParams& p, uint64_t q, uint32_t v, uint32_t inst, uint32_t u)
{
    p.out_src[q] = v;
    p.out_dst[q] = u;
    if (p.out_cand) p.out_cand[q] = ((uint64_t)inst << p.vbits) | u;
}

// Smallest i in [0, d) with S[i] > x (S inclusive prefix sums, x < S[d-1]).
__device__ __forceinline__ uint32_t upper_bound_S(const uint64_t* S, uint32_t d, uint64_t x)
{
    uint32_t lo = 0, hi = d;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (S[mid] > x) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Attempt rounds of one warp over a built prefix array S[0..d) with total T.
// bits: d-bit chosen set, already cleared.  Emits picks at q0 + have.
__device__ void draw_picks(const SelParams& p, const uint64_t* S, uint32_t* bits, uint32_t d,
                           uint64_t T, uint32_t cnt, uint64_t q0, uint32_t v, uint32_t inst,
                           uint64_t beg, int lane)
{
    const uint32_t lt = lanemask_lt();
    uint32_t have = 0;
    uint32_t a0 = 0;
    while (have < cnt && a0 < CSAW_ATTEMPT_CAP) {
        const uint64_t r = philox_draw(p.k0, p.k1, a0 + lane, v, p.layer, inst);
        const uint32_t i = upper_bound_S(S, d, scale_draw(r, T));
        const bool chosen = (bits[i >> 5] >> (i & 31)) & 1u;
        const uint32_t peers = __match_any_sync(CSAW_FULL_MASK, i);
        const bool fresh = !chosen && lane == __ffs(peers) - 1;
        const uint32_t bal = __ballot_sync(CSAW_FULL_MASK, fresh);
        const uint32_t rank = __popc(bal & lt);
        const uint32_t need = cnt - have;
        if (fresh && rank < need) {
            emit(p, q0 + have + rank, v, inst, __ldg(p.col + beg + i));
            atomicOr(bits + (i >> 5), 1u << (i & 31));
        }
        have += min((uint32_t)__popc(bal), need);
        a0 += 32;
        __syncwarp();
    }
    if (have >= cnt) return;
    // Updated sampling for the remaining picks (attempts CSAW_ATTEMPT_CAP, ...).
    const uint32_t nwords = (d + 31) >> 5;
    uint64_t R = 0;
    for (uint32_t wi = lane; wi < nwords; wi += 32) {
        uint32_t m = bits[wi];
        while (m) {
            const uint32_t i = (wi << 5) + __ffs(m) - 1;
            m &= m - 1;
            R += S[i] - (i ? S[i - 1] : 0);
        }
    }
    R = warp_sum_u64(R);
    if (lane == 0) {
        for (uint32_t a = CSAW_ATTEMPT_CAP; have < cnt; ++a) {
            const uint64_t r = philox_draw(p.k0, p.k1, a, v, p.layer, inst);
            uint64_t x = scale_draw(r, T - R);
            // Walk the picked intervals in ascending order, skipping each one
            // that starts at or below the running position.
            bool done = false;
            for (uint32_t wi = 0; wi < nwords && !done; ++wi) {
                uint32_t m = bits[wi];
                while (m) {
                    const uint32_t i = (wi << 5) + __ffs(m) - 1;
                    m &= m - 1;
                    const uint64_t start = i ? S[i - 1] : 0;
                    if (x >= start) x += S[i] - start;
                    else { done = true; break; }
                }
            }
            const uint32_t i = min(upper_bound_S(S, d, x), d - 1);   // x < T: always inside
            bits[i >> 5] |= 1u << (i & 31);
            R += S[i] - (i ? S[i - 1] : 0);
            emit(p, q0 + have, v, inst, __ldg(p.col + beg + i));
            ++have;
        }
    }
    __syncwarp();
}

// One warp item: all positive neighbours (any degree), or a draw over at most
// WARP_MAX_DEG neighbours with S in this warp's shared slot.
template <int KIND>
__device__ void warp_item(const SelParams& p, uint32_t e, uint64_t* sS, uint32_t* sBits, int lane)
{
    const uint64_t key = p.fkeys[e];
    const uint32_t v = (uint32_t)(key & p.vmask);
    const uint32_t inst = (uint32_t)(key >> p.vbits);
    const uint64_t beg = __ldg(p.off + v);
    const uint32_t d = (uint32_t)(__ldg(p.off + v + 1) - beg);
    const uint64_t q0 = p.pos[e];
    const uint32_t cnt = (uint32_t)(p.pos[e + 1] - q0);
    const uint32_t lt = lanemask_lt();
    if (d > WARP_MAX_DEG) {
        // Take-all over a long row: stream it, keeping positive biases in CSR order.
        uint64_t q = q0;
        for (uint32_t base = 0; base < d; base += 32) {
            const uint32_t j = base + lane;
            bool take = false;
            uint32_t u = 0;
            if (j < d) {
                u = __ldg(p.col + beg + j);
                take = p.zero_bias ? sel_bias<KIND>(p, beg + j) > 0 : true;
            }
            const uint32_t bal = __ballot_sync(CSAW_FULL_MASK, take);
            if (take) emit(p, q + __popc(bal & lt), v, inst, u);
            q += __popc(bal);
        }
        return;
    }
    constexpr int TILES = WARP_MAX_DEG / 32;
    const uint32_t ntiles = (d + 31) >> 5;
    uint32_t b[TILES];
#pragma unroll
    for (int t = 0; t < TILES; ++t) {
        const uint32_t j = 32u * t + lane;
        b[t] = ((uint32_t)t < ntiles && j < d) ? sel_bias<KIND>(p, beg + j) : 0u;
    }
    uint64_t run = 0;
    uint32_t npos = 0;
#pragma unroll
    for (int t = 0; t < TILES; ++t) {
        if ((uint32_t)t < ntiles) {
            const uint64_t incl = warp_inclusive_scan_u64(b[t], lane) + run;
            const uint32_t j = 32u * t + lane;
            if (j < d) sS[j] = incl;
            run = __shfl_sync(CSAW_FULL_MASK, incl, 31);
            npos += __popc(__ballot_sync(CSAW_FULL_MASK, b[t] > 0));
        }
    }
    if (npos <= p.k) {
        uint64_t q = q0;
#pragma unroll
        for (int t = 0; t < TILES; ++t) {
            if ((uint32_t)t < ntiles) {
                const bool take = b[t] > 0;
                const uint32_t bal = __ballot_sync(CSAW_FULL_MASK, take);
                if (take) emit(p, q + __popc(bal & lt), v, inst, __ldg(p.col + beg + 32u * t + lane));
                q += __popc(bal);
            }
        }
        return;
    }
    if (lane < (int)(WARP_MAX_DEG / 32)) sBits[lane] = 0;
    __syncwarp();
    draw_picks(p, sS, sBits, d, run, cnt, q0, v, inst, beg, lane);
    __syncwarp();
}

// One CTA item: degree > WARP_MAX_DEG and more positive neighbours than k.
template <int KIND>
__device__ void cta_item(const SelParams& p, uint32_t e, uint64_t* S, uint32_t* bits,
                         uint64_t* s_wsum)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t key = p.fkeys[e];
    const uint32_t v = (uint32_t)(key & p.vmask);
    const uint32_t inst = (uint32_t)(key >> p.vbits);
    const uint64_t beg = __ldg(p.off + v);
    const uint32_t d = (uint32_t)(__ldg(p.off + v + 1) - beg);
    const uint64_t q0 = p.pos[e];
    const uint32_t cnt = (uint32_t)(p.pos[e + 1] - q0);
    const uint32_t nwords = (d + 31) >> 5;
    for (uint32_t i = threadIdx.x; i < nwords; i += SEL_THREADS) bits[i] = 0;
    // Build S: each warp scans a contiguous 256-neighbour segment of the
    // 2048-neighbour tile, then segment offsets are added in warp order.
    uint64_t carry = 0;
    for (uint32_t base = 0; base < d; base += SEL_WARPS * 256u) {
        const uint32_t seg = base + (uint32_t)wid * 256u;
        uint32_t b[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const uint32_t j = seg + 32u * t + lane;
            b[t] = j < d ? sel_bias<KIND>(p, beg + j) : 0u;
        }
        uint64_t incl[8];
        uint64_t run = 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            incl[t] = warp_inclusive_scan_u64(b[t], lane) + run;
            run = __shfl_sync(CSAW_FULL_MASK, incl[t], 31);
        }
        if (lane == 0) s_wsum[wid] = run;
        __syncthreads();
        uint64_t offw = carry, tile = 0;
#pragma unroll
        for (int w2 = 0; w2 < SEL_WARPS; ++w2) {
            const uint64_t sw = s_wsum[w2];
            if (w2 < wid) offw += sw;
            tile += sw;
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const uint32_t j = seg + 32u * t + lane;
            if (j < d) S[j] = offw + incl[t];
        }
        carry += tile;
        __syncthreads();
    }
    if (wid == 0) draw_picks(p, S, bits, d, carry, cnt, q0, v, inst, beg, lane);
    __syncthreads();
}

template <int KIND>
__global__ void __launch_bounds__(SEL_THREADS) select_kernel(SelParams p)
{
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ uint64_t s_wsum[SEL_WARPS];
    __shared__ unsigned long long s_item;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // CTA items first: the long rows.
    const unsigned long long n_cta = p.n_items[1];
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(p.next + 1, 1ull);
        __syncthreads();
        const unsigned long long it = s_item;
        __syncthreads();
        if (it >= n_cta) break;
        const uint32_t e = p.cta_list[it];
        const uint32_t d = (uint32_t)(__ldg(p.off + (uint32_t)(p.fkeys[e] & p.vmask) + 1) -
                                      __ldg(p.off + (uint32_t)(p.fkeys[e] & p.vmask)));
        uint64_t* S;
        uint32_t* bits;
        if (d <= CTA_SMEM_DEG) {
            S = (uint64_t*)s_dyn;
            bits = (uint32_t*)(s_dyn + (size_t)CTA_SMEM_DEG * 8);
        } else {
            S = p.scratch_S + (size_t)blockIdx.x * p.scratch_stride;
            bits = p.scratch_bits + (size_t)blockIdx.x * ((p.scratch_stride + 31) / 32);
        }
        cta_item<KIND>(p, e, S, bits, s_wsum);
    }
    // Warp items: each warp uses its own slice of the dynamic region.
    uint64_t* sS = (uint64_t*)(s_dyn + (size_t)wid * WARP_SLOT);
    uint32_t* sBits = (uint32_t*)(s_dyn + (size_t)wid * WARP_SLOT + WARP_MAX_DEG * 8);
    const unsigned long long n_warp = p.n_items[0];
    while (true) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(p.next, 1ull);
        it = __shfl_sync(CSAW_FULL_MASK, it, 0);
        if (it >= n_warp) break;
        warp_item<KIND>(p, p.warp_list[it], sS, sBits, lane);
    }
}

// ---------------------------------------------------------------------------
// Per-entry counts and work lists.

struct CountParams {
    const uint64_t* __restrict__ off;
    const uint32_t* __restrict__ col;
    const uint32_t* __restrict__ w;
    const uint32_t* __restrict__ deg;
    const uint64_t* __restrict__ fkeys;
    const unsigned long long* n_dev;
    uint64_t vmask;
    uint32_t k;
    bool zero_bias;
    uint32_t* __restrict__ cnt;
    uint32_t* __restrict__ warp_list;
    uint32_t* __restrict__ cta_list;
    unsigned long long* n_items;   // [0] warp, [1] CTA
};

// Number of positive biases of v's neighbours (only when zeros are possible).
template <int KIND>
__device__ uint32_t count_positive(const CountParams& p, uint64_t beg, uint32_t d, int lane)
{
    uint32_t c = 0;
    for (uint32_t j = lane; j < d; j += 32) {
        uint32_t b;
        if constexpr (KIND == CSAW_BIAS_UNIFORM) b = 1u;
        else if constexpr (KIND == CSAW_BIAS_EDGE_WEIGHT) b = __ldg(p.w + beg + j);
        else b = __ldg(p.deg + __ldg(p.col + beg + j));
        c += b > 0;
    }
    return __reduce_add_sync(CSAW_FULL_MASK, c);
}

template <int KIND>
__global__ void count_kernel(CountParams p)
{
    const int lane = threadIdx.x & 31;
    const uint64_t n = *p.n_dev;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    // one warp handles 32 consecutive entries; the positive count (if needed)
    // is computed cooperatively entry by entry
    for (uint64_t base = gw * 32; base < n; base += nw * 32) {
        const uint64_t e = base + lane;
        uint32_t v = 0, d = 0;
        uint64_t beg = 0;
        if (e < n) {
            v = (uint32_t)(p.fkeys[e] & p.vmask);
            beg = __ldg(p.off + v);
            d = (uint32_t)(__ldg(p.off + v + 1) - beg);
        }
        uint32_t npos = d;
        if (p.zero_bias) {
            for (int l = 0; l < 32; ++l) {
                const uint64_t bl = __shfl_sync(CSAW_FULL_MASK, beg, l);
                const uint32_t dl = __shfl_sync(CSAW_FULL_MASK, d, l);
                const uint32_t c = count_positive<KIND>(p, bl, dl, lane);
                if (lane == l) npos = c;
            }
        }
        const uint32_t c = min(p.k, npos);
        const bool take_all = npos <= p.k;
        const bool to_warp = e < n && c > 0 && (take_all || d <= WARP_MAX_DEG);
        const bool to_cta = e < n && c > 0 && !to_warp;
        if (e < n) p.cnt[e] = c;
        // warp-aggregated appends
        const uint32_t bw = __ballot_sync(CSAW_FULL_MASK, to_warp);
        const uint32_t bc = __ballot_sync(CSAW_FULL_MASK, to_cta);
        unsigned long long basew = 0, basec = 0;
        if (lane == 0) {
            if (bw) basew = atomicAdd(p.n_items, (unsigned long long)__popc(bw));
            if (bc) basec = atomicAdd(p.n_items + 1, (unsigned long long)__popc(bc));
        }
        basew = __shfl_sync(CSAW_FULL_MASK, basew, 0);
        basec = __shfl_sync(CSAW_FULL_MASK, basec, 0);
        const uint32_t lt = lanemask_lt();
        if (to_warp) p.warp_list[basew + __popc(bw & lt)] = (uint32_t)e;
        if (to_cta) p.cta_list[basec + __popc(bc & lt)] = (uint32_t)e;
    }
}

// ---------------------------------------------------------------------------
// Frontier construction.

// Keys of the seeds: instance of seed j from the offsets, checks ranges.
__global__ void seed_keys_kernel(const uint32_t* __restrict__ seeds, const uint64_t* __restrict__ inst_off,
                                 uint32_t n_inst, uint64_t n_seeds, uint32_t V, uint32_t vbits,
                                 uint64_t* __restrict__ keys, uint32_t* __restrict__ err)
{
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_seeds;
         j += (uint64_t)gridDim.x * blockDim.x) {
        // instance = last i with inst_off[i] <= j
        uint32_t lo = 0, hi = n_inst;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (inst_off[mid] <= j) lo = mid; else hi = mid - 1;
        }
        const uint32_t s = seeds[j];
        if (s >= V) atomicOr(err, 1u);
        keys[j] = ((uint64_t)lo << vbits) | (s < V ? s : 0u);
    }
}

__global__ void check_inst_off_kernel(const uint64_t* __restrict__ inst_off, uint32_t n_inst,
                                      uint32_t* __restrict__ err)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_inst;
         i += (uint64_t)gridDim.x * blockDim.x)
        if (inst_off[i + 1] < inst_off[i]) atomicOr(err, 2u);
    if (blockIdx.x == 0 && threadIdx.x == 0 && inst_off[0] != 0) atomicOr(err, 2u);
}

struct Visited {
    const uint64_t* keys[CSAW_MAX_DEPTH];
    const uint64_t* foff[CSAW_MAX_DEPTH];
    int n;
};

// kept[i] = 1 for the first of each run of equal sorted keys that no earlier
// frontier of its instance holds.
__global__ void unique_filter_kernel(const uint64_t* __restrict__ sorted, const uint64_t* n_dev,
                                     Visited vis, uint32_t vbits, uint32_t* __restrict__ kept)
{
    const uint64_t n = *n_dev;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t key = sorted[i];
        bool keep = i == 0 || sorted[i - 1] != key;
        const uint32_t inst = (uint32_t)(key >> vbits);
        for (int j = 0; j < vis.n && keep; ++j) {
            uint64_t lo = vis.foff[j][inst], hi = vis.foff[j][inst + 1];
            const uint64_t end = hi;
            while (lo < hi) {
                const uint64_t mid = lo + ((hi - lo) >> 1);
                if (vis.keys[j][mid] < key) lo = mid + 1; else hi = mid;
            }
            if (lo < end && vis.keys[j][lo] == key) keep = false;
        }
        kept[i] = keep ? 1u : 0u;
    }
}

__global__ void scatter_kept_kernel(const uint64_t* __restrict__ sorted, const uint64_t* n_dev,
                                    const uint32_t* __restrict__ kept, const uint64_t* __restrict__ kpos,
                                    uint64_t* __restrict__ out)
{
    const uint64_t n = *n_dev;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        if (kept[i]) out[kpos[i]] = sorted[i];
}

// foff[i] = first position of instance i in the sorted frontier, i <= n_inst.
__global__ void inst_bounds_kernel(const uint64_t* __restrict__ keys, const uint64_t* n_dev,
                                   uint32_t n_inst, uint32_t vbits, uint64_t* __restrict__ foff)
{
    const uint64_t n = *n_dev;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n_inst;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t key = i << vbits;
        uint64_t lo = 0, hi = n;
        while (lo < hi) {
            const uint64_t mid = lo + ((hi - lo) >> 1);
            if (keys[mid] < key) lo = mid + 1; else hi = mid;
        }
        foff[i] = i == n_inst ? n : lo;
    }
}

// Edge offsets and frontier sizes of one layer:
// eoff[i] = base + pos[foff[i]] for i <= n_inst; fsize[i] = foff[i+1] - foff[i].
__global__ void layer_offsets_kernel(const uint64_t* __restrict__ foff, const uint64_t* __restrict__ pos,
                                     uint32_t n_inst, uint64_t base, uint64_t* __restrict__ eoff,
                                     uint64_t* __restrict__ fsize)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n_inst;
         i += (uint64_t)gridDim.x * blockDim.x) {
        eoff[i] = base + pos[foff[i]];
        if (i < n_inst) fsize[i] = foff[i + 1] - foff[i];
    }
}

static inline unsigned grid_for(uint64_t n, int threads, int sm_count)
{
    uint64_t b = (n + threads - 1) / threads;
    const uint64_t cap = (uint64_t)sm_count * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

static int bits_for(uint64_t maxval)
{
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) ++b;
    return b;
}

}  // namespace csaw

// ---------------------------------------------------------------------------
// Result object.
struct csaw_sample_result {
    uint32_t depth = 0;
    uint32_t n_instances = 0;
    uint64_t n_edges = 0;
    std::vector<uint64_t> edge_offsets;     // host
    std::vector<uint64_t> frontier_sizes;   // host
    std::vector<uint32_t*> src, dst;        // device, per layer
    std::vector<const uint32_t*> src_c, dst_c;
    std::vector<uint64_t> layer_edges;
    int device = 0;
    ~csaw_sample_result()
    {
        for (auto p : src) cudaFree(p);
        for (auto p : dst) cudaFree(p);
    }
};

namespace csaw {

// RAII list of stream-ordered temporaries.
struct Temps {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Temps(cudaStream_t st) : s(st) {}
    ~Temps() { for (void* p : ptrs) dfree(p, s); }
    template <class T>
    csaw_status get(T** out, size_t count)
    {
        void* p = nullptr;
        CSAW_TRY(dalloc(&p, count * sizeof(T), s));
        ptrs.push_back(p);
        *out = (T*)p;
        return CSAW_OK;
    }
};

template <int KIND>
static csaw_status launch_select(const SelParams& p, int blocks, cudaStream_t s)
{
    select_kernel<KIND><<<blocks, SEL_THREADS, SEL_DYN_SMEM, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "select_kernel");
    return CSAW_OK;
}

template <int KIND>
static csaw_status launch_count(const CountParams& p, uint64_t n, int sm_count, cudaStream_t s)
{
    count_kernel<KIND><<<grid_for((n + 31) / 32 * 32, 256, sm_count), 256, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "count_kernel");
    return CSAW_OK;
}

static int select_blocks(int kind, int sm_count)
{
    static int cached[4] = {0, 0, 0, 0};
    if (!cached[kind]) {
        int per_sm = 1;
        cudaError_t e = cudaSuccess;
        switch (kind) {
        case CSAW_BIAS_UNIFORM:
            cudaFuncSetAttribute(select_kernel<CSAW_BIAS_UNIFORM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SEL_DYN_SMEM);
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_kernel<CSAW_BIAS_UNIFORM>, SEL_THREADS, SEL_DYN_SMEM);
            break;
        case CSAW_BIAS_EDGE_WEIGHT:
            cudaFuncSetAttribute(select_kernel<CSAW_BIAS_EDGE_WEIGHT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SEL_DYN_SMEM);
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_kernel<CSAW_BIAS_EDGE_WEIGHT>, SEL_THREADS, SEL_DYN_SMEM);
            break;
        default:
            cudaFuncSetAttribute(select_kernel<CSAW_BIAS_NEIGHBOR_DEGREE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SEL_DYN_SMEM);
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_kernel<CSAW_BIAS_NEIGHBOR_DEGREE>, SEL_THREADS, SEL_DYN_SMEM);
            break;
        }
        if (e != cudaSuccess || per_sm < 1) per_sm = 1;
        cached[kind] = per_sm;
    }
    return sm_count * cached[kind];
}

static csaw_status run_sample(csaw_graph* g, const uint32_t* seeds, const uint64_t* inst_off,
                              uint32_t n_inst, uint64_t n_seeds, uint32_t depth, const uint32_t* fanout,
                              int kind, uint64_t rng_seed, cudaStream_t s, csaw_sample_result* R)
{
    Temps tmp(s);
    const int vbits = bits_for(g->V - 1) > 0 ? bits_for(g->V - 1) : 1;
    const int ibits = bits_for(n_inst > 0 ? n_inst - 1 : 0);
    const int kbits = vbits + ibits;
    const uint64_t vmask = (vbits >= 64) ? ~0ull : ((1ull << vbits) - 1);
    const bool zero_bias = (kind == CSAW_BIAS_EDGE_WEIGHT && g->min_weight == 0) ||
                           (kind == CSAW_BIAS_NEIGHBOR_DEGREE && g->zero_degree_target);

    uint64_t* d_scalars;   // [0] err flags, [1] n_seeds, [2] total, [3] frontier count ...
    CSAW_TRY(tmp.get(&d_scalars, 16));
    CSAW_CUDA(cudaMemsetAsync(d_scalars, 0, 16 * sizeof(uint64_t), s));
    uint32_t* d_err = (uint32_t*)d_scalars;
    uint64_t* d_nseeds = d_scalars + 1;
    CSAW_CUDA(cudaMemcpyAsync(d_nseeds, &n_seeds, sizeof(uint64_t), cudaMemcpyHostToDevice, s));

    void* scan_scr;
    CSAW_TRY(tmp.get((unsigned char**)&scan_scr, scan_scratch_bytes(0)));
    void* sort_scr;
    CSAW_TRY(tmp.get((unsigned char**)&sort_scr, sort_scratch_bytes(0)));

    // Layer-0 frontier: sorted unique (instance, seed) keys.
    std::vector<uint64_t*> F(depth, nullptr), FO(depth, nullptr);
    std::vector<uint64_t> fcount(depth, 0);
    {
        uint64_t *keys, *alt, *kpos;
        uint32_t* kept;
        const uint64_t ns = n_seeds ? n_seeds : 1;
        CSAW_TRY(tmp.get(&keys, ns));
        CSAW_TRY(tmp.get(&alt, ns));
        CSAW_TRY(tmp.get(&kept, ns));
        CSAW_TRY(tmp.get(&kpos, ns + 1));
        check_inst_off_kernel<<<grid_for(n_inst, 256, g->sm_count), 256, 0, s>>>(inst_off, n_inst, d_err);
        if (n_seeds)
            seed_keys_kernel<<<grid_for(n_seeds, 256, g->sm_count), 256, 0, s>>>(
                seeds, inst_off, n_inst, n_seeds, g->V, vbits, keys, d_err);
        uint64_t* sorted = keys;
        if (n_seeds) CSAW_TRY(radix_sort_u64(keys, alt, d_nseeds, n_seeds, kbits, g->sm_count, sort_scr, s, &sorted));
        Visited none;
        none.n = 0;
        unique_filter_kernel<<<grid_for(n_seeds, 256, g->sm_count), 256, 0, s>>>(sorted, d_nseeds, none, vbits, kept);
        uint64_t* d_fc = d_scalars + 3;
        CSAW_TRY(scan_u32(kept, kpos, d_nseeds, n_seeds, scan_scr, d_fc, s));
        uint64_t h[2];
        CSAW_CUDA(cudaMemcpyAsync(h, d_scalars, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        uint64_t hfc = 0;
        CSAW_CUDA(cudaMemcpyAsync(&hfc, d_fc, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        CSAW_CUDA(cudaStreamSynchronize(s));
        const uint32_t err = (uint32_t)h[0];
        if (err & 1u) return fail(CSAW_ERR_INVALID, "a seed is not a vertex of the graph");
        if (err & 2u) return fail(CSAW_ERR_INVALID, "inst_offsets must start at 0 and be non-decreasing");
        fcount[0] = hfc;
        CSAW_TRY(tmp.get(&F[0], hfc ? hfc : 1));
        CSAW_TRY(tmp.get(&FO[0], (uint64_t)n_inst + 1));
        scatter_kept_kernel<<<grid_for(n_seeds, 256, g->sm_count), 256, 0, s>>>(sorted, d_nseeds, kept, kpos, F[0]);
        inst_bounds_kernel<<<grid_for((uint64_t)n_inst + 1, 256, g->sm_count), 256, 0, s>>>(F[0], d_fc, n_inst, vbits, FO[0]);
        CSAW_CUDA(cudaGetLastError());
    }

    // Result arrays for offsets and sizes (device), copied to the host at the end.
    uint64_t *d_eoff, *d_fsize;
    CSAW_TRY(tmp.get(&d_eoff, (uint64_t)depth * n_inst + 1));
    CSAW_TRY(tmp.get(&d_fsize, (uint64_t)depth * n_inst + 1));
    R->src.assign(depth, nullptr);
    R->dst.assign(depth, nullptr);
    R->layer_edges.assign(depth, 0);
    uint64_t base = 0;
    const int sel_blocks = select_blocks(kind, g->sm_count);
    uint64_t* scratch_S = nullptr;
    uint32_t* scratch_bits = nullptr;
    if (g->max_degree > CTA_SMEM_DEG) {
        CSAW_TRY(tmp.get(&scratch_S, (uint64_t)sel_blocks * g->max_degree));
        CSAW_TRY(tmp.get(&scratch_bits, (uint64_t)sel_blocks * ((g->max_degree + 31) / 32)));
    }

    for (uint32_t l = 0; l < depth; ++l) {
        const uint64_t n = fcount[l];
        const uint32_t k = fanout[l];
        uint64_t* d_n = d_scalars + 4;   // entries of this layer
        CSAW_CUDA(cudaMemcpyAsync(d_n, &fcount[l], sizeof(uint64_t), cudaMemcpyHostToDevice, s));
        uint32_t *cnt, *wlist, *clist;
        uint64_t* pos;
        const uint64_t nn = n ? n : 1;
        CSAW_TRY(tmp.get(&cnt, nn));
        CSAW_TRY(tmp.get(&wlist, nn));
        CSAW_TRY(tmp.get(&clist, nn));
        CSAW_TRY(tmp.get(&pos, nn + 1));
        unsigned long long* d_items = (unsigned long long*)(d_scalars + 6);   // [6],[7] sizes, [8],[9] counters
        CSAW_CUDA(cudaMemsetAsync(d_items, 0, 4 * sizeof(uint64_t), s));
        CountParams cp;
        cp.off = g->off; cp.col = g->col; cp.w = g->w; cp.deg = g->deg;
        cp.fkeys = F[l]; cp.n_dev = (const unsigned long long*)d_n; cp.vmask = vmask; cp.k = k;
        cp.zero_bias = zero_bias; cp.cnt = cnt; cp.warp_list = wlist; cp.cta_list = clist;
        cp.n_items = d_items;
        if (n) {
            switch (kind) {
            case CSAW_BIAS_UNIFORM: CSAW_TRY(launch_count<CSAW_BIAS_UNIFORM>(cp, n, g->sm_count, s)); break;
            case CSAW_BIAS_EDGE_WEIGHT: CSAW_TRY(launch_count<CSAW_BIAS_EDGE_WEIGHT>(cp, n, g->sm_count, s)); break;
            default: CSAW_TRY(launch_count<CSAW_BIAS_NEIGHBOR_DEGREE>(cp, n, g->sm_count, s)); break;
            }
        }
        uint64_t* d_total = d_scalars + 5;
        CSAW_TRY(scan_u32(cnt, pos, d_n, n, scan_scr, d_total, s));
        uint64_t total = 0;
        CSAW_CUDA(cudaMemcpyAsync(&total, d_total, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        CSAW_CUDA(cudaStreamSynchronize(s));
        R->layer_edges[l] = total;
        void* ps = nullptr;
        void* pd = nullptr;
        CSAW_CUDA(cudaMalloc(&ps, (total ? total : 1) * sizeof(uint32_t)));
        R->src[l] = (uint32_t*)ps;
        CSAW_CUDA(cudaMalloc(&pd, (total ? total : 1) * sizeof(uint32_t)));
        R->dst[l] = (uint32_t*)pd;
        const bool last = l + 1 == depth;
        uint64_t *cand = nullptr, *cand_alt = nullptr;
        if (!last) {
            CSAW_TRY(tmp.get(&cand, total ? total : 1));
            CSAW_TRY(tmp.get(&cand_alt, total ? total : 1));
        }
        if (n) {
            SelParams sp;
            sp.off = g->off; sp.col = g->col; sp.w = g->w; sp.deg = g->deg;
            sp.fkeys = F[l]; sp.vbits = vbits; sp.vmask = vmask; sp.k = k; sp.layer = l;
            sp.k0 = (uint32_t)rng_seed; sp.k1 = (uint32_t)(rng_seed >> 32);
            sp.zero_bias = zero_bias; sp.pos = pos; sp.warp_list = wlist; sp.cta_list = clist;
            sp.n_items = d_items; sp.next = d_items + 2;
            sp.out_src = R->src[l]; sp.out_dst = R->dst[l]; sp.out_cand = cand;
            sp.scratch_S = scratch_S; sp.scratch_bits = scratch_bits; sp.scratch_stride = g->max_degree;
            switch (kind) {
            case CSAW_BIAS_UNIFORM: CSAW_TRY(launch_select<CSAW_BIAS_UNIFORM>(sp, sel_blocks, s)); break;
            case CSAW_BIAS_EDGE_WEIGHT: CSAW_TRY(launch_select<CSAW_BIAS_EDGE_WEIGHT>(sp, sel_blocks, s)); break;
            default: CSAW_TRY(launch_select<CSAW_BIAS_NEIGHBOR_DEGREE>(sp, sel_blocks, s)); break;
            }
        }
        layer_offsets_kernel<<<grid_for((uint64_t)n_inst + 1, 256, g->sm_count), 256, 0, s>>>(
            FO[l], pos, n_inst, base, d_eoff + (uint64_t)l * n_inst, d_fsize + (uint64_t)l * n_inst);
        CSAW_CUDA(cudaGetLastError());
        base += total;
        if (last) break;
        // Update: next frontier = sorted unique picks minus visited.
        uint64_t* sorted = cand;
        if (total) CSAW_TRY(radix_sort_u64(cand, cand_alt, d_total, total, kbits, g->sm_count, sort_scr, s, &sorted));
        uint32_t* kept;
        uint64_t* kpos;
        CSAW_TRY(tmp.get(&kept, total ? total : 1));
        CSAW_TRY(tmp.get(&kpos, (total ? total : 1) + 1));
        Visited vis;
        vis.n = (int)l + 1;
        for (uint32_t j = 0; j <= l; ++j) { vis.keys[j] = F[j]; vis.foff[j] = FO[j]; }
        unique_filter_kernel<<<grid_for(total, 256, g->sm_count), 256, 0, s>>>(sorted, d_total, vis, vbits, kept);
        uint64_t* d_fc = d_scalars + 10;
        CSAW_TRY(scan_u32(kept, kpos, d_total, total, scan_scr, d_fc, s));
        uint64_t hfc = 0;
        CSAW_CUDA(cudaMemcpyAsync(&hfc, d_fc, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        CSAW_CUDA(cudaStreamSynchronize(s));
        fcount[l + 1] = hfc;
        CSAW_TRY(tmp.get(&F[l + 1], hfc ? hfc : 1));
        CSAW_TRY(tmp.get(&FO[l + 1], (uint64_t)n_inst + 1));
        scatter_kept_kernel<<<grid_for(total, 256, g->sm_count), 256, 0, s>>>(sorted, d_total, kept, kpos, F[l + 1]);
        inst_bounds_kernel<<<grid_for((uint64_t)n_inst + 1, 256, g->sm_count), 256, 0, s>>>(F[l + 1], d_fc, n_inst, vbits, FO[l + 1]);
        CSAW_CUDA(cudaGetLastError());
    }
    R->n_edges = base;
    R->edge_offsets.assign((size_t)depth * n_inst + 1, 0);
    R->frontier_sizes.assign((size_t)depth * n_inst, 0);
    if (depth * (uint64_t)n_inst > 0) {
        CSAW_CUDA(cudaMemcpyAsync(R->edge_offsets.data(), d_eoff, sizeof(uint64_t) * ((size_t)depth * n_inst + 1),
                                  cudaMemcpyDeviceToHost, s));
        CSAW_CUDA(cudaMemcpyAsync(R->frontier_sizes.data(), d_fsize, sizeof(uint64_t) * (size_t)depth * n_inst,
                                  cudaMemcpyDeviceToHost, s));
    }
    CSAW_CUDA(cudaStreamSynchronize(s));
    R->edge_offsets[(size_t)depth * n_inst] = base;
    R->src_c.assign(R->src.begin(), R->src.end());
    R->dst_c.assign(R->dst.begin(), R->dst.end());
    return CSAW_OK;
}

}  // namespace csaw

using namespace csaw;

extern "C" csaw_status csaw_sample(csaw_graph* g, const uint32_t* seeds, const uint64_t* inst_offsets,
                                   uint32_t n_instances, uint32_t depth, const uint32_t* fanout,
                                   const csaw_bias* bias, uint64_t rng_seed, int mem_kind, void* stream,
                                   csaw_sample_result** out)
{
    clear_error();
    if (!out) return fail(CSAW_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!g) return fail(CSAW_ERR_INVALID, "graph is NULL");
    int kind;
    CSAW_TRY(check_bias(g, bias, false, &kind));
    if (depth < 1 || depth > CSAW_MAX_DEPTH) return fail(CSAW_ERR_INVALID, "depth must be 1..%u", CSAW_MAX_DEPTH);
    if (!fanout) return fail(CSAW_ERR_INVALID, "fanout is NULL");
    if (!inst_offsets) return fail(CSAW_ERR_INVALID, "inst_offsets is NULL");
    if (mem_kind != CSAW_MEM_HOST && mem_kind != CSAW_MEM_DEVICE)
        return fail(CSAW_ERR_INVALID, "bad mem_kind %d", mem_kind);
    if (n_instances == 0xFFFFFFFFu) return fail(CSAW_ERR_INVALID, "too many instances");
    cudaStream_t s = (cudaStream_t)stream;

    csaw_sample_result* R = new (std::nothrow) csaw_sample_result();
    if (!R) return fail(CSAW_ERR_NOMEM, "host allocation failed");
    R->depth = depth;
    R->n_instances = n_instances;
    cudaGetDevice(&R->device);

    uint64_t n_seeds = 0;
    const uint32_t* d_seeds = seeds;
    const uint64_t* d_io = inst_offsets;
    void* own_seeds = nullptr;
    void* own_io = nullptr;
    csaw_status st = CSAW_OK;
    if (mem_kind == CSAW_MEM_HOST) {
        if (inst_offsets[0] != 0) st = fail(CSAW_ERR_INVALID, "inst_offsets must start at 0");
        for (uint32_t i = 0; st == CSAW_OK && i < n_instances; ++i)
            if (inst_offsets[i + 1] < inst_offsets[i])
                st = fail(CSAW_ERR_INVALID, "inst_offsets must be non-decreasing");
        if (st == CSAW_OK) n_seeds = inst_offsets[n_instances];
        for (uint64_t j = 0; st == CSAW_OK && j < n_seeds; ++j)
            if (seeds[j] >= g->V) st = fail(CSAW_ERR_INVALID, "seed %llu out of range", (unsigned long long)j);
        if (st == CSAW_OK) st = dalloc(&own_io, sizeof(uint64_t) * ((size_t)n_instances + 1), s);
        if (st == CSAW_OK) st = dalloc(&own_seeds, sizeof(uint32_t) * (n_seeds ? n_seeds : 1), s);
        if (st == CSAW_OK) {
            cudaError_t e = cudaMemcpyAsync(own_io, inst_offsets, sizeof(uint64_t) * ((size_t)n_instances + 1),
                                            cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess && n_seeds)
                e = cudaMemcpyAsync(own_seeds, seeds, sizeof(uint32_t) * n_seeds, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) st = cuda_fail(e, "copy seeds");
        }
        d_seeds = (const uint32_t*)own_seeds;
        d_io = (const uint64_t*)own_io;
    } else {
        cudaError_t e = cudaMemcpyAsync(&n_seeds, inst_offsets + n_instances, sizeof(uint64_t),
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "read inst_offsets");
    }
    if (st == CSAW_OK && n_seeds >= 0xFFFFFFFFull) st = fail(CSAW_ERR_INVALID, "too many seeds");
    if (st == CSAW_OK && n_seeds > 0 && !seeds) st = fail(CSAW_ERR_INVALID, "seeds is NULL");
    if (st == CSAW_OK)
        st = run_sample(g, d_seeds, d_io, n_instances, n_seeds, depth, fanout, kind, rng_seed, s, R);
    dfree(own_seeds, s);
    dfree(own_io, s);
    if (st != CSAW_OK) {
        cudaStreamSynchronize(s);
        delete R;
        return st;
    }
    *out = R;
    return CSAW_OK;
}

extern "C" csaw_status csaw_sample_get_view(csaw_sample_result* r, csaw_sample_view* view)
{
    clear_error();
    if (!r || !view) return fail(CSAW_ERR_INVALID, "NULL argument");
    view->depth = r->depth;
    view->n_instances = r->n_instances;
    view->n_edges = r->n_edges;
    view->edge_offsets = r->edge_offsets.data();
    view->frontier_sizes = r->frontier_sizes.data();
    view->src = r->src_c.data();
    view->dst = r->dst_c.data();
    return CSAW_OK;
}

extern "C" csaw_status csaw_sample_copy_edges(csaw_sample_result* r, uint32_t* src, uint32_t* dst)
{
    clear_error();
    if (!r) return fail(CSAW_ERR_INVALID, "result is NULL");
    if (r->n_edges && (!src || !dst)) return fail(CSAW_ERR_INVALID, "NULL output");
    uint64_t at = 0;
    for (uint32_t l = 0; l < r->depth; ++l) {
        const uint64_t n = r->layer_edges[l];
        if (n) {
            CSAW_CUDA(cudaMemcpy(src + at, r->src[l], n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
            CSAW_CUDA(cudaMemcpy(dst + at, r->dst[l], n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
        }
        at += n;
    }
    return CSAW_OK;
}

extern "C" void csaw_result_free(void* result)
{
    delete (csaw_sample_result*)result;
}

// ---------------------------------------------------------------------------
// One selection layer without any device allocation.
//
// Some callers cannot allocate device memory while they run this library:
// code executing inside another framework's memory budget, allocator-less
// embedded runtimes, or a host thread that must not contend on the device
// allocator.  For them csaw_select_noalloc runs one layer of selection (the
// count, scan and select kernels above) with every temporary placed in the
// fixed device array below.  The array is a file-scope __device__ variable:
// every GPU that loads this library holds its CSAW_NOALLOC_SCRATCH_BYTES until
// the process exits.  All calls share it, so calls that overlap on the GPU
// (different streams, or other host threads) race on it; the counters that
// must start at zero are cleared by every call.

namespace csaw {

static __device__ __align__(256) unsigned char g_noalloc_scratch[CSAW_NOALLOC_SCRATCH_BYTES];

constexpr size_t NA_HEAD = 256;   // counters
constexpr size_t NA_KEYS = NA_HEAD;
constexpr size_t NA_CNT = NA_KEYS + sizeof(uint64_t) * CSAW_NOALLOC_MAX_ITEMS;
constexpr size_t NA_WLIST = NA_CNT + sizeof(uint32_t) * CSAW_NOALLOC_MAX_ITEMS;
constexpr size_t NA_CLIST = NA_WLIST + sizeof(uint32_t) * CSAW_NOALLOC_MAX_ITEMS;
constexpr size_t NA_BSUM = NA_CLIST + sizeof(uint32_t) * CSAW_NOALLOC_MAX_ITEMS;
constexpr size_t NA_HUB = (NA_BSUM + 8 * 1040 + 255) / 256 * 256;
static_assert(NA_HUB < CSAW_NOALLOC_SCRATCH_BYTES, "scratch layout does not fit");

// Host-side device addresses of the array, one per device, looked up on the
// first call made with that device current.
static std::mutex g_na_mutex;
static void* g_na_ptr[256];

static csaw_status noalloc_scratch(int device, unsigned char** out)
{
    if (device < 0 || device >= 256) return fail(CSAW_ERR_INVALID, "device ordinal %d", device);
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_na_ptr[device] = p;
    }
    *out = (unsigned char*)g_na_ptr[device];
    return CSAW_OK;
}

// keys[e] = instances[e] << vbits | vertices[e]; flags any vertex >= V.
__global__ void noalloc_keys_kernel(const uint32_t* __restrict__ vertices,
                                    const uint32_t* __restrict__ instances, uint32_t n, uint32_t V,
                                    uint32_t vbits, uint64_t* __restrict__ keys, uint32_t* __restrict__ err)
{
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const uint32_t v = vertices[e];
        if (v >= V) atomicOr(err, 1u);
        keys[e] = ((uint64_t)instances[e] << vbits) | (v < V ? v : 0u);
    }
}

}  // namespace csaw

extern "C" csaw_status csaw_select_noalloc(csaw_graph* g, const uint32_t* vertices,
                                           const uint32_t* instances, uint32_t n, uint32_t k,
                                           uint32_t layer, const csaw_bias* bias, uint64_t rng_seed,
                                           uint32_t* out_src, uint32_t* out_dst, uint64_t capacity,
                                           uint64_t* out_offsets, void* stream)
{
    clear_error();
    if (!g) return fail(CSAW_ERR_INVALID, "graph is NULL");
    int kind;
    CSAW_TRY(check_bias(g, bias, false, &kind));
    if (n > CSAW_NOALLOC_MAX_ITEMS)
        return fail(CSAW_ERR_INVALID, "csaw_select_noalloc takes at most %u vertices per call, got %u",
                    CSAW_NOALLOC_MAX_ITEMS, n);
    if (!out_offsets) return fail(CSAW_ERR_INVALID, "out_offsets is NULL");
    if (n > 0 && (!vertices || !instances || !out_src || !out_dst))
        return fail(CSAW_ERR_INVALID, "NULL vertex, instance or output array");
    if (k == 0) return fail(CSAW_ERR_INVALID, "k must be at least 1");
    const uint64_t per = k < g->max_degree ? k : g->max_degree;
    if (capacity < (uint64_t)n * per)
        return fail(CSAW_ERR_INVALID, "capacity %llu is below n * min(k, max degree) = %llu",
                    (unsigned long long)capacity, (unsigned long long)((uint64_t)n * per));
    int device = 0;
    CSAW_CUDA(cudaGetDevice(&device));
    int sel_blocks = select_blocks(kind, g->sm_count);
    if (g->max_degree > CTA_SMEM_DEG) {
        const uint64_t slot = (uint64_t)g->max_degree * 8 + ((uint64_t)g->max_degree + 31) / 32 * 4;
        const uint64_t slots = (CSAW_NOALLOC_SCRATCH_BYTES - NA_HUB) / slot;
        if (slots == 0)
            return fail(CSAW_ERR_INVALID, "graph max degree %u needs %llu scratch bytes per CTA; the "
                        "no-allocation scratch holds %llu", g->max_degree, (unsigned long long)slot,
                        (unsigned long long)(CSAW_NOALLOC_SCRATCH_BYTES - NA_HUB));
        if ((uint64_t)sel_blocks > slots) sel_blocks = (int)slots;
    }
    unsigned char* base;
    CSAW_TRY(noalloc_scratch(device, &base));
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t* head = (uint64_t*)base;              // [0] n, [1] total, [2..5] items/counters, [6] err
    uint64_t* d_n = head;
    uint64_t* d_total = head + 1;
    unsigned long long* d_items = (unsigned long long*)(head + 2);
    uint32_t* d_err = (uint32_t*)(head + 6);
    uint64_t* keys = (uint64_t*)(base + NA_KEYS);
    uint32_t* cnt = (uint32_t*)(base + NA_CNT);
    uint32_t* wlist = (uint32_t*)(base + NA_WLIST);
    uint32_t* clist = (uint32_t*)(base + NA_CLIST);
    void* bsum = base + NA_BSUM;
    unsigned char* hub = base + NA_HUB;

    const uint64_t n64 = n;
    CSAW_CUDA(cudaMemsetAsync(head, 0, NA_HEAD, s));
    CSAW_CUDA(cudaMemcpyAsync(d_n, &n64, sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    const int vbits = bits_for(g->V - 1) > 0 ? bits_for(g->V - 1) : 1;
    const uint64_t vmask = (1ull << vbits) - 1;
    if (n) {
        noalloc_keys_kernel<<<grid_for(n, 256, g->sm_count), 256, 0, s>>>(vertices, instances, n, g->V,
                                                                          vbits, keys, d_err);
        CSAW_CUDA(cudaGetLastError());
        uint32_t h_err = 0;
        CSAW_CUDA(cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CSAW_CUDA(cudaStreamSynchronize(s));
        if (h_err) return fail(CSAW_ERR_INVALID, "a vertex is not in the graph");
    }
    const bool zero_bias = (kind == CSAW_BIAS_EDGE_WEIGHT && g->min_weight == 0) ||
                           (kind == CSAW_BIAS_NEIGHBOR_DEGREE && g->zero_degree_target);
    CountParams cp;
    cp.off = g->off; cp.col = g->col; cp.w = g->w; cp.deg = g->deg;
    cp.fkeys = keys; cp.n_dev = (const unsigned long long*)d_n; cp.vmask = vmask; cp.k = k;
    cp.zero_bias = zero_bias; cp.cnt = cnt; cp.warp_list = wlist; cp.cta_list = clist;
    cp.n_items = d_items;
    if (n) {
        switch (kind) {
        case CSAW_BIAS_UNIFORM: CSAW_TRY(launch_count<CSAW_BIAS_UNIFORM>(cp, n, g->sm_count, s)); break;
        case CSAW_BIAS_EDGE_WEIGHT: CSAW_TRY(launch_count<CSAW_BIAS_EDGE_WEIGHT>(cp, n, g->sm_count, s)); break;
        default: CSAW_TRY(launch_count<CSAW_BIAS_NEIGHBOR_DEGREE>(cp, n, g->sm_count, s)); break;
        }
    }
    CSAW_TRY(scan_u32(cnt, out_offsets, d_n, n, bsum, d_total, s));
    if (n) {
        SelParams sp;
        sp.off = g->off; sp.col = g->col; sp.w = g->w; sp.deg = g->deg;
        sp.fkeys = keys; sp.vbits = vbits; sp.vmask = vmask; sp.k = k; sp.layer = layer;
        sp.k0 = (uint32_t)rng_seed; sp.k1 = (uint32_t)(rng_seed >> 32);
        sp.zero_bias = zero_bias; sp.pos = out_offsets; sp.warp_list = wlist; sp.cta_list = clist;
        sp.n_items = d_items; sp.next = d_items + 2;
        sp.out_src = out_src; sp.out_dst = out_dst; sp.out_cand = nullptr;
        sp.scratch_S = (uint64_t*)hub;
        sp.scratch_bits = (uint32_t*)(hub + (size_t)sel_blocks * g->max_degree * 8);
        sp.scratch_stride = g->max_degree;
        switch (kind) {
        case CSAW_BIAS_UNIFORM: CSAW_TRY(launch_select<CSAW_BIAS_UNIFORM>(sp, sel_blocks, s)); break;
        case CSAW_BIAS_EDGE_WEIGHT: CSAW_TRY(launch_select<CSAW_BIAS_EDGE_WEIGHT>(sp, sel_blocks, s)); break;
        default: CSAW_TRY(launch_select<CSAW_BIAS_NEIGHBOR_DEGREE>(sp, sel_blocks, s)); break;
        }
    }
    return CSAW_OK;
}
