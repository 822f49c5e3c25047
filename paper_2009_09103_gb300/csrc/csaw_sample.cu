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
#include <algorithm>
#include <atomic>
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
// Warp items alone use only the warps' slots: a launch that can hold no CTA
// item takes this much, and more blocks fit an SM.
constexpr size_t SEL_WARP_SMEM = (size_t)(SEL_THREADS / 32) * WARP_SLOT;
constexpr uint32_t PICK_MAX = 256;         // picks a cached-array warp item may hold

static_assert(SEL_WARPS * WARP_SLOT <= SEL_DYN_SMEM, "warp slots reuse the CTA region");

// Selection counters, compiled in with -DCSAW_STATS (the library built for
// the attempts-per-pick measurement; the default build has none):
// [0] draws consumed (a selection consumes attempts up to the one that gave
// its last pick), [1] picks of the selections that drew, [2] draws evaluated
// (whole warp rounds of 32, plus updated-sampling draws), [3] picks by
// updated sampling, [4] warp items, [5] CTA items, [6] hub items.
#ifdef CSAW_STATS
__device__ unsigned long long g_sel_stats[8];
#define CSAW_STAT_ADD(i, v) atomicAdd(&g_sel_stats[i], (unsigned long long)(v))
#else
#define CSAW_STAT_ADD(i, v) ((void)0)
#endif

// Position of the n-th set bit of m (n >= 1, m has at least n set bits).
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t n)
{
    for (uint32_t i = 1; i < n; ++i) m &= m - 1;
    return (uint32_t)(__ffs(m) - 1);
}

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
    const uint32_t* key_dev;              // if set, the Philox key {k0, k1} is read here
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
    const uint64_t* __restrict__ cdf;     // cached cumulative array (select_cdf_kernel)
    bool skip_warp_items;                 // warp items are served by select_cdf_kernel
    uint32_t attempt_cap;                 // repeated-sampling attempts before updated sampling
    // shared hub arrays of the layer (select_cdf_kernel over hub items):
    // item q is frontier entry item_e[q] of distinct hub item_h[q], whose
    // prefix sums are hubS[hub_off[h] ..]; null outside that mode
    const uint32_t* __restrict__ item_e = nullptr;
    const uint32_t* __restrict__ item_h = nullptr;
    const uint64_t* __restrict__ hub_off = nullptr;
    const uint64_t* __restrict__ hubS = nullptr;
    uint64_t hubS_cap = 0;                // entries of hubS
    CdfView cv;                           // the cached array and its search aids (cv.cdf == cdf)
    uint32_t* err = nullptr;              // error flags (8: a hub range beyond hubS_cap)
    // instances of several requests in one run (null: one request): per
    // instance its Philox key, its index within its request (the draw
    // counter's instance word) and its picks per vertex at this layer
    const uint32_t* __restrict__ inst_key = nullptr;   // [2 * n_inst]
    const uint32_t* __restrict__ inst_id = nullptr;    // [n_inst]
    const uint32_t* __restrict__ inst_k = nullptr;     // [n_inst]
};

// The draw key of one frontier entry: Philox key words and the instance word
// of the counter.
struct DrawKey {
    uint32_t k0, k1, id;
};

__device__ __forceinline__ DrawKey draw_key(const SelParams& p, uint32_t inst)
{
    if (p.inst_key) return {__ldg(p.inst_key + 2 * inst), __ldg(p.inst_key + 2 * inst + 1), __ldg(p.inst_id + inst)};
    return {p.k0, p.k1, inst};
}

__device__ __forceinline__ uint32_t picks_of(const SelParams& p, uint32_t inst)
{
    return p.inst_k ? __ldg(p.inst_k + inst) : p.k;
}

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
    const DrawKey dk = draw_key(p, inst);
    const uint32_t lt = lanemask_lt();
    uint32_t have = 0;
    uint32_t a0 = 0;
    uint32_t used = 0, rounds = 0;   // counters (CSAW_STATS)
    (void)used;
    (void)rounds;
    while (have < cnt && a0 < p.attempt_cap) {
        const bool live = a0 + lane < p.attempt_cap;   // the last round may be partial
        const uint64_t r = philox_draw(dk.k0, dk.k1, a0 + lane, v, p.layer, dk.id);
        const uint32_t i = live ? upper_bound_S(S, d, scale_draw(r, T)) : 0xFFFFFFFFu;
        const bool chosen = live && ((bits[i >> 5] >> (i & 31)) & 1u);
        const uint32_t peers = __match_any_sync(CSAW_FULL_MASK, i);
        const bool fresh = live && !chosen && lane == __ffs(peers) - 1;
        const uint32_t bal = __ballot_sync(CSAW_FULL_MASK, fresh);
        const uint32_t rank = __popc(bal & lt);
        const uint32_t need = cnt - have;
        if (fresh && rank < need) {
            emit(p, q0 + have + rank, v, inst, __ldg(p.col + beg + i));
            atomicOr(bits + (i >> 5), 1u << (i & 31));
        }
#ifdef CSAW_STATS
        used = (uint32_t)__popc(bal) >= need ? a0 + nth_set_bit(bal, need) + 1 : min(a0 + 32, p.attempt_cap);
        ++rounds;
#endif
        have += min((uint32_t)__popc(bal), need);
        a0 += 32;
        __syncwarp();
    }
    if (have >= cnt) {
        if (lane == 0) {
            CSAW_STAT_ADD(0, used);
            CSAW_STAT_ADD(1, cnt);
            CSAW_STAT_ADD(2, 32u * rounds);
        }
        return;
    }
    const uint32_t have0 = have;
    (void)have0;
    // Updated sampling for the remaining picks (attempts attempt_cap, ...).
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
        for (uint32_t a = p.attempt_cap; have < cnt; ++a) {
            const uint64_t r = philox_draw(dk.k0, dk.k1, a, v, p.layer, dk.id);
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
        // every repeated attempt was consumed, then one draw per remaining pick
        CSAW_STAT_ADD(0, p.attempt_cap + (cnt - have0));
        CSAW_STAT_ADD(1, cnt);
        CSAW_STAT_ADD(2, 32u * rounds + (cnt - have0));
        CSAW_STAT_ADD(3, cnt - have0);
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
    if (npos <= picks_of(p, inst)) {
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
__global__ void __launch_bounds__(SEL_THREADS, 6) select_kernel(SelParams p)
{
    if (p.key_dev) {
        p.k0 = p.key_dev[0];
        p.k1 = p.key_dev[1];
    }
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
    const unsigned long long n_warp = p.skip_warp_items ? 0ull : p.n_items[0];
    while (true) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(p.next, 1ull);
        it = __shfl_sync(CSAW_FULL_MASK, it, 0);
        if (it >= n_warp) break;
        warp_item<KIND>(p, p.warp_list[it], sS, sBits, lane);
    }
}

// ---------------------------------------------------------------------------
// Selection over a cached cumulative array (static biases): one warp per
// frontier vertex of any degree.  T is the row's last prefix sum; each of the
// 32 attempts of a round binary-searches the row's prefix sums in global
// memory (uniform bias: the pick is x itself), so a hub costs O(log d) per
// attempt instead of a pass over its row.  Picks so far are kept in a
// per-warp list in shared memory (at most PICK_MAX); collision resolution and
// the updated-sampling fallback are those of draw_picks.

__device__ __forceinline__ uint64_t cdf_at(const uint64_t* __restrict__ row, bool implicit, uint32_t i)
{
    return implicit ? (uint64_t)i + 1 : __ldg(row + i);
}

// CACHED: rows of the graph's cumulative array, searched through its
// summaries (cdf_search); otherwise bisected directly (shared hub arrays).
// G: lanes per item -- 32, or 16 (two items per warp, rounds of 16
// attempts; for layers whose fanout is at most 16, where a hub row's first
// round nearly always holds the picks).  Attempts are taken in the same
// order either way, so the picks do not depend on G.
template <bool IMPLICIT, bool CACHED = false, int G = 32>
__global__ void __launch_bounds__(SEL_THREADS, CACHED ? 6 : 8) select_cdf_kernel(SelParams p)
{
    static_assert(G == 32 || G == 16, "16 or 32 lanes per item");
    __shared__ uint32_t s_picks[SEL_WARPS][PICK_MAX];
    if (p.key_dev) {
        p.k0 = p.key_dev[0];
        p.k1 = p.key_dev[1];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gb = lane & ~(G - 1), gl = lane & (G - 1);   // the group's first lane; this lane in it
    const uint32_t gmask = G == 32 ? CSAW_FULL_MASK : (0xFFFFu << gb);
    uint32_t* picks = s_picks[wid] + gb * (PICK_MAX / 32);     // PICK_MAX * G / 32 entries per group
    const uint32_t lt = (1u << gl) - 1u;                   // group lanes before this one
    const bool hub = p.item_e != nullptr;   // hub items (vertex order): shared array or cached one
    const unsigned long long n_warp = hub ? p.n_items[2] : p.n_items[0];
    unsigned long long* counter = hub ? p.next + 2 : p.next;
    while (true) {
        unsigned long long it = 0;
        if (gl == 0) it = atomicAdd(counter, 1ull);
        it = __shfl_sync(gmask, it, gb);
        if (it >= n_warp) break;
        const uint32_t e = hub ? p.item_e[it] : p.warp_list[it];
        const uint64_t key = p.fkeys[e];
        const uint32_t v = (uint32_t)(key & p.vmask);
        const uint32_t inst = (uint32_t)(key >> p.vbits);
        const uint64_t beg = __ldg(p.off + v);
        const uint32_t d = (uint32_t)(__ldg(p.off + v + 1) - beg);
        const uint64_t q0 = p.pos[e];
        const uint32_t cnt = (uint32_t)(p.pos[e + 1] - q0);
        if (cnt >= d) {
            // every neighbour (all biases are positive here), CSR order
            for (uint32_t j = gl; j < d; j += G) emit(p, q0 + j, v, inst, __ldg(p.col + beg + j));
            continue;
        }
        if (hub && p.hubS && p.hub_off[p.item_h[it]] + d > p.hubS_cap) {
            if (gl == 0) atomicOr(p.err, 8u);   // never happens when the scratch is sized right
            continue;
        }
        const uint64_t* row = hub && p.hubS ? p.hubS + p.hub_off[p.item_h[it]] : p.cdf ? p.cdf + beg : nullptr;
        const DrawKey dk = draw_key(p, inst);
        const uint64_t T = cdf_at(row, IMPLICIT, d - 1);
        uint32_t have = 0, a0 = 0;
        uint32_t used = 0, rounds = 0;   // counters (CSAW_STATS)
        (void)used;
        (void)rounds;
        while (have < cnt && a0 < p.attempt_cap) {
            const bool live = a0 + gl < p.attempt_cap;   // the last round may be partial
            const uint64_t x = scale_draw(philox_draw(dk.k0, dk.k1, a0 + gl, v, p.layer, dk.id), T);
            uint32_t i = 0xFFFFFFFFu;
            if (!live) {
            } else if (IMPLICIT) {
                i = (uint32_t)x;
            } else if (CACHED) {
                i = (uint32_t)(cdf_search(p.cv, beg, beg + d, x) - beg);   // the cached array
            } else {
                uint32_t lo = 0, hi = d - 1;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (__ldg(row + mid) > x) hi = mid; else lo = mid + 1;
                }
                i = lo;
            }
            bool chosen = false;
            for (uint32_t j = 0; j < have; ++j) chosen |= picks[j] == i;
            const uint32_t peers = __match_any_sync(gmask, i);
            const bool fresh = live && !chosen && lane == __ffs(peers) - 1;
            const uint32_t bal = (__ballot_sync(gmask, fresh) & gmask) >> gb;   // the group's lanes, from bit 0
            const uint32_t rank = __popc(bal & lt);
            const uint32_t need = cnt - have;
            if (fresh && rank < need) {
                picks[have + rank] = i;
                emit(p, q0 + have + rank, v, inst, __ldg(p.col + beg + i));
            }
#ifdef CSAW_STATS
            used = (uint32_t)__popc(bal) >= need ? a0 + nth_set_bit(bal, need) + 1 : min(a0 + G, p.attempt_cap);
            ++rounds;
#endif
            have += min((uint32_t)__popc(bal), need);
            a0 += G;
            __syncwarp(gmask);
        }
        if (gl == 0) {
            // draws consumed: to the last pick's attempt, or every repeated
            // attempt and then one per updated-sampling pick
            const uint32_t f = cnt - have;
            CSAW_STAT_ADD(0, f ? p.attempt_cap + f : used);
            CSAW_STAT_ADD(1, cnt);
            CSAW_STAT_ADD(2, (uint32_t)G * rounds + f);
            CSAW_STAT_ADD(3, f);
        }
        if (have < cnt && gl == 0) {
            // Updated sampling (attempts attempt_cap, ...): picks sorted
            // ascending, the draw scaled to the unpicked total and moved past
            // every picked interval that starts at or below it.
            for (uint32_t a = 1; a < have; ++a) {
                const uint32_t t = picks[a];
                uint32_t b = a;
                while (b > 0 && picks[b - 1] > t) { picks[b] = picks[b - 1]; --b; }
                picks[b] = t;
            }
            uint64_t R = 0;
            for (uint32_t j = 0; j < have; ++j) {
                const uint32_t q = picks[j];
                R += cdf_at(row, IMPLICIT, q) - (q ? cdf_at(row, IMPLICIT, q - 1) : 0);
            }
            for (uint32_t a = p.attempt_cap; have < cnt; ++a) {
                uint64_t x = scale_draw(philox_draw(dk.k0, dk.k1, a, v, p.layer, dk.id), T - R);
                for (uint32_t j = 0; j < have; ++j) {
                    const uint32_t q = picks[j];
                    const uint64_t start = q ? cdf_at(row, IMPLICIT, q - 1) : 0;
                    if (x >= start) x += cdf_at(row, IMPLICIT, q) - start;
                    else break;
                }
                uint32_t lo = 0, hi = d - 1;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (cdf_at(row, IMPLICIT, mid) > x) hi = mid; else lo = mid + 1;
                }
                const uint32_t i = lo;
                uint32_t b = have;
                while (b > 0 && picks[b - 1] > i) { picks[b] = picks[b - 1]; --b; }
                picks[b] = i;
                R += cdf_at(row, IMPLICIT, i) - (i ? cdf_at(row, IMPLICIT, i - 1) : 0);
                emit(p, q0 + have, v, inst, __ldg(p.col + beg + i));
                ++have;
            }
        }
        __syncwarp(gmask);
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
    uint32_t theta_w;              // warp items: degree <= theta_w (<= WARP_MAX_DEG), or take-all
    bool cached;                   // cached cumulative array: warp items up to PICK_MAX picks
    bool zero_bias;
    uint32_t* __restrict__ cnt;
    uint32_t* __restrict__ warp_list;
    uint32_t* __restrict__ cta_list;
    unsigned long long* n_items;   // [0] warp, [1] CTA, [2] hub
    // hub items (degree above theta_w, at most PICK_MAX picks) when the layer
    // shares one cumulative array per distinct hub; null: they are CTA items
    uint32_t* __restrict__ hub_list = nullptr;
    // picks per vertex of each instance at this layer (null: k for all)
    const uint32_t* __restrict__ inst_k = nullptr;
    uint32_t vbits = 0;
    // only entries whose vertex is in [v_lo, v_hi) go to the lists (a graph
    // partition that is loaded); write_cnt: store every entry's count
    uint32_t v_lo = 0, v_hi = 0xFFFFFFFFu;
    bool write_cnt = true;
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
        const uint32_t k = (p.inst_k && e < n) ? __ldg(p.inst_k + (uint32_t)(p.fkeys[e] >> p.vbits)) : p.k;
        const uint32_t c = min(k, npos);
        const bool take_all = npos <= k;
        const bool listed = e < n && c > 0 && v >= p.v_lo && v < p.v_hi;
        const bool to_warp = listed && (take_all || (p.cached && !p.hub_list ? c <= PICK_MAX : d <= p.theta_w));
        const bool to_hub = listed && !to_warp && p.hub_list != nullptr && c <= PICK_MAX;
        const bool to_cta = listed && !to_warp && !to_hub;
        if (e < n && p.write_cnt) p.cnt[e] = c;
        // warp-aggregated appends
        const uint32_t bw = __ballot_sync(CSAW_FULL_MASK, to_warp);
        const uint32_t bc = __ballot_sync(CSAW_FULL_MASK, to_cta);
        const uint32_t bh = __ballot_sync(CSAW_FULL_MASK, to_hub);
        unsigned long long basew = 0, basec = 0, baseh = 0;
        if (lane == 0) {
            if (bw) basew = atomicAdd(p.n_items, (unsigned long long)__popc(bw));
            if (bc) basec = atomicAdd(p.n_items + 1, (unsigned long long)__popc(bc));
            if (bh) baseh = atomicAdd(p.n_items + 2, (unsigned long long)__popc(bh));
            CSAW_STAT_ADD(4, __popc(bw));
            CSAW_STAT_ADD(5, __popc(bc));
            CSAW_STAT_ADD(6, __popc(bh));
        }
        basew = __shfl_sync(CSAW_FULL_MASK, basew, 0);
        basec = __shfl_sync(CSAW_FULL_MASK, basec, 0);
        baseh = __shfl_sync(CSAW_FULL_MASK, baseh, 0);
        const uint32_t lt = lanemask_lt();
        if (to_warp) p.warp_list[basew + __popc(bw & lt)] = (uint32_t)e;
        if (to_cta) p.cta_list[basec + __popc(bc & lt)] = (uint32_t)e;
        if (to_hub) p.hub_list[baseh + __popc(bh & lt)] = (uint32_t)e;
    }
}

// ---------------------------------------------------------------------------
// Shared hub arrays.  With a static bias the cumulative array of a vertex is
// the same for every instance (the draws differ, the biases do not), and
// under neighbour-degree bias the same hubs recur in the frontiers of
// thousands of instances.  So the layer's hub items (degree above theta_w)
// are grouped by vertex: the distinct hub vertices H[h] get consecutive
// ranges hubS[hub_off[h] .. hub_off[h] + d) of one scratch array, each
// vertex's inclusive prefix sums are built there once, and every (instance,
// hub) item draws from them by binary search (select_cdf_kernel in hub
// mode).  Same prefix sums, same draws: the picks are unchanged.

// keys[j] = e << vshift | v for hub item j (entry e at vertex v), vshift =
// the vertex bits rounded up to whole bytes: the radix sort orders whole
// bytes, so the sorted low vshift bits hold the vertex alone.  Sorted stably,
// the items of one vertex end up adjacent.
__global__ void hub_keys_kernel(const uint32_t* __restrict__ hub_list, const unsigned long long* n_dev,
                                const uint64_t* __restrict__ fkeys, uint64_t vmask, uint32_t vshift,
                                uint64_t* __restrict__ keys)
{
    const uint64_t n = *n_dev;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t e = hub_list[j];
        keys[j] = ((uint64_t)e << vshift) | (fkeys[e] & vmask);
    }
}

// flag[q] = 1 where a new vertex starts in the sorted keys.
__global__ void hub_flag_kernel(const uint64_t* __restrict__ sorted, const unsigned long long* n_dev,
                                uint64_t vmask, uint32_t* __restrict__ flag)
{
    const uint64_t n = *n_dev;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (uint64_t)gridDim.x * blockDim.x)
        flag[q] = (q == 0 || ((sorted[q] ^ sorted[q - 1]) & vmask) != 0) ? 1u : 0u;
}

// item_e[q] = the entry of sorted key q (cached arrays: vertex order only).
__global__ void hub_order_kernel(const uint64_t* __restrict__ sorted, const unsigned long long* n_dev,
                                 uint32_t vshift, uint32_t* __restrict__ item_e)
{
    const uint64_t n = *n_dev;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (uint64_t)gridDim.x * blockDim.x)
        item_e[q] = (uint32_t)(sorted[q] >> vshift);
}

constexpr uint32_t HUB_WARP_DEG = 2048;   // hubs up to this degree: one warp builds each

// Item q: its entry and its hub index (hpos = exclusive scan of flag); the
// first item of each vertex records the distinct hub and its degree, and
// lists the hub for a whole CTA when it is above HUB_WARP_DEG.
__global__ void hub_items_kernel(const uint64_t* __restrict__ sorted, const unsigned long long* n_dev,
                                 const uint32_t* __restrict__ flag, const uint64_t* __restrict__ hpos,
                                 uint64_t vmask, uint32_t vshift, const uint64_t* __restrict__ off,
                                 uint32_t* __restrict__ item_e, uint32_t* __restrict__ item_h,
                                 uint32_t* __restrict__ H, uint32_t* __restrict__ dh,
                                 uint32_t* __restrict__ big_list, unsigned long long* n_big)
{
    const uint64_t n = *n_dev;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t key = sorted[q];
        const uint32_t v = (uint32_t)(key & vmask);
        const uint32_t h = (uint32_t)(hpos[q] + flag[q] - 1);
        item_e[q] = (uint32_t)(key >> vshift);
        item_h[q] = h;
        if (flag[q]) {
            const uint32_t d = (uint32_t)(__ldg(off + v + 1) - __ldg(off + v));
            H[h] = v;
            dh[h] = d;
            if (d > HUB_WARP_DEG) big_list[atomicAdd(n_big, 1ull)] = h;
        }
    }
}

struct HubBuildParams {
    const uint64_t* __restrict__ off;
    const uint32_t* __restrict__ col;
    const uint32_t* __restrict__ w;
    const uint32_t* __restrict__ deg;
    const uint32_t* __restrict__ H;
    const uint32_t* __restrict__ dh;
    const uint64_t* __restrict__ hub_off;
    const unsigned long long* nh;    // distinct hubs
    const uint32_t* __restrict__ big_list;
    const unsigned long long* n_big; // hubs above HUB_WARP_DEG
    unsigned long long* next;        // [0] CTA counter, [1] warp counter
    uint64_t* __restrict__ S;
    uint64_t S_cap;                  // entries of S
    uint32_t* err;                   // flag 8: a hub range beyond S_cap (skipped)
};

// Bias of edge e (static kinds).
template <int KIND>
__device__ __forceinline__ uint32_t hub_bias(const HubBuildParams& p, uint64_t e)
{
    if constexpr (KIND == CSAW_BIAS_EDGE_WEIGHT) return __ldg(p.w + e);
    else return __ldg(p.deg + __ldg(p.col + e));
}

// Inclusive prefix sums of the biases of row [beg, beg + d) into out, by one
// warp: rounds of 256 neighbours, eight per lane in lane-interleaved tiles.
template <int KIND>
__device__ void hub_row_scan_warp(const HubBuildParams& p, uint64_t beg, uint32_t d, uint64_t* out, int lane)
{
    uint64_t carry = 0;
    for (uint32_t base = 0; base < d; base += 256) {
        uint32_t b[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const uint32_t j = base + 32u * t + lane;
            b[t] = j < d ? hub_bias<KIND>(p, beg + j) : 0u;
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const uint64_t incl = warp_inclusive_scan_u64(b[t], lane) + carry;
            const uint32_t j = base + 32u * t + lane;
            if (j < d) out[j] = incl;
            carry = __shfl_sync(CSAW_FULL_MASK, incl, 31);
        }
    }
}

// One kernel for all distinct hubs of the layer: CTAs first take the hubs
// above HUB_WARP_DEG from their list (eight warps scan 2048-neighbour tiles,
// segment offsets added in warp order, as in cta_item), then every warp
// takes the smaller hubs one at a time.  Work is claimed from two counters.
template <int KIND>
__global__ void __launch_bounds__(SEL_THREADS, 8) hub_cdf_kernel(HubBuildParams p)
{
    __shared__ uint64_t s_wsum[SEL_WARPS];
    __shared__ unsigned long long s_item;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long nh = *p.nh, n_big = *p.n_big;
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(p.next, 1ull);
        __syncthreads();
        const unsigned long long it = s_item;
        __syncthreads();
        if (it >= n_big) break;
        const uint32_t h = p.big_list[it];
        const uint32_t d = p.dh[h];
        if (p.hub_off[h] + d > p.S_cap) {
            if (threadIdx.x == 0) atomicOr(p.err, 8u);
            continue;
        }
        const uint64_t beg = __ldg(p.off + p.H[h]);
        uint64_t* out = p.S + p.hub_off[h];
        uint64_t carry = 0;
        for (uint32_t base = 0; base < d; base += SEL_WARPS * 256u) {
            const uint32_t seg = base + (uint32_t)wid * 256u;
            uint32_t b[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const uint32_t j = seg + 32u * t + lane;
                b[t] = j < d ? hub_bias<KIND>(p, beg + j) : 0u;
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
                if (j < d) out[j] = offw + incl[t];
            }
            carry += tile;
            __syncthreads();
        }
    }
    // small hubs: one warp each
    while (true) {
        unsigned long long h = 0;
        if (lane == 0) h = atomicAdd(p.next + 1, 1ull);
        h = __shfl_sync(CSAW_FULL_MASK, h, 0);
        if (h >= nh) break;
        const uint32_t d = p.dh[h];
        if (d > HUB_WARP_DEG) continue;
        if (p.hub_off[h] + d > p.S_cap) {
            if (lane == 0) atomicOr(p.err, 8u);
            continue;
        }
        hub_row_scan_warp<KIND>(p, __ldg(p.off + p.H[h]), d, p.S + p.hub_off[h], lane);
    }
}

// Edges in rows longer than theta: the size of the shared hub scratch when
// every such row is a hub of the layer.
__global__ void hub_edges_kernel(const uint64_t* __restrict__ off, uint32_t V, uint32_t theta,
                                 unsigned long long* __restrict__ out)
{
    unsigned long long t = 0;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t d = off[v + 1] - off[v];
        if (d > theta) t += d;
    }
    t = warp_sum_u64(t);
    if ((threadIdx.x & 31) == 0 && t) atomicAdd(out, t);
}

// ---------------------------------------------------------------------------
// Frontier construction.

// Keys of the seeds: instance of seed j from the offsets, checks ranges.  The
// seed count is inst_off[n_inst] (clamped to cap, flag 4 when above); block 0
// stores it in *n_out for the kernels that follow.
__global__ void seed_keys_kernel(const uint32_t* __restrict__ seeds, const uint64_t* __restrict__ inst_off,
                                 uint32_t n_inst, uint64_t cap, uint32_t V, uint32_t vbits,
                                 uint64_t* __restrict__ keys, uint32_t* __restrict__ err,
                                 uint64_t* __restrict__ n_out)
{
    uint64_t n_seeds = inst_off[n_inst];
    if (n_seeds > cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, 4u);
        n_seeds = cap;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_out = n_seeds;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_seeds;
         j += (uint64_t)gridDim.x * blockDim.x) {
        // instance = last i with inst_off[i] <= j
        uint32_t lo = 0, hi = n_inst;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (inst_off[mid] <= j) lo = mid; else hi = mid - 1;
        }
        const uint32_t sd = seeds[j];
        if (sd >= V) atomicOr(err, 1u);
        keys[j] = ((uint64_t)lo << vbits) | (sd < V ? sd : 0u);
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
// eoff[i] = base + pos[foff[i]] for i <= n_inst; fsize[i] = foff[i+1] - foff[i];
// *next_base = base + (edges of this layer).
__global__ void layer_offsets_kernel(const uint64_t* __restrict__ foff, const uint64_t* __restrict__ pos,
                                     uint32_t n_inst, const uint64_t* __restrict__ base_dev,
                                     uint64_t* __restrict__ eoff, uint64_t* __restrict__ fsize,
                                     uint64_t* __restrict__ next_base)
{
    const uint64_t base = *base_dev;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n_inst;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t e = base + pos[foff[i]];
        eoff[i] = e;
        if (i < n_inst) fsize[i] = foff[i + 1] - foff[i];
        else *next_base = e;
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
// Host pipeline.
//
// One sampling call is: the layer-0 frontier from the seeds, then per layer a
// count/classify pass, a scan for edge positions, the persistent selection
// kernel, and (but for the last layer) compaction into the next frontier.
// Every kernel reads its element count from device memory, so the same
// sequence serves two modes:
//   - csaw_sample: waits once per layer to size that layer's edge buffers
//     exactly (frontier arrays take the previous layer's edge count as bound);
//   - a sample plan: every buffer at its upper bound, no waits, captured once
//     into a CUDA graph and replayed for each new batch of seeds.

struct csaw_sample_result {
    uint32_t magic = 0x43534d50u;   // "CSMP"
    uint32_t depth = 0;
    uint32_t n_instances = 0;
    uint64_t n_edges = 0;
    std::vector<uint64_t> edge_offsets;     // host
    std::vector<uint64_t> frontier_sizes;   // host
    std::vector<uint32_t*> src, dst;        // device, per layer (owned)
    std::vector<const uint32_t*> src_c, dst_c;
    std::vector<uint64_t> layer_edges;
    DevAllocator alloc;               // the caller's allocator of src/dst, if any
    cudaStream_t stream = nullptr;          // the stream they were allocated on
    ~csaw_sample_result()
    {
        for (auto p : src) release(p);
        for (auto p : dst) release(p);
    }
    void release(void* p)
    {
        if (!p) return;
        if (alloc.free) alloc.free(p, (void*)stream, alloc.ctx);
        else cudaFree(p);
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
static csaw_status launch_select(const SelParams& p, int blocks, cudaStream_t s, size_t smem = SEL_DYN_SMEM)
{
    select_kernel<KIND><<<blocks, SEL_THREADS, smem, s>>>(p);
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

// Resident blocks of the selection kernel per SM (occupancy limit).
static int select_occupancy(int kind)
{
    // looked up once per kind; the attribute is set before the value is
    // published, so a thread that reads it may launch (calls may come from
    // several threads, e.g. the request server's slots)
    static std::atomic<int> cached[4];
    const int have = cached[kind].load(std::memory_order_acquire);
    if (have) return have;
    {
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
        cached[kind].store(per_sm, std::memory_order_release);
        return per_sm;
    }
}

static int select_blocks(int kind, int sm_count)
{
    return sm_count * select_occupancy(kind);
}

// Resident blocks per SM of a launch with warp items only (SEL_WARP_SMEM).
static int select_occupancy_warp(int kind)
{
    static std::atomic<int> cached[4];
    const int have = cached[kind].load(std::memory_order_acquire);
    if (have) return have;
    int per_sm = 1;
    cudaError_t e = cudaSuccess;
    switch (kind) {
    case CSAW_BIAS_UNIFORM:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_kernel<CSAW_BIAS_UNIFORM>, SEL_THREADS, SEL_WARP_SMEM);
        break;
    case CSAW_BIAS_EDGE_WEIGHT:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_kernel<CSAW_BIAS_EDGE_WEIGHT>, SEL_THREADS, SEL_WARP_SMEM);
        break;
    default:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_kernel<CSAW_BIAS_NEIGHBOR_DEGREE>, SEL_THREADS, SEL_WARP_SMEM);
        break;
    }
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    cached[kind].store(per_sm, std::memory_order_release);
    return per_sm;
}

// Launch shape of the selection kernel for this graph and kind: the tuned
// values when set (csaw_set_select_tuning / csaw_autotune_select).
static void select_shape(const csaw_graph* g, int kind, uint32_t* theta_w, int* blocks)
{
    const uint32_t tw = g->tune_theta_w[kind];
    *theta_w = (tw == 0 || tw > WARP_MAX_DEG) ? WARP_MAX_DEG : tw;
    const int occ = select_occupancy(kind);
    int per = (int)g->tune_blocks_per_sm[kind];
    if (per <= 0 || per > occ) per = occ;
    *blocks = g->sm_count * per;
}

// Device counters of one call (zeroed at its start): error flags, the seed
// count, the edge base of each layer, and sixteen words per layer.
constexpr int L_WORDS = 16;
enum : int {
    CT_ERR = 0,
    CT_NSEEDS = 1,
    CT_BASE = 2,                      // CT_BASE + l: first edge of layer l (l <= depth)
    CT_LAYER = CT_BASE + CSAW_MAX_DEPTH + 2,
    CT_WORDS = CT_LAYER + L_WORDS * CSAW_MAX_DEPTH,
};
// per layer: frontier entries, edges, item counts (warp, CTA, hub) and their
// work counters, distinct hubs, their edges, hubs built by a whole CTA and
// the two build counters
enum : int { L_N = 0, L_TOTAL = 1, L_ITEMS = 2, L_NEXT = 5, L_NH = 8, L_HUBE = 9, L_NBIG = 10,
             L_HNEXT = 11 };

// ---------------------------------------------------------------------------
// Layer sampling (Sec. II-A; Fig. 2(b) with the whole frontier as the current
// frontier).  Per instance and layer, the NeighborPool is every edge of the
// instance's frontier, ascending source then CSR order, with its edge bias;
// Select picks k entries without replacement by the rule of draw_picks
// (repeated sampling for attempt_cap attempts, then updated sampling; all
// positive entries when there are at most k), draws keyed {attempt, NONE,
// layer, instance}.  One warp per instance.  The count kernel writes
// min(k, positive entries) at the instance's first frontier entry and 0 at
// its others, so the layer's scan places each instance's picks; the select
// kernel writes them in pick order.  A pick is found in two levels: the
// entry (frontier vertex) by a binary search of the inclusive prefix of
// entry totals, then the row position by a warp scan of the row's biases
// (a binary search of the cached cumulative array when present; the draw
// itself for uniform bias).
struct LayerSelParams {
    SelParams s;                         // graph, frontier keys, k, layer, key, outputs, pos
    const uint64_t* __restrict__ FO;     // [n_inst + 1] frontier bounds of each instance
    uint32_t n_inst;
    uint32_t* cnt;                       // count kernel: [frontier]
    uint64_t* VP;                        // select: [frontier] prefix of entry totals in the instance
    uint64_t* p_eid;                     // select: [edges] edge index of each pick
    uint64_t* p_start;                   // select: [edges] pool prefix before each pick
    uint32_t* p_bias;                    // select: [edges] bias of each pick
    uint64_t* ctb;                       // select: [frontier] chunk table base of each entry (~0: none)
    uint64_t* ct;                        // select: [warps][LAYER_CT_CAP] chunk prefix tables
};

// Rows longer than LAYER_CHUNK keep the running sum at the end of every
// LAYER_CHUNK biases (taken in the totals pass) in the warp's table of
// LAYER_CT_CAP entries, so a pick bisects the table and scans one chunk.
constexpr uint32_t LAYER_CHUNK = 512;
constexpr uint32_t LAYER_CT_CAP = 4096;

// Total and positive count of row v's biases (warp-cooperative).
template <int KIND>
__device__ __forceinline__ void layer_row_total(const SelParams& p, uint64_t beg, uint32_t d, int lane,
                                                uint64_t* total, uint32_t* npos)
{
    if constexpr (KIND == CSAW_BIAS_UNIFORM) {
        *total = d;
        *npos = d;
        return;
    }
    if (p.cdf && !p.zero_bias) {
        *total = d ? __ldg(p.cdf + beg + d - 1) : 0ull;
        *npos = d;
        return;
    }
    uint64_t t = 0;
    uint32_t c = 0;
    for (uint32_t j = lane; j < d; j += 32) {
        const uint32_t b = sel_bias<KIND>(p, beg + j);
        t += b;
        c += b > 0;
    }
    *total = warp_sum_u64(t);
    *npos = __reduce_add_sync(CSAW_FULL_MASK, c);
}

template <int KIND>
__global__ void __launch_bounds__(SEL_THREADS) layer_count_kernel(LayerSelParams P)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * SEL_THREADS + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * SEL_THREADS) >> 5;
    const SelParams& p = P.s;
    for (uint64_t i = gw; i < P.n_inst; i += nw) {
        const uint64_t a = P.FO[i], b = P.FO[i + 1];
        uint64_t npos = 0;
        for (uint64_t e = a; e < b; ++e) {
            const uint32_t v = (uint32_t)(p.fkeys[e] & p.vmask);
            const uint64_t beg = __ldg(p.off + v);
            const uint32_t d = (uint32_t)(__ldg(p.off + v + 1) - beg);
            if (!p.zero_bias) {
                npos += d;
            } else {
                uint64_t t;
                uint32_t c;
                layer_row_total<KIND>(p, beg, d, lane, &t, &c);
                npos += c;
            }
        }
        for (uint64_t e = a + lane; e < b; e += 32)
            P.cnt[e] = e == a ? (uint32_t)(npos < p.k ? npos : p.k) : 0u;
    }
}

template <int KIND>
__global__ void __launch_bounds__(SEL_THREADS) layer_select_kernel(LayerSelParams P)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    const uint64_t gw = ((uint64_t)blockIdx.x * SEL_THREADS + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * SEL_THREADS) >> 5;
    SelParams p = P.s;
    if (p.key_dev) {
        p.k0 = p.key_dev[0];
        p.k1 = p.key_dev[1];
    }
    for (uint64_t i = gw; i < P.n_inst; i += nw) {
        const uint64_t a = P.FO[i], b = P.FO[i + 1];
        if (a == b) continue;
        const uint64_t q0 = p.pos[a];
        const uint32_t k = (uint32_t)(p.pos[a + 1] - q0);
        if (k == 0) continue;
        const uint32_t inst = (uint32_t)i;
        // entry totals, their inclusive prefix (VP) and the positive entries;
        // long rows also leave their chunk prefixes in this warp's table
        uint64_t T = 0, npos = 0;
        uint64_t* ct = P.ct + gw * LAYER_CT_CAP;
        uint32_t ct_used = 0;
        for (uint64_t e = a; e < b; ++e) {
            const uint32_t v = (uint32_t)(p.fkeys[e] & p.vmask);
            const uint64_t beg = __ldg(p.off + v);
            const uint32_t d = (uint32_t)(__ldg(p.off + v + 1) - beg);
            uint64_t t = 0;
            uint32_t c = 0;
            const uint32_t nch = (d + LAYER_CHUNK - 1) / LAYER_CHUNK;
            const bool table = KIND != CSAW_BIAS_UNIFORM && !p.cdf && d > LAYER_CHUNK &&
                               ct_used + nch <= LAYER_CT_CAP;
            if (table) {
                for (uint32_t ch = 0; ch < nch; ++ch) {
                    uint64_t tt = 0;
                    uint32_t cc = 0;
                    for (uint32_t j = ch * LAYER_CHUNK + lane; j < min(d, (ch + 1) * LAYER_CHUNK); j += 32) {
                        const uint32_t bb = sel_bias<KIND>(p, beg + j);
                        tt += bb;
                        cc += bb > 0;
                    }
                    t += warp_sum_u64(tt);
                    c += __reduce_add_sync(CSAW_FULL_MASK, cc);
                    if (lane == 0) ct[ct_used + ch] = t;
                }
                if (lane == 0) P.ctb[e] = ct_used;
                ct_used += nch;
            } else {
                layer_row_total<KIND>(p, beg, d, lane, &t, &c);
                if (lane == 0) P.ctb[e] = ~0ull;
            }
            T += t;
            npos += c;
            if (lane == 0) P.VP[e] = T;
        }
        __syncwarp();
        if (npos <= p.k) {
            // take every positive entry, pool order
            uint64_t q = q0;
            for (uint64_t e = a; e < b; ++e) {
                const uint32_t v = (uint32_t)(p.fkeys[e] & p.vmask);
                const uint64_t beg = __ldg(p.off + v);
                const uint32_t d = (uint32_t)(__ldg(p.off + v + 1) - beg);
                for (uint32_t base = 0; base < d; base += 32) {
                    const uint32_t j = base + lane;
                    const bool take = j < d && (!p.zero_bias || sel_bias<KIND>(p, beg + j) > 0);
                    const uint32_t bal = __ballot_sync(CSAW_FULL_MASK, take);
                    if (take) emit(p, q + __popc(bal & lt), v, inst, __ldg(p.col + beg + j));
                    q += __popc(bal);
                }
            }
            continue;
        }
        uint32_t have = 0;
        uint64_t R = 0;   // sum of the picked biases
        for (uint32_t at = 0; have < k; ++at) {
            const uint64_t r = philox_draw(p.k0, p.k1, at, CSAW_NONE, p.layer, inst);
            uint64_t x;
            if (at < p.attempt_cap) {
                x = scale_draw(r, T);
            } else {
                // updated sampling: the draw over the unpicked total, mapped
                // past the picked intervals (fixpoint of y = x + picked
                // biases starting at or below y)
                x = scale_draw(r, T - R);
                uint64_t y = x;
                while (true) {
                    uint64_t add = 0;
                    for (uint32_t t = lane; t < have; t += 32)
                        if (P.p_start[q0 + t] <= y) add += P.p_bias[q0 + t];
                    const uint64_t ny = x + warp_sum_u64(add);
                    if (ny == y) break;
                    y = ny;
                }
                x = y;
            }
            // the entry: first with VP > x
            uint64_t lo = a, hi = b;
            while (lo < hi) {
                const uint64_t mid = lo + ((hi - lo) >> 1);
                if (P.VP[mid] > x) hi = mid; else lo = mid + 1;
            }
            const uint64_t e = lo;
            const uint64_t before = e > a ? P.VP[e - 1] : 0ull;
            const uint64_t xr = x - before;
            const uint32_t v = (uint32_t)(p.fkeys[e] & p.vmask);
            const uint64_t beg = __ldg(p.off + v);
            const uint32_t d = (uint32_t)(__ldg(p.off + v + 1) - beg);
            // the row position: first j with S_row[j] > xr, and S_row[j-1]
            uint32_t j = 0;
            uint64_t sprev = 0, sj = 0;
            if constexpr (KIND == CSAW_BIAS_UNIFORM) {
                j = (uint32_t)xr;
                sprev = xr;
                sj = xr + 1;
            } else if (p.cdf) {
                uint32_t l2 = 0, h2 = d;
                while (l2 < h2) {
                    const uint32_t mid = (l2 + h2) >> 1;
                    if (__ldg(p.cdf + beg + mid) > xr) h2 = mid; else l2 = mid + 1;
                }
                j = l2;
                sprev = j ? __ldg(p.cdf + beg + j - 1) : 0ull;
                sj = __ldg(p.cdf + beg + j);
            } else {
                uint64_t base = 0;
                uint32_t c_begin = 0;
                const uint64_t cb = P.ctb[e];
                if (cb != ~0ull) {
                    // the chunk holding xr: first whose running sum exceeds it
                    const uint32_t nch = (d + LAYER_CHUNK - 1) / LAYER_CHUNK;
                    uint32_t l2 = 0, h2 = nch;
                    while (l2 < h2) {
                        const uint32_t mid = (l2 + h2) >> 1;
                        if (ct[cb + mid] > xr) h2 = mid; else l2 = mid + 1;
                    }
                    c_begin = l2 * LAYER_CHUNK;
                    base = l2 ? ct[cb + l2 - 1] : 0ull;
                }
                for (uint32_t c0 = c_begin; c0 < d; c0 += 32) {
                    const uint32_t jj = c0 + lane;
                    const uint32_t bl = jj < d ? sel_bias<KIND>(p, beg + jj) : 0u;
                    const uint64_t incl = base + warp_inclusive_scan_u64(bl, lane);
                    const uint32_t hit = __ballot_sync(CSAW_FULL_MASK, incl > xr);
                    if (hit) {
                        const int L = __ffs(hit) - 1;
                        j = c0 + (uint32_t)L;
                        sj = __shfl_sync(CSAW_FULL_MASK, incl, L);
                        sprev = sj - __shfl_sync(CSAW_FULL_MASK, (uint64_t)bl, L);
                        break;
                    }
                    base = __shfl_sync(CSAW_FULL_MASK, incl, 31);
                }
            }
            const uint64_t eid = beg + j;
            bool dup = false;
            if (at < p.attempt_cap) {
                for (uint32_t t = lane; t < have; t += 32) dup |= P.p_eid[q0 + t] == eid;
                dup = __any_sync(CSAW_FULL_MASK, dup);
            }
            if (!dup) {
                if (lane == 0) {
                    P.p_eid[q0 + have] = eid;
                    P.p_start[q0 + have] = before + sprev;
                    P.p_bias[q0 + have] = (uint32_t)(sj - sprev);
                    emit(p, q0 + have, v, inst, __ldg(p.col + eid));
                }
                R += sj - sprev;
                ++have;
                __syncwarp();
            }
        }
    }
}

struct LayerBufs {
    uint64_t f_cap = 0, e_cap = 0;
    uint64_t* F = nullptr;       // frontier keys [f_cap], sorted
    uint64_t* FO = nullptr;      // instance bounds [n_inst + 1]
    uint32_t* cnt = nullptr;     // [f_cap]
    uint32_t* wlist = nullptr;   // [f_cap]
    uint32_t* clist = nullptr;   // [f_cap]
    uint64_t* pos = nullptr;     // [f_cap + 1]
    uint32_t* src = nullptr;     // [e_cap]
    uint32_t* dst = nullptr;     // [e_cap]
    uint64_t* cand = nullptr;    // [e_cap] candidate keys (not on the last layer)
    uint64_t* cand_alt = nullptr;
    uint32_t* kept = nullptr;
    uint64_t* kpos = nullptr;    // [e_cap + 1]
};

struct Pipeline {
    csaw_graph* g = nullptr;
    int kind = 0;
    uint32_t n_inst = 0, depth = 0;
    uint32_t fanout[CSAW_MAX_DEPTH] = {};
    bool zero_bias = false;
    int vbits = 1, kbits = 1;
    uint64_t vmask = 1;
    int sel_blocks = 1;
    uint32_t theta_w = WARP_MAX_DEG;
    bool cached = false;                 // selection over a cached cumulative array
    bool hub_path = false;               // shared hub arrays per layer (static bias, streamed)
    bool hub_order = false;              // cached static bias: hub items visited in vertex order
    bool cta_slots = false;              // CTA items may exceed CTA_SMEM_DEG: global slots
    uint32_t attempt_cap = CSAW_ATTEMPT_CAP;
    uint32_t k0 = 0, k1 = 0;
    const uint32_t* key_dev = nullptr;   // plan mode: Philox key in device memory
    // several requests in one run: per-instance draw keys and fanouts (device)
    const uint32_t* inst_key = nullptr;  // [2 * n_inst]
    const uint32_t* inst_id = nullptr;   // [n_inst]
    const uint32_t* inst_fan = nullptr;  // [depth][n_inst]
    uint64_t* ctr = nullptr;             // [CT_WORDS]
    void* scan_scr = nullptr;
    void* sort_scr = nullptr;
    uint64_t* hub_S = nullptr;
    uint32_t* hub_bits = nullptr;
    uint64_t* eoff = nullptr;            // [depth * n_inst + 1]
    uint64_t* fsize = nullptr;           // [depth * n_inst]
    uint64_t seeds_cap = 0;
    uint64_t* seed_keys = nullptr;       // [seeds_cap]
    uint64_t* seed_alt = nullptr;
    uint32_t* seed_kept = nullptr;
    uint64_t* seed_kpos = nullptr;       // [seeds_cap + 1]
    LayerBufs L[CSAW_MAX_DEPTH];
    // hub grouping of one layer at a time (hub_cap items), and the shared
    // hub prefix sums (hubS_cap entries)
    uint64_t hub_cap = 0, hubS_cap = 0;
    uint32_t* hlist = nullptr;           // [hub_cap] hub items in count order
    uint64_t* hkeys = nullptr;           // [hub_cap] sort keys
    uint64_t* halt = nullptr;            // [hub_cap]
    uint32_t* hflag = nullptr;           // [hub_cap]
    uint64_t* hpos = nullptr;            // [hub_cap + 1]
    uint32_t* item_e = nullptr;          // [hub_cap]
    uint32_t* item_h = nullptr;          // [hub_cap]
    uint32_t* hubH = nullptr;            // [hub_cap] distinct hub vertices
    uint32_t* hubD = nullptr;            // [hub_cap] their degrees
    uint32_t* hubBig = nullptr;          // [hub_cap] hubs built by a whole CTA
    uint64_t* hub_off = nullptr;         // [hub_cap + 1]
    uint64_t* hubS = nullptr;            // [hubS_cap]

    uint64_t* lc(uint32_t l, int w) const { return ctr + CT_LAYER + L_WORDS * l + w; }

    void init(csaw_graph* gr, int k, uint32_t ninst, uint32_t dep, const uint32_t* fan, uint64_t seed)
    {
        g = gr;
        kind = k;
        n_inst = ninst;
        depth = dep;
        for (uint32_t l = 0; l < dep; ++l) fanout[l] = fan[l];
        const int vb = bits_for(g->V - 1);
        vbits = vb > 0 ? vb : 1;
        kbits = vbits + bits_for(n_inst > 0 ? n_inst - 1 : 0);
        vmask = (1ull << vbits) - 1;
        zero_bias = (kind == CSAW_BIAS_EDGE_WEIGHT && g->min_weight == 0) ||
                    (kind == CSAW_BIAS_NEIGHBOR_DEGREE && g->zero_degree_target);
        select_shape(g, kind, &theta_w, &sel_blocks);
        cached = cached_cdf_usable(g, kind);
        // shared hub arrays pay when several instances can reach the same
        // hub; a single instance's frontier holds each vertex once, and its
        // long rows take the CTA path without the grouping kernels
        hub_path = !cached && n_inst > 1 && (kind == CSAW_BIAS_EDGE_WEIGHT || kind == CSAW_BIAS_NEIGHBOR_DEGREE);
        // vertex order pays only when several instances can hold the same hub
        hub_order = cached && n_inst > 1 && (kind == CSAW_BIAS_EDGE_WEIGHT || kind == CSAW_BIAS_NEIGHBOR_DEGREE);
        // CTA items exist for picks above PICK_MAX (or, without the hub
        // path, any long row); only rows above CTA_SMEM_DEG need a slot
        bool big_k = false;
        for (uint32_t l = 0; l < dep; ++l) big_k |= fan[l] > PICK_MAX && fan[l] != CSAW_FANOUT_ALL;
        cta_slots = g->max_degree > CTA_SMEM_DEG && (big_k || (!cached && !hub_path));
        k0 = (uint32_t)seed;
        k1 = (uint32_t)(seed >> 32);
    }

    // Capacities of a layer's per-entry and edge arrays.
    uint64_t edge_bound(uint32_t l, uint64_t f) const
    {
        const uint64_t k = fanout[l] < g->max_degree ? fanout[l] : g->max_degree;
        return f * k;
    }
};

// Layer-0 frontier: sorted distinct (instance, seed) keys.
static csaw_status enqueue_frontier0(Pipeline& P, const uint32_t* seeds, const uint64_t* inst_off,
                                     cudaStream_t s)
{
    csaw_graph* g = P.g;
    const uint64_t cap = P.seeds_cap;
    check_inst_off_kernel<<<grid_for(P.n_inst, 256, g->sm_count), 256, 0, s>>>(inst_off, P.n_inst, (uint32_t*)(P.ctr + CT_ERR));
    seed_keys_kernel<<<grid_for(cap, 256, g->sm_count), 256, 0, s>>>(
        seeds, inst_off, P.n_inst, cap, g->V, P.vbits, P.seed_keys, (uint32_t*)(P.ctr + CT_ERR), P.ctr + CT_NSEEDS);
    uint64_t* sorted = P.seed_keys;
    if (cap) CSAW_TRY(radix_sort_u64(P.seed_keys, P.seed_alt, P.ctr + CT_NSEEDS, cap, P.kbits, g->sm_count, P.sort_scr, s, &sorted));
    Visited none;
    none.n = 0;
    unique_filter_kernel<<<grid_for(cap, 256, g->sm_count), 256, 0, s>>>(sorted, P.ctr + CT_NSEEDS, none, P.vbits, P.seed_kept);
    CSAW_TRY(scan_u32(P.seed_kept, P.seed_kpos, P.ctr + CT_NSEEDS, cap, P.scan_scr, P.lc(0, L_N), s));
    scatter_kept_kernel<<<grid_for(cap, 256, g->sm_count), 256, 0, s>>>(sorted, P.ctr + CT_NSEEDS, P.seed_kept, P.seed_kpos, P.L[0].F);
    inst_bounds_kernel<<<grid_for((uint64_t)P.n_inst + 1, 256, g->sm_count), 256, 0, s>>>(P.L[0].F, P.lc(0, L_N), P.n_inst, P.vbits, P.L[0].FO);
    CSAW_CUDA(cudaGetLastError());
    return CSAW_OK;
}

// Hub grouping of layer l: sort the hub items by vertex, number the distinct
// hub vertices, and give each a range of the shared scratch (exclusive scan
// of their degrees; the layer's total is L_HUBE).
static csaw_status enqueue_hub_groups(Pipeline& P, uint32_t l, cudaStream_t s)
{
    csaw_graph* g = P.g;
    const uint64_t cap = P.L[l].f_cap;
    const unsigned long long* n_hub = (const unsigned long long*)P.lc(l, L_ITEMS + 2);
    const unsigned grid = grid_for(cap, 256, g->sm_count);
    const uint32_t vshift = ((uint32_t)P.vbits + 7u) & ~7u;
    hub_keys_kernel<<<grid, 256, 0, s>>>(P.hlist, n_hub, P.L[l].F, P.vmask, vshift, P.hkeys);
    uint64_t* sorted = P.hkeys;
    CSAW_TRY(radix_sort_u64(P.hkeys, P.halt, (const uint64_t*)n_hub, cap, (int)vshift, g->sm_count, P.sort_scr,
                            s, &sorted));
    hub_flag_kernel<<<grid, 256, 0, s>>>(sorted, n_hub, P.vmask, P.hflag);
    CSAW_TRY(scan_u32(P.hflag, P.hpos, (const uint64_t*)n_hub, cap, P.scan_scr, P.lc(l, L_NH), s));
    hub_items_kernel<<<grid, 256, 0, s>>>(sorted, n_hub, P.hflag, P.hpos, P.vmask, vshift, g->off,
                                          P.item_e, P.item_h, P.hubH, P.hubD, P.hubBig,
                                          (unsigned long long*)P.lc(l, L_NBIG));
    CSAW_TRY(scan_u32(P.hubD, P.hub_off, P.lc(l, L_NH), cap, P.scan_scr, P.lc(l, L_HUBE), s));
    CSAW_CUDA(cudaGetLastError());
    return CSAW_OK;
}

// Cached arrays: the layer's hub items in vertex order (item_e), so that the
// warps drawing from one hub's row run back to back and share its lines in L2.
static csaw_status enqueue_hub_order(Pipeline& P, uint32_t l, cudaStream_t s)
{
    csaw_graph* g = P.g;
    const uint64_t cap = P.L[l].f_cap;
    const unsigned long long* n_hub = (const unsigned long long*)P.lc(l, L_ITEMS + 2);
    const unsigned grid = grid_for(cap, 256, g->sm_count);
    const uint32_t vshift = ((uint32_t)P.vbits + 7u) & ~7u;
    hub_keys_kernel<<<grid, 256, 0, s>>>(P.hlist, n_hub, P.L[l].F, P.vmask, vshift, P.hkeys);
    uint64_t* sorted = P.hkeys;
    CSAW_TRY(radix_sort_u64(P.hkeys, P.halt, (const uint64_t*)n_hub, cap, (int)vshift, g->sm_count, P.sort_scr,
                            s, &sorted));
    hub_order_kernel<<<grid, 256, 0, s>>>(sorted, n_hub, vshift, P.item_e);
    CSAW_CUDA(cudaGetLastError());
    return CSAW_OK;
}

// Count/classify of layer l's entries (vertices in [v_lo, v_hi) listed;
// write_cnt: store the counts).
static csaw_status enqueue_classify(Pipeline& P, uint32_t l, uint32_t v_lo, uint32_t v_hi, bool write_cnt,
                                   cudaStream_t s)
{
    csaw_graph* g = P.g;
    LayerBufs& B = P.L[l];
    CountParams cp;
    cp.off = g->off; cp.col = g->col; cp.w = g->w; cp.deg = g->deg;
    cp.fkeys = B.F; cp.n_dev = (const unsigned long long*)P.lc(l, L_N); cp.vmask = P.vmask;
    cp.k = P.fanout[l]; cp.theta_w = P.theta_w; cp.cached = P.cached; cp.zero_bias = P.zero_bias;
    cp.cnt = B.cnt; cp.warp_list = B.wlist; cp.cta_list = B.clist;
    cp.n_items = (unsigned long long*)P.lc(l, L_ITEMS);
    cp.hub_list = P.hub_path || P.hub_order ? P.hlist : nullptr;
    cp.inst_k = P.inst_fan ? P.inst_fan + (uint64_t)l * P.n_inst : nullptr;
    cp.vbits = (uint32_t)P.vbits;
    cp.v_lo = v_lo; cp.v_hi = v_hi; cp.write_cnt = write_cnt;
    if (B.f_cap) {
        switch (P.kind) {
        case CSAW_BIAS_UNIFORM: CSAW_TRY(launch_count<CSAW_BIAS_UNIFORM>(cp, B.f_cap, g->sm_count, s)); break;
        case CSAW_BIAS_EDGE_WEIGHT: CSAW_TRY(launch_count<CSAW_BIAS_EDGE_WEIGHT>(cp, B.f_cap, g->sm_count, s)); break;
        default: CSAW_TRY(launch_count<CSAW_BIAS_NEIGHBOR_DEGREE>(cp, B.f_cap, g->sm_count, s)); break;
        }
    }
    return CSAW_OK;
}

// Count/classify and the edge-position scan of layer l.
static csaw_status enqueue_count(Pipeline& P, uint32_t l, cudaStream_t s)
{
    LayerBufs& B = P.L[l];
    CSAW_TRY(enqueue_classify(P, l, 0, 0xFFFFFFFFu, true, s));
    CSAW_TRY(scan_u32(B.cnt, B.pos, P.lc(l, L_N), B.f_cap, P.scan_scr, P.lc(l, L_TOTAL), s));
    if (P.hub_path && B.f_cap) CSAW_TRY(enqueue_hub_groups(P, l, s));
    if (P.hub_order && B.f_cap) CSAW_TRY(enqueue_hub_order(P, l, s));
    return CSAW_OK;
}

// The selection kernels of layer l (its listed items) into its edge buffers.
static csaw_status enqueue_select_items(Pipeline& P, uint32_t l, cudaStream_t s)
{
    csaw_graph* g = P.g;
    LayerBufs& B = P.L[l];
    if (B.f_cap) {
        SelParams sp;
        sp.off = g->off; sp.col = g->col; sp.w = g->w; sp.deg = g->deg;
        sp.fkeys = B.F; sp.vbits = P.vbits; sp.vmask = P.vmask; sp.k = P.fanout[l]; sp.layer = l;
        sp.k0 = P.k0; sp.k1 = P.k1; sp.key_dev = P.key_dev;
        sp.zero_bias = P.zero_bias; sp.pos = B.pos; sp.warp_list = B.wlist; sp.cta_list = B.clist;
        sp.n_items = (const unsigned long long*)P.lc(l, L_ITEMS);
        sp.next = (unsigned long long*)P.lc(l, L_NEXT);
        sp.out_src = B.src; sp.out_dst = B.dst; sp.out_cand = (l + 1 < P.depth) ? B.cand : nullptr;
        sp.scratch_S = P.hub_S; sp.scratch_bits = P.hub_bits; sp.scratch_stride = g->max_degree;
        sp.cdf = P.cached && P.kind != CSAW_BIAS_UNIFORM ? g->cdf[P.kind] : nullptr;
    sp.cv = cdf_view(sp.cdf, g->E, g->V);
        sp.skip_warp_items = P.cached;
        sp.attempt_cap = P.attempt_cap;
        sp.inst_key = P.inst_key; sp.inst_id = P.inst_id;
        sp.inst_k = P.inst_fan ? P.inst_fan + (uint64_t)l * P.n_inst : nullptr;
        if (P.cached) {
            // warp items over the cached array; CTA items (more than PICK_MAX
            // picks) by the streaming kernel below
            const int blocks = g->sm_count * 8;
            if (P.kind == CSAW_BIAS_UNIFORM) select_cdf_kernel<true><<<blocks, SEL_THREADS, 0, s>>>(sp);
            else select_cdf_kernel<false, true><<<blocks, SEL_THREADS, 0, s>>>(sp);
            if (P.hub_order) {
                // the hub items in vertex order, over the same array
                SelParams hs = sp;
                hs.item_e = P.item_e;
                if (P.fanout[l] <= 16) select_cdf_kernel<false, true, 16><<<blocks, SEL_THREADS, 0, s>>>(hs);
                else select_cdf_kernel<false, true><<<blocks, SEL_THREADS, 0, s>>>(hs);
            }
            CSAW_CUDA(cudaGetLastError());
        }
        // with shared hub arrays a CTA item needs more than PICK_MAX picks: a
        // layer whose fanout is at most that holds warp items only, launched
        // with their slots alone (more resident blocks hide the gathers)
        const bool warp_only = P.hub_path && P.fanout[l] <= PICK_MAX;
        int blocks = P.sel_blocks;
        size_t smem = SEL_DYN_SMEM;
        if (warp_only) {
            const int occ = select_occupancy_warp(P.kind);
            const int per = (int)g->tune_blocks_per_sm[P.kind];
            blocks = g->sm_count * (per > 0 && per < occ ? per : occ);
            smem = SEL_WARP_SMEM;
        }
        switch (P.kind) {
        case CSAW_BIAS_UNIFORM: CSAW_TRY(launch_select<CSAW_BIAS_UNIFORM>(sp, blocks, s, smem)); break;
        case CSAW_BIAS_EDGE_WEIGHT: CSAW_TRY(launch_select<CSAW_BIAS_EDGE_WEIGHT>(sp, blocks, s, smem)); break;
        default: CSAW_TRY(launch_select<CSAW_BIAS_NEIGHBOR_DEGREE>(sp, blocks, s, smem)); break;
        }
        if (P.hub_path) {
            // the layer's distinct hubs: prefix sums built once each, then
            // every hub item draws from them
            HubBuildParams hp;
            hp.off = g->off; hp.col = g->col; hp.w = g->w; hp.deg = g->deg;
            hp.H = P.hubH; hp.dh = P.hubD; hp.hub_off = P.hub_off;
            hp.nh = (const unsigned long long*)P.lc(l, L_NH);
            hp.big_list = P.hubBig; hp.n_big = (const unsigned long long*)P.lc(l, L_NBIG);
            hp.next = (unsigned long long*)P.lc(l, L_HNEXT); hp.S = P.hubS;
            hp.S_cap = P.hubS_cap; hp.err = (uint32_t*)(P.ctr + CT_ERR);
            const int blocks = g->sm_count * 8;
            if (P.kind == CSAW_BIAS_EDGE_WEIGHT) hub_cdf_kernel<CSAW_BIAS_EDGE_WEIGHT><<<blocks, SEL_THREADS, 0, s>>>(hp);
            else hub_cdf_kernel<CSAW_BIAS_NEIGHBOR_DEGREE><<<blocks, SEL_THREADS, 0, s>>>(hp);
            SelParams hs = sp;
            hs.cdf = nullptr;
            hs.item_e = P.item_e; hs.item_h = P.item_h; hs.hub_off = P.hub_off; hs.hubS = P.hubS;
            hs.hubS_cap = P.hubS_cap; hs.err = (uint32_t*)(P.ctr + CT_ERR);
            // hub rows are long, so with at most 16 picks two items share a warp
            if (P.fanout[l] <= 16) select_cdf_kernel<false, false, 16><<<g->sm_count * 8, SEL_THREADS, 0, s>>>(hs);
            else select_cdf_kernel<false><<<g->sm_count * 8, SEL_THREADS, 0, s>>>(hs);
            CSAW_CUDA(cudaGetLastError());
        }
    }
    return CSAW_OK;
}

// Edge offsets and frontier sizes of layer l.
static csaw_status enqueue_layer_offsets(Pipeline& P, uint32_t l, cudaStream_t s)
{
    csaw_graph* g = P.g;
    LayerBufs& B = P.L[l];
    layer_offsets_kernel<<<grid_for((uint64_t)P.n_inst + 1, 256, g->sm_count), 256, 0, s>>>(
        B.FO, B.pos, P.n_inst, P.ctr + CT_BASE + l, P.eoff + (uint64_t)l * P.n_inst,
        P.fsize + (uint64_t)l * P.n_inst, P.ctr + CT_BASE + l + 1);
    CSAW_CUDA(cudaGetLastError());
    return CSAW_OK;
}

// Selection of layer l into its edge buffers, then its offsets.
static csaw_status enqueue_select(Pipeline& P, uint32_t l, cudaStream_t s)
{
    CSAW_TRY(enqueue_select_items(P, l, s));
    return enqueue_layer_offsets(P, l, s);
    return CSAW_OK;
}

// Update (Eq. 4): next frontier = sorted distinct picks of layer l that the
// instance has not visited in layers 0..l.
static csaw_status enqueue_compact(Pipeline& P, uint32_t l, cudaStream_t s)
{
    csaw_graph* g = P.g;
    LayerBufs& B = P.L[l];
    LayerBufs& N = P.L[l + 1];
    uint64_t* sorted = B.cand;
    if (B.e_cap) CSAW_TRY(radix_sort_u64(B.cand, B.cand_alt, P.lc(l, L_TOTAL), B.e_cap, P.kbits, g->sm_count, P.sort_scr, s, &sorted));
    Visited vis;
    vis.n = (int)l + 1;
    for (uint32_t j = 0; j <= l; ++j) { vis.keys[j] = P.L[j].F; vis.foff[j] = P.L[j].FO; }
    unique_filter_kernel<<<grid_for(B.e_cap, 256, g->sm_count), 256, 0, s>>>(sorted, P.lc(l, L_TOTAL), vis, P.vbits, B.kept);
    CSAW_TRY(scan_u32(B.kept, B.kpos, P.lc(l, L_TOTAL), B.e_cap, P.scan_scr, P.lc(l + 1, L_N), s));
    scatter_kept_kernel<<<grid_for(B.e_cap, 256, g->sm_count), 256, 0, s>>>(sorted, P.lc(l, L_TOTAL), B.kept, B.kpos, N.F);
    inst_bounds_kernel<<<grid_for((uint64_t)P.n_inst + 1, 256, g->sm_count), 256, 0, s>>>(N.F, P.lc(l + 1, L_N), P.n_inst, P.vbits, N.FO);
    CSAW_CUDA(cudaGetLastError());
    return CSAW_OK;
}

// Buffers shared by every layer (counters, scratch, offsets, seed arrays).
template <class Alloc>
static csaw_status alloc_common(Pipeline& P, Alloc&& get)
{
    CSAW_TRY(get((void**)&P.ctr, sizeof(uint64_t) * CT_WORDS));
    CSAW_TRY(get(&P.scan_scr, scan_scratch_bytes(0)));
    CSAW_TRY(get(&P.sort_scr, sort_scratch_bytes(0)));
    if (P.cta_slots) {
        CSAW_TRY(get((void**)&P.hub_S, sizeof(uint64_t) * (size_t)P.sel_blocks * P.g->max_degree));
        CSAW_TRY(get((void**)&P.hub_bits, sizeof(uint32_t) * (size_t)P.sel_blocks * ((P.g->max_degree + 31) / 32)));
    }
    const uint64_t ng = (uint64_t)P.depth * P.n_inst + 1;
    CSAW_TRY(get((void**)&P.eoff, sizeof(uint64_t) * ng));
    CSAW_TRY(get((void**)&P.fsize, sizeof(uint64_t) * ng));
    const uint64_t sc = P.seeds_cap ? P.seeds_cap : 1;
    CSAW_TRY(get((void**)&P.seed_keys, sizeof(uint64_t) * sc));
    CSAW_TRY(get((void**)&P.seed_alt, sizeof(uint64_t) * sc));
    CSAW_TRY(get((void**)&P.seed_kept, sizeof(uint32_t) * sc));
    CSAW_TRY(get((void**)&P.seed_kpos, sizeof(uint64_t) * (sc + 1)));
    return CSAW_OK;
}

// Hub grouping buffers for layers of up to `cap` frontier entries.
template <class Alloc>
static csaw_status alloc_hub(Pipeline& P, uint64_t cap, Alloc&& get)
{
    P.hub_cap = cap;
    const uint64_t c = cap ? cap : 1;
    CSAW_TRY(get((void**)&P.hlist, sizeof(uint32_t) * c));
    CSAW_TRY(get((void**)&P.hkeys, sizeof(uint64_t) * c));
    CSAW_TRY(get((void**)&P.halt, sizeof(uint64_t) * c));
    CSAW_TRY(get((void**)&P.hflag, sizeof(uint32_t) * c));
    CSAW_TRY(get((void**)&P.hpos, sizeof(uint64_t) * (c + 1)));
    CSAW_TRY(get((void**)&P.item_e, sizeof(uint32_t) * c));
    CSAW_TRY(get((void**)&P.item_h, sizeof(uint32_t) * c));
    CSAW_TRY(get((void**)&P.hubH, sizeof(uint32_t) * c));
    CSAW_TRY(get((void**)&P.hubD, sizeof(uint32_t) * c));
    CSAW_TRY(get((void**)&P.hubBig, sizeof(uint32_t) * c));
    CSAW_TRY(get((void**)&P.hub_off, sizeof(uint64_t) * (c + 1)));
    return CSAW_OK;
}

// Per-entry arrays of layer l (frontier capacity f_cap) and its frontier keys.
template <class Alloc>
static csaw_status alloc_entries(Pipeline& P, uint32_t l, uint64_t f_cap, Alloc&& get)
{
    LayerBufs& B = P.L[l];
    B.f_cap = f_cap;
    const uint64_t f = f_cap ? f_cap : 1;
    CSAW_TRY(get((void**)&B.F, sizeof(uint64_t) * f));
    CSAW_TRY(get((void**)&B.FO, sizeof(uint64_t) * ((uint64_t)P.n_inst + 1)));
    CSAW_TRY(get((void**)&B.cnt, sizeof(uint32_t) * f));
    CSAW_TRY(get((void**)&B.wlist, sizeof(uint32_t) * f));
    CSAW_TRY(get((void**)&B.clist, sizeof(uint32_t) * f));
    CSAW_TRY(get((void**)&B.pos, sizeof(uint64_t) * (f + 1)));
    return CSAW_OK;
}

// Edge arrays of layer l (capacity e_cap); src/dst come from `get_out`.
template <class Alloc, class AllocOut>
static csaw_status alloc_edges(Pipeline& P, uint32_t l, uint64_t e_cap, Alloc&& get, AllocOut&& get_out)
{
    LayerBufs& B = P.L[l];
    B.e_cap = e_cap;
    const uint64_t e = e_cap ? e_cap : 1;
    CSAW_TRY(get_out((void**)&B.src, sizeof(uint32_t) * e));
    CSAW_TRY(get_out((void**)&B.dst, sizeof(uint32_t) * e));
    if (l + 1 < P.depth) {
        if (e_cap >= 0xFFFFFFFFull)
            return fail(CSAW_ERR_INVALID, "layer %u may produce %llu edges; frontier compaction sorts "
                        "at most 2^32-1", l, (unsigned long long)e_cap);
        CSAW_TRY(get((void**)&B.cand, sizeof(uint64_t) * e));
        CSAW_TRY(get((void**)&B.cand_alt, sizeof(uint64_t) * e));
        CSAW_TRY(get((void**)&B.kept, sizeof(uint32_t) * e));
        CSAW_TRY(get((void**)&B.kpos, sizeof(uint64_t) * (e + 1)));
    }
    return CSAW_OK;
}

static csaw_status check_errors(uint64_t err)
{
    if (err & 1u) return fail(CSAW_ERR_INVALID, "a seed is not a vertex of the graph");
    if (err & 2u) return fail(CSAW_ERR_INVALID, "inst_offsets must start at 0 and be non-decreasing");
    if (err & 4u) return fail(CSAW_ERR_INVALID, "more seeds than the plan was created for");
    if (err & 8u) return fail(CSAW_ERR_CUDA, "internal: the shared hub scratch was too small");
    return CSAW_OK;
}

// Layer sampling: the parameters of layer l's count and select kernels.
static LayerSelParams layer_params(const Pipeline& P, uint32_t l)
{
    const csaw_graph* g = P.g;
    const LayerBufs& B = P.L[l];
    LayerSelParams lp = {};
    SelParams& sp = lp.s;
    sp.off = g->off; sp.col = g->col; sp.w = g->w; sp.deg = g->deg;
    sp.fkeys = B.F; sp.vbits = P.vbits; sp.vmask = P.vmask; sp.k = P.fanout[l]; sp.layer = l;
    sp.k0 = P.k0; sp.k1 = P.k1; sp.key_dev = P.key_dev;
    sp.zero_bias = P.zero_bias; sp.pos = B.pos;
    sp.out_src = B.src; sp.out_dst = B.dst; sp.out_cand = (l + 1 < P.depth) ? B.cand : nullptr;
    sp.cdf = P.cached && P.kind != CSAW_BIAS_UNIFORM ? g->cdf[P.kind] : nullptr;
    sp.cv = cdf_view(sp.cdf, g->E, g->V);
    sp.attempt_cap = P.attempt_cap;
    lp.FO = B.FO;
    lp.n_inst = P.n_inst;
    lp.cnt = B.cnt;
    return lp;
}

static int layer_grid(const Pipeline& P)
{
    const uint64_t want = ((uint64_t)P.n_inst + SEL_WARPS - 1) / SEL_WARPS;
    const uint64_t cap = (uint64_t)P.g->sm_count * 8;
    return (int)(want < 1 ? 1 : want < cap ? want : cap);
}

// Layer l of layer sampling: per-instance pick counts, then their scan.
static csaw_status enqueue_layer_count(Pipeline& P, uint32_t l, cudaStream_t s)
{
    LayerBufs& B = P.L[l];
    if (B.f_cap && P.n_inst) {
        const LayerSelParams lp = layer_params(P, l);
        switch (P.kind) {
        case CSAW_BIAS_UNIFORM: layer_count_kernel<CSAW_BIAS_UNIFORM><<<layer_grid(P), SEL_THREADS, 0, s>>>(lp); break;
        case CSAW_BIAS_EDGE_WEIGHT: layer_count_kernel<CSAW_BIAS_EDGE_WEIGHT><<<layer_grid(P), SEL_THREADS, 0, s>>>(lp); break;
        default: layer_count_kernel<CSAW_BIAS_NEIGHBOR_DEGREE><<<layer_grid(P), SEL_THREADS, 0, s>>>(lp); break;
        }
        CSAW_CUDA(cudaGetLastError());
    }
    return scan_u32(B.cnt, B.pos, P.lc(l, L_N), B.f_cap, P.scan_scr, P.lc(l, L_TOTAL), s);
}

// Layer l of layer sampling: the picks of every instance, then the offsets.
static csaw_status enqueue_layer_select(Pipeline& P, uint32_t l, uint64_t* VP, uint64_t* p_eid,
                                        uint64_t* p_start, uint32_t* p_bias, uint64_t* ctb, uint64_t* ct,
                                        cudaStream_t s)
{
    csaw_graph* g = P.g;
    LayerBufs& B = P.L[l];
    if (B.f_cap && P.n_inst) {
        LayerSelParams lp = layer_params(P, l);
        lp.VP = VP; lp.p_eid = p_eid; lp.p_start = p_start; lp.p_bias = p_bias;
        lp.ctb = ctb; lp.ct = ct;
        switch (P.kind) {
        case CSAW_BIAS_UNIFORM: layer_select_kernel<CSAW_BIAS_UNIFORM><<<layer_grid(P), SEL_THREADS, 0, s>>>(lp); break;
        case CSAW_BIAS_EDGE_WEIGHT: layer_select_kernel<CSAW_BIAS_EDGE_WEIGHT><<<layer_grid(P), SEL_THREADS, 0, s>>>(lp); break;
        default: layer_select_kernel<CSAW_BIAS_NEIGHBOR_DEGREE><<<layer_grid(P), SEL_THREADS, 0, s>>>(lp); break;
        }
        CSAW_CUDA(cudaGetLastError());
    }
    layer_offsets_kernel<<<grid_for((uint64_t)P.n_inst + 1, 256, g->sm_count), 256, 0, s>>>(
        B.FO, B.pos, P.n_inst, P.ctr + CT_BASE + l, P.eoff + (uint64_t)l * P.n_inst,
        P.fsize + (uint64_t)l * P.n_inst, P.ctr + CT_BASE + l + 1);
    CSAW_CUDA(cudaGetLastError());
    return CSAW_OK;
}

// csaw_sample: exact edge buffers, one wait per layer.
static csaw_status run_sample(csaw_graph* g, const uint32_t* seeds, const uint64_t* inst_off,
                              uint32_t n_inst, uint64_t n_seeds, uint32_t depth, const uint32_t* fanout,
                              int kind, uint64_t rng_seed, uint32_t attempt_cap, bool layer_mode,
                              cudaStream_t s, csaw_sample_result* R, const SampleTables* tabs = nullptr)
{
    Temps tmp(s);
    auto get = [&](void** p, size_t bytes) -> csaw_status {
        CSAW_TRY(dalloc(p, bytes, s));
        tmp.ptrs.push_back(*p);
        return CSAW_OK;
    };
    auto get_out = [&](void** p, size_t bytes) -> csaw_status { return dalloc(p, bytes, s); };
    if (const DevAllocator* a = current_allocator()) R->alloc = *a;
    R->stream = s;
    Pipeline P;
    P.init(g, kind, n_inst, depth, fanout, rng_seed);
    P.attempt_cap = attempt_cap;
    P.seeds_cap = n_seeds;
    if (tabs) {
        P.inst_key = tabs->inst_key;
        P.inst_id = tabs->inst_id;
        P.inst_fan = tabs->inst_fan;
    }
    CSAW_TRY(alloc_common(P, get));
    CSAW_CUDA(cudaMemsetAsync(P.ctr, 0, sizeof(uint64_t) * CT_WORDS, s));
    CSAW_TRY(alloc_entries(P, 0, n_seeds, get));
    CSAW_TRY(enqueue_frontier0(P, seeds, inst_off, s));
    R->src.assign(depth, nullptr);
    R->dst.assign(depth, nullptr);
    R->layer_edges.assign(depth, 0);
    const bool hubs = (P.hub_path || P.hub_order) && !layer_mode;
    for (uint32_t l = 0; l < depth; ++l) {
        // the layer's hub grouping buffers and shared hub prefix sums live
        // until its selection is done
        Temps layer_tmp(s);
        auto get_layer = [&](void** p, size_t bytes) -> csaw_status {
            CSAW_TRY(dalloc(p, bytes, s));
            layer_tmp.ptrs.push_back(*p);
            return CSAW_OK;
        };
        if (hubs) CSAW_TRY(alloc_hub(P, P.L[l].f_cap, get_layer));
        CSAW_TRY(layer_mode ? enqueue_layer_count(P, l, s) : enqueue_count(P, l, s));
        uint64_t h[3] = {0, 0, 0};
        CSAW_CUDA(cudaMemcpyAsync(&h[0], P.ctr + CT_ERR, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        CSAW_CUDA(cudaMemcpyAsync(&h[1], P.lc(l, L_TOTAL), sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        const bool shared = hubs && P.hub_path;   // shared hub arrays (streamed biases)
        if (shared) CSAW_CUDA(cudaMemcpyAsync(&h[2], P.lc(l, L_HUBE), sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        CSAW_CUDA(cudaStreamSynchronize(s));
        CSAW_TRY(check_errors(h[0]));
        const uint64_t total = h[1];
        if (shared) {
            P.hubS_cap = h[2];
            CSAW_TRY(get_layer((void**)&P.hubS, sizeof(uint64_t) * (h[2] ? h[2] : 1)));
        }
        R->layer_edges[l] = total;
        CSAW_TRY(alloc_edges(P, l, total, get, get_out));
        R->src[l] = P.L[l].src;
        R->dst[l] = P.L[l].dst;
        if (layer_mode) {
            uint64_t *VP = nullptr, *p_eid = nullptr, *p_start = nullptr;
            uint32_t* p_bias = nullptr;
            const uint64_t f = P.L[l].f_cap ? P.L[l].f_cap : 1, e = total ? total : 1;
            CSAW_TRY(get((void**)&VP, sizeof(uint64_t) * f));
            CSAW_TRY(get((void**)&p_eid, sizeof(uint64_t) * e));
            CSAW_TRY(get((void**)&p_start, sizeof(uint64_t) * e));
            CSAW_TRY(get((void**)&p_bias, sizeof(uint32_t) * e));
            uint64_t *ctb = nullptr, *ct = nullptr;
            CSAW_TRY(get((void**)&ctb, sizeof(uint64_t) * f));
            CSAW_TRY(get((void**)&ct, sizeof(uint64_t) * LAYER_CT_CAP * (uint64_t)layer_grid(P) * SEL_WARPS));
            CSAW_TRY(enqueue_layer_select(P, l, VP, p_eid, p_start, p_bias, ctb, ct, s));
        } else {
            CSAW_TRY(enqueue_select(P, l, s));
        }
        if (l + 1 < depth) {
            CSAW_TRY(alloc_entries(P, l + 1, total, get));
            CSAW_TRY(enqueue_compact(P, l, s));
        }
    }
    const uint64_t ng = (uint64_t)depth * n_inst;
    R->edge_offsets.assign(ng + 1, 0);
    R->frontier_sizes.assign(ng, 0);
    if (ng) {
        CSAW_CUDA(cudaMemcpyAsync(R->edge_offsets.data(), P.eoff, sizeof(uint64_t) * (ng + 1), cudaMemcpyDeviceToHost, s));
        CSAW_CUDA(cudaMemcpyAsync(R->frontier_sizes.data(), P.fsize, sizeof(uint64_t) * ng, cudaMemcpyDeviceToHost, s));
    }
    uint64_t err_end = 0;
    CSAW_CUDA(cudaMemcpyAsync(&err_end, P.ctr + CT_ERR, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    CSAW_CUDA(cudaStreamSynchronize(s));
    CSAW_TRY(check_errors(err_end));
    uint64_t total = 0;
    for (uint32_t l = 0; l < depth; ++l) total += R->layer_edges[l];
    R->n_edges = total;
    R->edge_offsets[ng] = total;
    R->src_c.assign(R->src.begin(), R->src.end());
    R->dst_c.assign(R->dst.begin(), R->dst.end());
    return CSAW_OK;
}

csaw_status sample_batch(csaw_graph* g, const uint32_t* d_seeds, const uint64_t* d_inst_off, uint32_t n_inst,
                         uint64_t n_seeds, uint32_t depth, const uint32_t* fan_max, const SampleTables& t,
                         int kind, cudaStream_t s, csaw_sample_result** out)
{
    *out = nullptr;
    csaw_sample_result* R = new (std::nothrow) csaw_sample_result();
    if (!R) return fail(CSAW_ERR_NOMEM, "host allocation failed");
    R->depth = depth;
    R->n_instances = n_inst;
    const csaw_status st = run_sample(g, d_seeds, d_inst_off, n_inst, n_seeds, depth, fan_max, kind, 0,
                                      CSAW_ATTEMPT_CAP, false, s, R, &t);
    if (st != CSAW_OK) {
        cudaStreamSynchronize(s);
        delete R;
        return st;
    }
    *out = R;
    return CSAW_OK;
}

void free_sample_result_on(csaw_sample_result* R, cudaStream_t s)
{
    if (!R) return;
    for (std::vector<uint32_t*>* arrs : {&R->src, &R->dst})
        for (uint32_t*& p : *arrs) {
            if (p) {
                if (R->alloc.free) R->alloc.free(p, (void*)s, R->alloc.ctx);
                else cudaFreeAsync(p, s);
            }
            p = nullptr;
        }
    delete R;
}

}  // namespace csaw

using namespace csaw;

static csaw_status sample_entry(csaw_graph* g, const uint32_t* seeds, const uint64_t* inst_offsets,
                                uint32_t n_instances, uint32_t depth, const uint32_t* fanout,
                                const csaw_bias* bias, uint64_t rng_seed, int mem_kind, void* stream,
                                const csaw_sample_opts* opts, bool layer_mode, csaw_sample_result** out)
{
    clear_error();
    AllocScope alloc_scope(g);
    const uint32_t attempt_cap = opts ? opts->attempt_cap : CSAW_ATTEMPT_CAP;
    if (!out) return fail(CSAW_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!g) return fail(CSAW_ERR_INVALID, "graph is NULL");
    int kind;
    CSAW_TRY(check_bias(g, bias, false, &kind));
    if (depth < 1 || depth > CSAW_MAX_DEPTH) return fail(CSAW_ERR_INVALID, "depth must be 1..%u", CSAW_MAX_DEPTH);
    if (!fanout) return fail(CSAW_ERR_INVALID, "fanout is NULL");
    for (uint32_t l = 0; l < depth; ++l)
        if (fanout[l] == 0) return fail(CSAW_ERR_INVALID, "fanout[%u] is 0", l);
    if (!inst_offsets) return fail(CSAW_ERR_INVALID, "inst_offsets is NULL");
    if (mem_kind != CSAW_MEM_HOST && mem_kind != CSAW_MEM_DEVICE)
        return fail(CSAW_ERR_INVALID, "bad mem_kind %d", mem_kind);
    if (n_instances == 0xFFFFFFFFu) return fail(CSAW_ERR_INVALID, "too many instances");
    cudaStream_t s = (cudaStream_t)stream;

    csaw_sample_result* R = new (std::nothrow) csaw_sample_result();
    if (!R) return fail(CSAW_ERR_NOMEM, "host allocation failed");
    R->depth = depth;
    R->n_instances = n_instances;

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
        st = run_sample(g, d_seeds, d_io, n_instances, n_seeds, depth, fanout, kind, rng_seed, attempt_cap,
                        layer_mode, s, R);
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

extern "C" csaw_status csaw_sample_ex(csaw_graph* g, const uint32_t* seeds, const uint64_t* inst_offsets,
                                      uint32_t n_instances, uint32_t depth, const uint32_t* fanout,
                                      const csaw_bias* bias, uint64_t rng_seed, int mem_kind, void* stream,
                                      const csaw_sample_opts* opts, csaw_sample_result** out)
{
    return sample_entry(g, seeds, inst_offsets, n_instances, depth, fanout, bias, rng_seed, mem_kind, stream,
                        opts, false, out);
}

extern "C" csaw_status csaw_layer_sample(csaw_graph* g, const uint32_t* seeds, const uint64_t* inst_offsets,
                                         uint32_t n_instances, uint32_t depth, const uint32_t* layer_size,
                                         const csaw_bias* bias, uint64_t rng_seed, int mem_kind, void* stream,
                                         const csaw_sample_opts* opts, csaw_sample_result** out)
{
    return sample_entry(g, seeds, inst_offsets, n_instances, depth, layer_size, bias, rng_seed, mem_kind,
                        stream, opts, true, out);
}

extern "C" csaw_status csaw_sample(csaw_graph* g, const uint32_t* seeds, const uint64_t* inst_offsets,
                                   uint32_t n_instances, uint32_t depth, const uint32_t* fanout,
                                   const csaw_bias* bias, uint64_t rng_seed, int mem_kind, void* stream,
                                   csaw_sample_result** out)
{
    return csaw_sample_ex(g, seeds, inst_offsets, n_instances, depth, fanout, bias, rng_seed, mem_kind,
                          stream, nullptr, out);
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

// ---------------------------------------------------------------------------
// Sample plans: the whole multi-layer pipeline for a fixed instance count and
// seed budget, with every buffer at its upper bound, captured once into a
// CUDA graph.  Each run copies new seeds in and launches the graph: no host
// waits, no allocation, one launch for all instances and layers.

struct csaw_sample_plan {
    uint32_t magic = 0x43504c4eu;   // "CPLN"
    csaw::Pipeline P;
    std::vector<void*> allocs;
    DevAllocator alloc;       // the allocator of the buffers (the graph's at creation)
    uint32_t* in_seeds = nullptr;
    uint64_t* in_io = nullptr;
    uint32_t* in_key = nullptr;
    uint64_t max_seeds = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t last = nullptr;
    bool ran = false;
    std::vector<uint64_t> h_eoff, h_fsize, h_layer_edges;
    std::vector<const uint32_t*> src_c, dst_c;
    ~csaw_sample_plan()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (void* p : allocs) csaw::free_with(alloc, p, nullptr);
    }
};

namespace csaw {

static inline uint64_t sat_mul(uint64_t a, uint64_t b)
{
    if (a == 0 || b == 0) return 0;
    return a > UINT64_MAX / b ? UINT64_MAX : a * b;
}

}  // namespace csaw

extern "C" csaw_status csaw_sample_plan_create_ex(csaw_graph* g, uint32_t n_instances, uint64_t max_seeds,
                                                  uint32_t depth, const uint32_t* fanout, const csaw_bias* bias,
                                                  const csaw_sample_opts* opts, csaw_sample_plan** out)
{
    clear_error();
    if (!out) return fail(CSAW_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!g) return fail(CSAW_ERR_INVALID, "graph is NULL");
    int kind;
    CSAW_TRY(check_bias(g, bias, false, &kind));
    if (depth < 1 || depth > CSAW_MAX_DEPTH) return fail(CSAW_ERR_INVALID, "depth must be 1..%u", CSAW_MAX_DEPTH);
    if (!fanout) return fail(CSAW_ERR_INVALID, "fanout is NULL");
    for (uint32_t l = 0; l < depth; ++l)
        if (fanout[l] == 0) return fail(CSAW_ERR_INVALID, "fanout[%u] is 0", l);
    if (n_instances == 0 || n_instances == 0xFFFFFFFFu) return fail(CSAW_ERR_INVALID, "bad instance count");
    if (max_seeds == 0 || max_seeds >= 0xFFFFFFFFull) return fail(CSAW_ERR_INVALID, "bad seed budget");
    csaw_sample_plan* pl = new (std::nothrow) csaw_sample_plan();
    if (!pl) return fail(CSAW_ERR_NOMEM, "host allocation failed");
    Pipeline& P = pl->P;
    P.init(g, kind, n_instances, depth, fanout, 0);
    P.attempt_cap = opts ? opts->attempt_cap : CSAW_ATTEMPT_CAP;
    P.seeds_cap = max_seeds;
    pl->max_seeds = max_seeds;
    pl->alloc = g->allocator;
    auto get = [&](void** p, size_t bytes) -> csaw_status {
        CSAW_TRY(alloc_with(&pl->alloc, p, bytes ? bytes : 16, nullptr));
        pl->allocs.push_back(*p);
        return CSAW_OK;
    };
    csaw_status st = alloc_common(P, get);
    // Upper bounds: a layer emits at most min(k, max degree) edges per
    // frontier vertex; a frontier is at most the previous layer's edges and
    // at most one entry per (instance, vertex).
    uint64_t f = max_seeds, f_max = 0;
    const uint64_t fmax = sat_mul(n_instances, g->V);
    for (uint32_t l = 0; st == CSAW_OK && l < depth; ++l) {
        st = alloc_entries(P, l, f, get);
        if (f > f_max) f_max = f;
        const uint64_t e = P.edge_bound(l, f);
        if (st == CSAW_OK) st = alloc_edges(P, l, e, get, get);
        f = e < fmax ? e : fmax;
    }
    if (st == CSAW_OK && P.hub_order) st = alloc_hub(P, f_max, get);   // vertex order of hub items
    if (st == CSAW_OK && P.hub_path) {
        // shared hub prefix sums: at most every edge of the rows above
        // theta_w, and at most max degree per hub item
        st = alloc_hub(P, f_max, get);
        uint64_t e_hub = 0;
        unsigned long long* d_sum = nullptr;
        if (st == CSAW_OK) st = get((void**)&d_sum, sizeof(unsigned long long));
        if (st == CSAW_OK) {
            cudaError_t e = cudaMemset(d_sum, 0, sizeof(unsigned long long));
            if (e == cudaSuccess) {
                hub_edges_kernel<<<grid_for(g->V, 256, g->sm_count), 256>>>(g->off, g->V, P.theta_w, d_sum);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaMemcpy(&e_hub, d_sum, sizeof(uint64_t), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) st = cuda_fail(e, "hub edge count");
        }
        const uint64_t by_items = sat_mul(f_max, g->max_degree);
        P.hubS_cap = e_hub < by_items ? e_hub : by_items;
        if (st == CSAW_OK) st = get((void**)&P.hubS, sizeof(uint64_t) * (P.hubS_cap ? P.hubS_cap : 1));
    }
    if (st == CSAW_OK) st = get((void**)&pl->in_seeds, sizeof(uint32_t) * max_seeds);
    if (st == CSAW_OK) st = get((void**)&pl->in_io, sizeof(uint64_t) * ((size_t)n_instances + 1));
    if (st == CSAW_OK) st = get((void**)&pl->in_key, 2 * sizeof(uint32_t));
    if (st != CSAW_OK) { delete pl; return st; }
    P.key_dev = pl->in_key;
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete pl; return cuda_fail(e, "cudaStreamCreate"); }
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        e = cudaMemsetAsync(P.ctr, 0, sizeof(uint64_t) * CT_WORDS, cs);
        if (e != cudaSuccess) st = cuda_fail(e, "memset");
        if (st == CSAW_OK) st = enqueue_frontier0(P, pl->in_seeds, pl->in_io, cs);
        for (uint32_t l = 0; st == CSAW_OK && l < depth; ++l) {
            st = enqueue_count(P, l, cs);
            if (st == CSAW_OK) st = enqueue_select(P, l, cs);
            if (st == CSAW_OK && l + 1 < depth) st = enqueue_compact(P, l, cs);
        }
        cudaGraph_t gr = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
        if (st == CSAW_OK && e2 != cudaSuccess) st = cuda_fail(e2, "cudaStreamEndCapture");
        if (st == CSAW_OK) {
            pl->graph = gr;
            e2 = cudaGraphInstantiate(&pl->exec, gr, 0);
            if (e2 != cudaSuccess) st = cuda_fail(e2, "cudaGraphInstantiate");
        } else if (gr) {
            cudaGraphDestroy(gr);
        }
    } else {
        st = cuda_fail(e, "cudaStreamBeginCapture");
    }
    cudaStreamDestroy(cs);
    if (st != CSAW_OK) { delete pl; return st; }
    *out = pl;
    return CSAW_OK;
}

extern "C" csaw_status csaw_sample_plan_create(csaw_graph* g, uint32_t n_instances, uint64_t max_seeds,
                                               uint32_t depth, const uint32_t* fanout, const csaw_bias* bias,
                                               csaw_sample_plan** out)
{
    return csaw_sample_plan_create_ex(g, n_instances, max_seeds, depth, fanout, bias, nullptr, out);
}

extern "C" csaw_status csaw_sample_plan_run(csaw_sample_plan* pl, const uint32_t* seeds, uint64_t n_seeds,
                                            const uint64_t* inst_offsets, uint64_t rng_seed, int mem_kind,
                                            void* stream)
{
    clear_error();
    if (!pl) return fail(CSAW_ERR_INVALID, "plan is NULL");
    if (!inst_offsets || (n_seeds && !seeds)) return fail(CSAW_ERR_INVALID, "NULL input");
    if (n_seeds > pl->max_seeds)
        return fail(CSAW_ERR_INVALID, "%llu seeds, plan holds %llu", (unsigned long long)n_seeds,
                    (unsigned long long)pl->max_seeds);
    if (mem_kind != CSAW_MEM_HOST && mem_kind != CSAW_MEM_DEVICE)
        return fail(CSAW_ERR_INVALID, "bad mem_kind %d", mem_kind);
    const uint32_t n_inst = pl->P.n_inst;
    if (mem_kind == CSAW_MEM_HOST) {
        if (inst_offsets[0] != 0 || inst_offsets[n_inst] != n_seeds)
            return fail(CSAW_ERR_INVALID, "inst_offsets must run from 0 to n_seeds");
        for (uint32_t i = 0; i < n_inst; ++i)
            if (inst_offsets[i + 1] < inst_offsets[i]) return fail(CSAW_ERR_INVALID, "inst_offsets must be non-decreasing");
        for (uint64_t j = 0; j < n_seeds; ++j)
            if (seeds[j] >= pl->P.g->V) return fail(CSAW_ERR_INVALID, "seed %llu out of range", (unsigned long long)j);
    }
    cudaStream_t s = (cudaStream_t)stream;
    const cudaMemcpyKind k = mem_kind == CSAW_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const uint32_t key[2] = {(uint32_t)rng_seed, (uint32_t)(rng_seed >> 32)};
    if (n_seeds) CSAW_CUDA(cudaMemcpyAsync(pl->in_seeds, seeds, sizeof(uint32_t) * n_seeds, k, s));
    CSAW_CUDA(cudaMemcpyAsync(pl->in_io, inst_offsets, sizeof(uint64_t) * ((size_t)n_inst + 1), k, s));
    CSAW_CUDA(cudaMemcpyAsync(pl->in_key, key, sizeof(key), cudaMemcpyHostToDevice, s));
    CSAW_CUDA(cudaGraphLaunch(pl->exec, s));
    pl->last = s;
    pl->ran = true;
    return CSAW_OK;
}

// Wait for the plan's last run and read its offsets and sizes.
static csaw_status plan_collect(csaw_sample_plan* pl)
{
    if (!pl->ran) return fail(CSAW_ERR_INVALID, "the plan has not run");
    Pipeline& P = pl->P;
    CSAW_CUDA(cudaStreamSynchronize(pl->last));
    const uint64_t ng = (uint64_t)P.depth * P.n_inst;
    pl->h_eoff.assign(ng + 1, 0);
    pl->h_fsize.assign(ng ? ng : 1, 0);
    std::vector<uint64_t> ctr(CT_WORDS, 0);
    CSAW_CUDA(cudaMemcpy(ctr.data(), P.ctr, sizeof(uint64_t) * CT_WORDS, cudaMemcpyDeviceToHost));
    CSAW_TRY(check_errors(ctr[CT_ERR]));
    CSAW_CUDA(cudaMemcpy(pl->h_eoff.data(), P.eoff, sizeof(uint64_t) * (ng + 1), cudaMemcpyDeviceToHost));
    if (ng) CSAW_CUDA(cudaMemcpy(pl->h_fsize.data(), P.fsize, sizeof(uint64_t) * ng, cudaMemcpyDeviceToHost));
    pl->h_layer_edges.assign(P.depth, 0);
    for (uint32_t l = 0; l < P.depth; ++l) pl->h_layer_edges[l] = ctr[CT_LAYER + L_WORDS * l + L_TOTAL];
    pl->src_c.assign(P.depth, nullptr);
    pl->dst_c.assign(P.depth, nullptr);
    for (uint32_t l = 0; l < P.depth; ++l) { pl->src_c[l] = P.L[l].src; pl->dst_c[l] = P.L[l].dst; }
    return CSAW_OK;
}

extern "C" csaw_status csaw_sample_plan_get_view(csaw_sample_plan* pl, csaw_sample_view* view)
{
    clear_error();
    if (!pl || !view) return fail(CSAW_ERR_INVALID, "NULL argument");
    CSAW_TRY(plan_collect(pl));
    view->depth = pl->P.depth;
    view->n_instances = pl->P.n_inst;
    view->n_edges = pl->h_eoff.back();
    view->edge_offsets = pl->h_eoff.data();
    view->frontier_sizes = pl->h_fsize.data();
    view->src = pl->src_c.data();
    view->dst = pl->dst_c.data();
    return CSAW_OK;
}

extern "C" csaw_status csaw_sample_plan_copy_edges(csaw_sample_plan* pl, uint32_t* src, uint32_t* dst)
{
    clear_error();
    if (!pl) return fail(CSAW_ERR_INVALID, "plan is NULL");
    CSAW_TRY(plan_collect(pl));
    uint64_t at = 0;
    for (uint32_t l = 0; l < pl->P.depth; ++l) {
        const uint64_t n = pl->h_layer_edges[l];
        if (n) {
            if (!src || !dst) return fail(CSAW_ERR_INVALID, "NULL output");
            CSAW_CUDA(cudaMemcpy(src + at, pl->P.L[l].src, n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
            CSAW_CUDA(cudaMemcpy(dst + at, pl->P.L[l].dst, n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
        }
        at += n;
    }
    return CSAW_OK;
}

extern "C" csaw_status csaw_sample_plan_get_info(const csaw_sample_plan* pl, uint64_t* device_bytes,
                                                 uint32_t* theta_warp, uint32_t* select_blocks)
{
    clear_error();
    if (!pl) return fail(CSAW_ERR_INVALID, "plan is NULL");
    if (device_bytes) {
        uint64_t b = 0;
        // sizes are not recorded per allocation; report capacities
        const Pipeline& P = pl->P;
        for (uint32_t l = 0; l < P.depth; ++l)
            b += P.L[l].f_cap * 28 + P.L[l].e_cap * (8 + (l + 1 < P.depth ? 28 : 0));
        b += P.seeds_cap * 28 + pl->max_seeds * 4;
        *device_bytes = b;
    }
    if (theta_warp) *theta_warp = pl->P.theta_w;
    if (select_blocks) *select_blocks = (uint32_t)pl->P.sel_blocks;
    return CSAW_OK;
}

extern "C" csaw_status csaw_sample_plan_destroy(csaw_sample_plan* pl)
{
    clear_error();
    if (pl && pl->ran) cudaStreamSynchronize(pl->last);
    delete pl;
    return CSAW_OK;
}

// ---------------------------------------------------------------------------
// Layered sampling over a graph kept in host memory (out-of-memory sampling,
// Sec. V-A; partitions loaded in the background while others are sampled,
// Sec. V-B).  The CSR stays in host memory, cut into vertex ranges whose
// columns (and weights), plus room for their shared hub prefix sums, fit one
// device slot of the budget.  The row offsets and the degrees stay resident
// (16 bytes per vertex beyond the budget), so each layer's counts and edge
// positions are computed once; then the partitions holding frontier vertices
// are taken in the order of how many entries they hold (workload-aware
// scheduling, Sec. V-A), and for each one the selection kernels run over the
// entries whose vertex lies in it, with the column and weight bases pointed
// into the slot.  With two or more slots the next partition's copies run on
// their own stream while the current one is sampled.  Draws, prefix sums and
// output are those of csaw_sample: results are identical.

namespace csaw {

// Frontier entries of positive degree per partition (bounds vb[0..np]).
__global__ void oom_part_count_kernel(const uint64_t* __restrict__ fkeys, const unsigned long long* n_dev,
                                      uint64_t vmask, const uint64_t* __restrict__ off,
                                      const uint32_t* __restrict__ vb, uint32_t np,
                                      unsigned long long* __restrict__ counts)
{
    const uint64_t n = *n_dev;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)(fkeys[e] & vmask);
        if (off[v + 1] == off[v]) continue;
        uint32_t lo = 0, hi = np;   // last q with vb[q] <= v
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (vb[mid] <= v) lo = mid; else hi = mid;
        }
        atomicAdd(counts + lo, 1ull);
    }
}

__global__ void degrees_kernel(const uint64_t* __restrict__ off, uint32_t V, uint32_t* __restrict__ deg)
{
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t d = off[v + 1] - off[v];
        deg[v] = (uint32_t)(d > 0xFFFFFFFFull ? 0xFFFFFFFFull : d);
    }
}

// One device slot of the out-of-memory sampler.
struct OomSlot {
    uint32_t* col = nullptr;
    uint32_t* w = nullptr;
    uint64_t* hubS = nullptr;
    int64_t part = -1;                 // partition it holds
    cudaEvent_t loaded = nullptr;      // its copies are done
    cudaEvent_t freed = nullptr;       // the selection that read it is done
};

}  // namespace csaw

extern "C" csaw_status csaw_sample_oom(const uint64_t* row_offsets, const uint32_t* cols, const uint32_t* weights,
                                       uint32_t n_vertices, uint64_t n_edges, uint64_t device_budget_bytes,
                                       const uint32_t* seeds, const uint64_t* inst_offsets, uint32_t n_instances,
                                       uint32_t depth, const uint32_t* fanout, const csaw_bias* bias,
                                       uint64_t rng_seed, const csaw_oom_opts* opts, csaw_oom_stats* stats,
                                       void* stream, csaw_sample_result** out)
{
    clear_error();
    if (stats) *stats = csaw_oom_stats{};
    if (!out) return fail(CSAW_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!row_offsets || (n_edges && !cols) || !inst_offsets || !fanout || !bias)
        return fail(CSAW_ERR_INVALID, "NULL argument");
    const int kind = bias->kind;
    if (kind != CSAW_BIAS_UNIFORM && kind != CSAW_BIAS_EDGE_WEIGHT && kind != CSAW_BIAS_NEIGHBOR_DEGREE)
        return fail(CSAW_ERR_INVALID, "out-of-memory sampling takes uniform, edge-weight or neighbour-degree bias");
    const int eff_kind = (kind == CSAW_BIAS_EDGE_WEIGHT && !weights) ? CSAW_BIAS_UNIFORM : kind;
    const bool weighted = eff_kind == CSAW_BIAS_EDGE_WEIGHT;
    if (depth < 1 || depth > CSAW_MAX_DEPTH) return fail(CSAW_ERR_INVALID, "depth must be 1..%u", CSAW_MAX_DEPTH);
    for (uint32_t l = 0; l < depth; ++l)
        if (fanout[l] == 0) return fail(CSAW_ERR_INVALID, "fanout[%u] is 0", l);
    if (n_instances == 0xFFFFFFFFu) return fail(CSAW_ERR_INVALID, "too many instances");
    const uint32_t n_slots = opts && opts->slots ? opts->slots : 2;
    if (n_slots > 8) return fail(CSAW_ERR_INVALID, "at most 8 slots");
    // host validation: the CSR, the seeds, and positive biases (the count of
    // positive biases is the degree, so counts need no partition)
    if (n_vertices == 0 || row_offsets[0] != 0 || row_offsets[n_vertices] != n_edges)
        return fail(CSAW_ERR_INVALID, "row_offsets must run from 0 to n_edges");
    uint32_t max_degree = 0;
    for (uint32_t v = 0; v < n_vertices; ++v) {
        if (row_offsets[v + 1] < row_offsets[v]) return fail(CSAW_ERR_INVALID, "row_offsets must not decrease");
        const uint64_t d = row_offsets[v + 1] - row_offsets[v];
        if (d > 0xFFFFFFFFull) return fail(CSAW_ERR_INVALID, "row %u longer than 2^32-1", v);
        if (d > max_degree) max_degree = (uint32_t)d;
    }
    // columns, weights and (neighbour degree) edge targets are checked on
    // the device as each partition arrives; the largest weight only sizes
    // the walk kernels' sums, which sampling does not use
    const uint32_t max_weight = 0xFFFFFFFFu;
    if (inst_offsets[0] != 0) return fail(CSAW_ERR_INVALID, "inst_offsets must start at 0");
    for (uint32_t i = 0; i < n_instances; ++i)
        if (inst_offsets[i + 1] < inst_offsets[i]) return fail(CSAW_ERR_INVALID, "inst_offsets must be non-decreasing");
    const uint64_t n_seeds = inst_offsets[n_instances];
    if (n_seeds >= 0xFFFFFFFFull) return fail(CSAW_ERR_INVALID, "too many seeds");
    if (n_seeds && !seeds) return fail(CSAW_ERR_INVALID, "seeds is NULL");
    for (uint64_t j = 0; j < n_seeds; ++j)
        if (seeds[j] >= n_vertices) return fail(CSAW_ERR_INVALID, "seed %llu out of range", (unsigned long long)j);

    // partitions: columns, weights and hub prefix sums (16 bytes per edge)
    uint32_t np = 0;
    CSAW_TRY(csaw_oom_plan(row_offsets, n_vertices, 1, device_budget_bytes, nullptr, 0, &np));
    std::vector<uint32_t> vb((size_t)np + 1);
    CSAW_TRY(csaw_oom_plan(row_offsets, n_vertices, 1, device_budget_bytes, vb.data(), np + 1, &np));
    uint64_t slot_edges = 1;
    for (uint32_t q = 0; q < np; ++q)
        slot_edges = std::max<uint64_t>(slot_edges, row_offsets[vb[q + 1]] - row_offsets[vb[q]]);

    cudaStream_t s = (cudaStream_t)stream;
    int device = 0;
    CSAW_CUDA(cudaGetDevice(&device));
    csaw_graph view;   // resident offsets and degrees; columns and weights point into a slot per round
    view.V = n_vertices;
    view.E = n_edges;
    view.max_degree = max_degree;
    view.max_weight = max_weight;
    view.min_weight = 1;
    view.zero_degree_target = false;
    view.device = device;
    CSAW_CUDA(cudaDeviceGetAttribute(&view.sm_count, cudaDevAttrMultiProcessorCount, device));

    csaw_sample_result* R = new (std::nothrow) csaw_sample_result();
    if (!R) return fail(CSAW_ERR_NOMEM, "host allocation failed");
    R->depth = depth;
    R->n_instances = n_instances;
    R->stream = s;
    std::vector<OomSlot> slot(n_slots);
    cudaStream_t cs = nullptr;   // copies
    Temps tmp(s);
    auto get = [&](void** p, size_t bytes) -> csaw_status {
        CSAW_TRY(dalloc(p, bytes, s));
        tmp.ptrs.push_back(*p);
        return CSAW_OK;
    };
    auto get_out = [&](void** p, size_t bytes) -> csaw_status { return dalloc(p, bytes, s); };
    csaw_oom_stats acc{};
    acc.partitions = np;
    bool registered_col = false, registered_w = false;
    csaw_status st = CSAW_OK;
    do {
        // pinned (registered) host arrays let the copies run behind the selection
        if (opts && opts->pin_host && n_edges) {
            registered_col = host_register((void*)cols, sizeof(uint32_t) * n_edges);
            if (weighted)
                registered_w = host_register((void*)weights, sizeof(uint32_t) * n_edges);
            cudaGetLastError();   // a refused registration leaves ordinary (pageable) copies
        }
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaStreamCreate"); break; }
        for (auto& sl : slot) {
            st = get((void**)&sl.col, sizeof(uint32_t) * slot_edges);
            if (st == CSAW_OK && weighted) st = get((void**)&sl.w, sizeof(uint32_t) * slot_edges);
            if (st == CSAW_OK) st = get((void**)&sl.hubS, sizeof(uint64_t) * slot_edges);
            if (st != CSAW_OK) break;
            e = cudaEventCreateWithFlags(&sl.loaded, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.freed, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(sl.freed, s);
            if (e != cudaSuccess) { st = cuda_fail(e, "cudaEvent"); break; }
        }
        if (st != CSAW_OK) break;
        uint64_t* d_off = nullptr;
        uint32_t* d_deg = nullptr;
        uint32_t* d_vb = nullptr;
        unsigned long long* d_pc = nullptr;
        uint32_t* d_chk = nullptr;
        void* d_seeds = nullptr;
        void* d_io = nullptr;
        st = get((void**)&d_off, sizeof(uint64_t) * ((uint64_t)n_vertices + 1));
        if (st == CSAW_OK) st = get((void**)&d_deg, sizeof(uint32_t) * n_vertices);
        if (st == CSAW_OK) st = get((void**)&d_vb, sizeof(uint32_t) * (np + 1));
        if (st == CSAW_OK) st = get((void**)&d_pc, sizeof(unsigned long long) * np);
        if (st == CSAW_OK) st = get((void**)&d_chk, sizeof(uint32_t));
        if (st == CSAW_OK) st = get(&d_seeds, sizeof(uint32_t) * (n_seeds ? n_seeds : 1));
        if (st == CSAW_OK) st = get(&d_io, sizeof(uint64_t) * ((uint64_t)n_instances + 1));
        if (st != CSAW_OK) break;
        e = cudaMemcpyAsync(d_off, row_offsets, sizeof(uint64_t) * ((uint64_t)n_vertices + 1), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_vb, vb.data(), sizeof(uint32_t) * (np + 1), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && n_seeds) e = cudaMemcpyAsync(d_seeds, seeds, sizeof(uint32_t) * n_seeds, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_io, inst_offsets, sizeof(uint64_t) * ((uint64_t)n_instances + 1), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_chk, 0, sizeof(uint32_t), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // before the copy stream uses them
        if (e != cudaSuccess) { st = cuda_fail(e, "copy inputs"); break; }
        degrees_kernel<<<grid_for(n_vertices, 256, view.sm_count), 256, 0, s>>>(d_off, n_vertices, d_deg);
        view.off = d_off;
        view.deg = d_deg;
        view.col = slot[0].col;
        view.w = weighted ? slot[0].w : nullptr;

        Pipeline P;
        P.init(&view, eff_kind, n_instances, depth, fanout, rng_seed);
        P.seeds_cap = n_seeds;
        st = alloc_common(P, get);
        if (st == CSAW_OK) {
            e = cudaMemsetAsync(P.ctr, 0, sizeof(uint64_t) * CT_WORDS, s);
            if (e != cudaSuccess) st = cuda_fail(e, "memset");
        }
        if (st == CSAW_OK) st = alloc_entries(P, 0, n_seeds, get);
        if (st == CSAW_OK) st = enqueue_frontier0(P, (const uint32_t*)d_seeds, (const uint64_t*)d_io, s);
        if (st != CSAW_OK) break;
        R->src.assign(depth, nullptr);
        R->dst.assign(depth, nullptr);
        R->layer_edges.assign(depth, 0);
        std::vector<unsigned long long> pc(np);
        for (uint32_t l = 0; st == CSAW_OK && l < depth; ++l) {
            LayerBufs& B = P.L[l];
            Temps layer_tmp(s);
            auto get_layer = [&](void** p, size_t bytes) -> csaw_status {
                CSAW_TRY(dalloc(p, bytes, s));
                layer_tmp.ptrs.push_back(*p);
                return CSAW_OK;
            };
            if (P.hub_path) st = alloc_hub(P, B.f_cap, get_layer);
            // counts and edge positions of every entry (degrees are resident)
            if (st == CSAW_OK) st = enqueue_classify(P, l, 0, 0, true, s);
            if (st == CSAW_OK) st = scan_u32(B.cnt, B.pos, P.lc(l, L_N), B.f_cap, P.scan_scr, P.lc(l, L_TOTAL), s);
            if (st != CSAW_OK) break;
            e = cudaMemsetAsync(d_pc, 0, sizeof(unsigned long long) * np, s);
            if (e == cudaSuccess && B.f_cap)
                oom_part_count_kernel<<<grid_for(B.f_cap, 256, view.sm_count), 256, 0, s>>>(
                    B.F, (const unsigned long long*)P.lc(l, L_N), P.vmask, d_off, d_vb, np, d_pc);
            uint64_t h[2] = {0, 0};
            if (e == cudaSuccess) e = cudaMemcpyAsync(pc.data(), d_pc, sizeof(unsigned long long) * np, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&h[0], P.ctr + CT_ERR, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&h[1], P.lc(l, L_TOTAL), sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { st = cuda_fail(e, "layer counts"); break; }
            st = check_errors(h[0]);
            if (st != CSAW_OK) break;
            const uint64_t total = h[1];
            R->layer_edges[l] = total;
            st = alloc_edges(P, l, total, get, get_out);
            if (st != CSAW_OK) break;
            R->src[l] = P.L[l].src;
            R->dst[l] = P.L[l].dst;
            // workload-aware order: the partitions with the most frontier entries first
            std::vector<uint32_t> order;
            for (uint32_t q = 0; q < np; ++q)
                if (pc[q]) order.push_back(q);
            std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return pc[a] > pc[b]; });
            // slot of each round: a partition already resident keeps its slot
            std::vector<int> use(order.size(), -1);
            auto load = [&](size_t i) -> csaw_status {
                const uint32_t q = order[i];
                for (uint32_t k = 0; k < n_slots; ++k)
                    if (slot[k].part == (int64_t)q) { use[i] = (int)k; ++acc.reuses; return CSAW_OK; }
                // the slot least recently needed: round i uses slot i mod n_slots
                // unless that one holds the partition of round i - 1
                uint32_t k = (uint32_t)(i % n_slots);
                if (i > 0 && (int)k == use[i - 1]) k = (k + 1) % n_slots;
                OomSlot& sl = slot[k];
                const uint64_t e0 = row_offsets[vb[q]], ne = row_offsets[vb[q + 1]] - e0;
                cudaError_t ce = cudaStreamWaitEvent(cs, sl.freed, 0);
                if (ce == cudaSuccess && ne)
                    ce = cudaMemcpyAsync(sl.col, cols + e0, sizeof(uint32_t) * ne, cudaMemcpyHostToDevice, cs);
                if (ce == cudaSuccess && weighted && ne)
                    ce = cudaMemcpyAsync(sl.w, weights + e0, sizeof(uint32_t) * ne, cudaMemcpyHostToDevice, cs);
                if (ce == cudaSuccess) {
                    launch_partition_check(sl.col, weighted ? sl.w : nullptr, ne, n_vertices,
                                           eff_kind == CSAW_BIAS_NEIGHBOR_DEGREE ? d_deg : nullptr, d_chk, cs);
                    ce = cudaGetLastError();
                }
                if (ce == cudaSuccess) ce = cudaEventRecord(sl.loaded, cs);
                if (ce != cudaSuccess) return cuda_fail(ce, "partition copy");
                sl.part = q;
                use[i] = (int)k;
                acc.loads += 1;
                acc.bytes_loaded += ne * (weighted ? 8 : 4);
                return CSAW_OK;
            };
            if (!order.empty()) st = load(0);
            for (size_t i = 0; st == CSAW_OK && i < order.size(); ++i) {
                const uint32_t q = order[i];
                OomSlot& sl = slot[use[i]];
                const uint64_t e0 = row_offsets[vb[q]];
                e = cudaStreamWaitEvent(s, sl.loaded, 0);
                // the round's item counters start at zero
                if (e == cudaSuccess)
                    e = cudaMemsetAsync(P.lc(l, L_ITEMS), 0, sizeof(uint64_t) * (L_HNEXT + 2 - L_ITEMS), s);
                if (e != cudaSuccess) { st = cuda_fail(e, "round"); break; }
                // rows of [vb[q], vb[q+1]) hold edges e0 ..; the slot holds them from 0
                view.col = sl.col - e0;
                view.w = weighted ? sl.w - e0 : nullptr;
                P.hubS = sl.hubS;
                P.hubS_cap = slot_edges;
                st = enqueue_classify(P, l, vb[q], vb[q + 1], false, s);
                if (st == CSAW_OK && P.hub_path) st = enqueue_hub_groups(P, l, s);
                if (st == CSAW_OK) st = enqueue_select_items(P, l, s);
                if (st != CSAW_OK) break;
                e = cudaEventRecord(sl.freed, s);
                if (e != cudaSuccess) { st = cuda_fail(e, "round"); break; }
                // the next round's copies run while this round's selection does
                if (i + 1 < order.size()) st = load(i + 1);
            }
            if (st == CSAW_OK) st = enqueue_layer_offsets(P, l, s);
            if (st == CSAW_OK && l + 1 < depth) {
                st = alloc_entries(P, l + 1, total, get);
                if (st == CSAW_OK) st = enqueue_compact(P, l, s);
            }
        }
        if (st != CSAW_OK) break;
        const uint64_t ng = (uint64_t)depth * n_instances;
        R->edge_offsets.assign(ng + 1, 0);
        R->frontier_sizes.assign(ng, 0);
        uint64_t err_end = 0;
        if (ng) {
            e = cudaMemcpyAsync(R->edge_offsets.data(), P.eoff, sizeof(uint64_t) * (ng + 1), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(R->frontier_sizes.data(), P.fsize, sizeof(uint64_t) * ng, cudaMemcpyDeviceToHost, s);
        }
        uint32_t chk = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&err_end, P.ctr + CT_ERR, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&chk, d_chk, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { st = cuda_fail(e, "out-of-memory sampling"); break; }
        if (chk & 1u) { st = fail(CSAW_ERR_INVALID, "a column is not a vertex of the graph"); break; }
        if (chk & 2u) { st = fail(CSAW_ERR_INVALID, "out-of-memory sampling needs positive weights"); break; }
        if (chk & 4u) {
            st = fail(CSAW_ERR_INVALID, "neighbour-degree bias: an edge points at a vertex without neighbours");
            break;
        }
        st = check_errors(err_end);
        if (st != CSAW_OK) break;
        uint64_t tot = 0;
        for (uint32_t l = 0; l < depth; ++l) tot += R->layer_edges[l];
        R->n_edges = tot;
        R->edge_offsets[ng] = tot;
        R->src_c.assign(R->src.begin(), R->src.end());
        R->dst_c.assign(R->dst.begin(), R->dst.end());
    } while (false);
    cudaStreamSynchronize(s);
    if (cs) {
        cudaStreamSynchronize(cs);
        cudaStreamDestroy(cs);
    }
    for (auto& sl : slot) {
        if (sl.loaded) cudaEventDestroy(sl.loaded);
        if (sl.freed) cudaEventDestroy(sl.freed);
    }
    acc.pinned_bytes = (registered_col ? sizeof(uint32_t) * n_edges : 0) + (registered_w ? sizeof(uint32_t) * n_edges : 0);
    if (registered_col) cudaHostUnregister((void*)cols);
    if (registered_w) cudaHostUnregister((void*)weights);
    if (st != CSAW_OK) {
        delete R;
        return st;
    }
    if (stats) *stats = acc;
    *out = R;
    return CSAW_OK;
}

// ---------------------------------------------------------------------------
// Launch-shape tuning of the selection path.

extern "C" csaw_status csaw_set_select_tuning(csaw_graph* g, int32_t bias_kind, const csaw_select_tuning* t)
{
    clear_error();
    if (!g || !t) return fail(CSAW_ERR_INVALID, "NULL argument");
    if (bias_kind < 0 || bias_kind > CSAW_BIAS_NEIGHBOR_DEGREE) return fail(CSAW_ERR_INVALID, "bad bias kind");
    if (t->theta_warp > WARP_MAX_DEG) return fail(CSAW_ERR_INVALID, "theta_warp above %u", WARP_MAX_DEG);
    g->tune_theta_w[bias_kind] = t->theta_warp;
    g->tune_blocks_per_sm[bias_kind] = t->blocks_per_sm;
    return CSAW_OK;
}

extern "C" csaw_status csaw_get_select_tuning(const csaw_graph* g, int32_t bias_kind, csaw_select_tuning* t)
{
    clear_error();
    if (!g || !t) return fail(CSAW_ERR_INVALID, "NULL argument");
    if (bias_kind < 0 || bias_kind > CSAW_BIAS_NEIGHBOR_DEGREE) return fail(CSAW_ERR_INVALID, "bad bias kind");
    uint32_t tw;
    int blocks;
    select_shape(g, bias_kind, &tw, &blocks);
    t->theta_warp = tw;
    t->blocks_per_sm = (uint32_t)(blocks / (g->sm_count > 0 ? g->sm_count : 1));
    return CSAW_OK;
}

extern "C" csaw_status csaw_autotune_select(csaw_graph* g, const uint32_t* seeds, const uint64_t* inst_offsets,
                                            uint32_t n_instances, uint32_t depth, const uint32_t* fanout,
                                            const csaw_bias* bias, uint64_t rng_seed, void* stream,
                                            csaw_select_tuning* best)
{
    clear_error();
    if (!g || !best) return fail(CSAW_ERR_INVALID, "NULL argument");
    int kind;
    CSAW_TRY(check_bias(g, bias, false, &kind));
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t thetas[] = {32, 64, 128, 256};
    const int occ = select_occupancy(kind);
    cudaEvent_t e0, e1;
    CSAW_CUDA(cudaEventCreate(&e0));
    CSAW_CUDA(cudaEventCreate(&e1));
    float best_ms = -1.f;
    csaw_select_tuning bt = {WARP_MAX_DEG, (uint32_t)occ};
    const uint32_t saved_t = g->tune_theta_w[kind], saved_b = g->tune_blocks_per_sm[kind];
    csaw_status st = CSAW_OK;
    for (uint32_t th : thetas) {
        for (int per = 1; per <= occ && st == CSAW_OK; ++per) {
            g->tune_theta_w[kind] = th;
            g->tune_blocks_per_sm[kind] = (uint32_t)per;
            float ms = 0.f;
            for (int rep = 0; rep < 2 && st == CSAW_OK; ++rep) {   // first run warms up
                csaw_sample_result* r = nullptr;
                cudaEventRecord(e0, s);
                st = csaw_sample(g, seeds, inst_offsets, n_instances, depth, fanout, bias, rng_seed,
                                 CSAW_MEM_HOST, stream, &r);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
                delete r;
            }
            if (st == CSAW_OK && (best_ms < 0.f || ms < best_ms)) {
                best_ms = ms;
                bt.theta_warp = th;
                bt.blocks_per_sm = (uint32_t)per;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != CSAW_OK) {
        g->tune_theta_w[kind] = saved_t;
        g->tune_blocks_per_sm[kind] = saved_b;
        return st;
    }
    g->tune_theta_w[kind] = bt.theta_warp;
    g->tune_blocks_per_sm[kind] = bt.blocks_per_sm;
    *best = bt;
    return CSAW_OK;
}

// ---------------------------------------------------------------------------
// Results returned by this library start with a tag naming their type.

extern "C" csaw_status csaw_selection_stats(uint64_t counters[8], int reset)
{
    clear_error();
    if (!counters) return fail(CSAW_ERR_INVALID, "counters is NULL");
#ifdef CSAW_STATS
    CSAW_CUDA(cudaDeviceSynchronize());
    CSAW_CUDA(cudaMemcpyFromSymbol(counters, csaw::g_sel_stats, sizeof(uint64_t) * 8));
    if (reset) {
        const unsigned long long zero[8] = {};
        CSAW_CUDA(cudaMemcpyToSymbol(csaw::g_sel_stats, zero, sizeof(zero)));
    }
    return CSAW_OK;
#else
    (void)reset;
    for (int i = 0; i < 8; ++i) counters[i] = 0;
    return fail(CSAW_ERR_INVALID, "this library was built without selection counters (CSAW_STATS)");
#endif
}

extern "C" void csaw_result_free(void* result)
{
    if (!result) return;
    const uint32_t tag = *(const uint32_t*)result;
    if (tag == 0x43534d50u) delete (csaw_sample_result*)result;
    else csaw::free_server_result(result);
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
    if (device != g->device)
        return fail(CSAW_ERR_INVALID, "the current device (%d) is not the graph's device (%d)", device,
                    g->device);
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
    cp.n_items = d_items; cp.theta_w = WARP_MAX_DEG; cp.cached = false;
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
        sp.k0 = (uint32_t)rng_seed; sp.k1 = (uint32_t)(rng_seed >> 32); sp.key_dev = nullptr;
        sp.zero_bias = zero_bias; sp.pos = out_offsets; sp.warp_list = wlist; sp.cta_list = clist;
        sp.n_items = d_items; sp.next = d_items + 2;
        sp.out_src = out_src; sp.out_dst = out_dst; sp.out_cand = nullptr;
        sp.scratch_S = (uint64_t*)hub;
        sp.scratch_bits = (uint32_t*)(hub + (size_t)sel_blocks * g->max_degree * 8);
        sp.scratch_stride = g->max_degree;
        sp.cdf = nullptr; sp.skip_warp_items = false; sp.attempt_cap = CSAW_ATTEMPT_CAP;
        switch (kind) {
        case CSAW_BIAS_UNIFORM: CSAW_TRY(launch_select<CSAW_BIAS_UNIFORM>(sp, sel_blocks, s)); break;
        case CSAW_BIAS_EDGE_WEIGHT: CSAW_TRY(launch_select<CSAW_BIAS_EDGE_WEIGHT>(sp, sel_blocks, s)); break;
        default: CSAW_TRY(launch_select<CSAW_BIAS_NEIGHBOR_DEGREE>(sp, sel_blocks, s)); break;
        }
    }
    return CSAW_OK;
}
