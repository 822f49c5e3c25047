// csaw_walk.cu -- biased random walks (Sec. II-A), one warp per walker.
//
// A walk step at vertex v with degree d is inverse transform sampling over
// v's neighbour list (Sec. II-B, Eq. 1) with a single draw, so the cumulative
// bias array never has to be stored: the warp streams the biases once to get
// the total T (keeping one running prefix per chunk in shared memory), maps
// the draw to x in [0, T), then rescans only the chunk that holds x.  Biases
// are read as 16-byte groups of four (a round is 4 groups per lane, 512
// neighbours per warp; interior rounds skip every bounds check); a lane sums
// its sixteen in 32 bits and the warp
// reduces with one redux.sync when the largest possible bias times 512 stays
// below 2^32 (64-bit otherwise).  Locating x inside a 128-neighbour tile takes
// one warp scan of per-lane sums and a four-step search in the hit lane.
// Rows that fit one round stay in registers and need one pass.
//
// Work distribution: a persistent grid; each warp takes the next walker from
// a global counter and runs all its steps.  (Walks over a cached cumulative
// array are in csaw_walk_cdf.cu.)  The path row is buffered one
// 32-entry block per warp (lane j holds entry 32*blk + j) and written with
// one coalesced store per block.
#include <atomic>

#include "csaw_internal.cuh"

namespace csaw {

constexpr int WALK_THREADS = 256;
constexpr int WALK_WARPS = WALK_THREADS / 32;
constexpr uint32_t TILE = 128;              // neighbours per 16-byte load across the warp
#ifndef CSAW_WALK_U
#define CSAW_WALK_U 4
#endif
constexpr int U = CSAW_WALK_U;              // tiles per round (U loads in flight per lane)
constexpr uint32_t ROUND = TILE * U;        // 512 neighbours per round
constexpr uint32_t CHUNK_SLOTS = 256;       // chunk prefixes per warp (shared memory)
#ifndef CSAW_WALK_UNROLL
#define CSAW_WALK_UNROLL 1
#endif
constexpr int PASS1_UNROLL = CSAW_WALK_UNROLL;   // rounds of pass 1 in flight

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
    PhiloxKeys keys;                      // round keys of the seed
    uint32_t m0, m1, m2;
    uint32_t tele;                        // CSAW_TELEPORT_RESTART or _JUMP (teleporting kernels)
    uint32_t tele_q32;                    // teleport probability per step, in units of 2^-32
    unsigned long long* next_walker;
    const uint64_t* __restrict__ cdfw;   // cached edge-weight prefix sums (node2vec fast path) or null
    WalkSegments seg;                     // batched kernels: several requests in one launch
};

struct PrevCtx {
    uint32_t prev;       // previous vertex (node2vec), CSAW_NONE on the first step
    uint64_t pbeg, pend; // its neighbour range
};

// Row geometry: biases are read in 16-byte groups aligned to 4 elements, so
// the row [beg, end) is covered from abeg = beg rounded down to 4.
struct Row {
    uint64_t beg, end, abeg;
    uint32_t d, span;    // span = end - abeg
    uint32_t lo;         // beg - abeg (0..3): leading elements that are not in the row
};

// EdgeBias (Eq. 3) of the four neighbours at positions q .. q+3 relative to
// abeg (q a multiple of 4).  Positions outside [lo, span) get bias 0; only the
// first and the last group of a row can be partial.
template <int KIND>
__device__ __forceinline__ void group_bias(const WalkParams& p, const Row& r, uint32_t q,
                                           const PrevCtx& c, uint32_t (&b)[4])
{
    b[0] = b[1] = b[2] = b[3] = 0u;
    if (q >= r.span) return;
    const bool full = q >= r.lo && q + 4 <= r.span;
    if constexpr (KIND == CSAW_BIAS_EDGE_WEIGHT) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(p.w + r.abeg) + (q >> 2));
        b[0] = v.x; b[1] = v.y; b[2] = v.z; b[3] = v.w;
    } else if constexpr (KIND == CSAW_BIAS_NEIGHBOR_DEGREE) {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(p.col + r.abeg) + (q >> 2));
        if (full) {
            b[0] = __ldg(p.deg + u.x); b[1] = __ldg(p.deg + u.y);
            b[2] = __ldg(p.deg + u.z); b[3] = __ldg(p.deg + u.w);
        } else {
            const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (q + j >= r.lo && q + j < r.span) b[j] = __ldg(p.deg + uu[j]);
        }
        return;
    } else {
        static_assert(KIND != CSAW_BIAS_NODE2VEC, "node2vec biases are formed per tile (n2v_tile_bias)");
    }
    if (!full) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (q + j < r.lo || q + j >= r.span) b[j] = 0u;
    }
}

// node2vec biases (Sec. II-A) of one 128-neighbour tile at positions
// q0 .. q0+127 relative to abeg; lane holds positions q0 + 4*lane .. +3.
//
// Membership of a neighbour u in N(prev) is a merge of two sorted lists.  A
// window of N(prev) is kept staged in this warp's shared buffer: it starts at
// A = lower_bound(N(prev), smallest id of the tile) and holds up to SEG_SMEM
// entries.  Tiles come in ascending id order, so the next tile's A is usually
// found inside the staged window (most often at the cursor left by the last
// tile) with no global access; the window is reloaded from A (SEG_GROUP
// entries, then as many as their density says the tile needs) only when it
// does not cover the tile's ids.  When at most N2V_SCAN staged entries fall in
// the tile's id range, each lane compares its ids with them; otherwise each id
// is searched in the window (a lane's first id by bisection, its later ones by
// galloping on from the last hit), and ids beyond the window's last entry in
// the rest of N(prev) in global memory.  All lanes call this together, for
// tiles in ascending order; win = {pbeg, 0, 0} restarts.
constexpr uint32_t SEG_SMEM = 1024;
constexpr uint32_t SEG_GROUP = 256;   // entries staged in the first coalesced step
constexpr uint32_t N2V_SCAN = 32;     // N(prev) entries in a tile's id range compared directly

struct N2vWin {
    uint64_t A;    // first staged index of N(prev) in col[]
    uint32_t n;    // staged entries
    uint32_t cur;  // staged entries before cur are below every later tile's ids
};

__device__ __forceinline__ uint64_t lower_bound_col(const uint32_t* __restrict__ col, uint64_t lo,
                                                    uint64_t hi, uint32_t u)
{
    while (lo < hi) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(col + mid) < u) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t lower_bound_smem(const uint32_t* s, uint32_t n, uint32_t u)
{
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s[mid] < u) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void n2v_tile_bias(const WalkParams& p, const Row& r, uint32_t q0,
                                              const PrevCtx& c, int lane, uint32_t* s_seg,
                                              N2vWin& win, uint32_t (&b)[4])
{
    const uint32_t q = q0 + 4u * lane;
    b[0] = b[1] = b[2] = b[3] = 0u;
    uint32_t uu[4] = {0u, 0u, 0u, 0u};
    bool valid[4] = {false, false, false, false};
    if (q < r.span) {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(p.col + r.abeg) + (q >> 2));
        uint4 wv = make_uint4(1u, 1u, 1u, 1u);
        if (p.w) wv = __ldg(reinterpret_cast<const uint4*>(p.w + r.abeg) + (q >> 2));
        uu[0] = u.x; uu[1] = u.y; uu[2] = u.z; uu[3] = u.w;
        b[0] = wv.x; b[1] = wv.y; b[2] = wv.z; b[3] = wv.w;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            valid[j] = q + j >= r.lo && q + j < r.span;
            if (!valid[j]) b[j] = 0u;
        }
    }
    if (c.prev == CSAW_NONE) return;   // first step: the edge weight alone
    // smallest and largest id of the tile
    uint32_t mn = 0xFFFFFFFFu, mx = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (valid[j]) { mn = min(mn, uu[j]); mx = max(mx, uu[j]); }
    mn = __reduce_min_sync(CSAW_FULL_MASK, mn);
    mx = __reduce_max_sync(CSAW_FULL_MASK, mx);
    if (mn > mx) return;   // no neighbour of the row in this tile
    // A = lower_bound(N(prev), mn): inside the staged window when its last
    // entry is >= mn, else in the rest of N(prev) after the window.
    const uint64_t wend = win.A + win.n;
    uint64_t A;
    if (win.n > 0 && mn <= s_seg[win.n - 1]) {
        // cur < n here, and usually s_seg[cur] >= mn already
        const uint32_t k0 = win.cur;
        A = win.A + (s_seg[k0] >= mn ? k0 : k0 + 1 + lower_bound_smem(s_seg + k0 + 1, win.n - k0 - 1, mn));
    } else {
        uint64_t a0 = 0;
        if (lane == 0) a0 = lower_bound_col(p.col, wend, c.pend, mn);
        A = __shfl_sync(CSAW_FULL_MASK, a0, 0);
    }
    // Re-stage only when the window does not cover the tile's ids: A lies
    // past it, or the window ends below mx before the end of N(prev).
    const bool covered = A < wend && (wend == c.pend || mx <= s_seg[win.n - 1]);
    __syncwarp();
    if (!covered) {
        // Stage from A in groups of SEG_GROUP until the tile's last id is
        // covered, the buffer is full, or the staged density says the
        // buffer cannot reach that id.
        const uint64_t left = c.pend - A;
        const uint32_t cap = left < SEG_SMEM ? (uint32_t)left : SEG_SMEM;
        uint32_t n = 0, g = min(cap, SEG_GROUP);
        while (true) {
            for (uint32_t i = lane; i < g; i += 32) s_seg[n + i] = __ldg(p.col + A + n + i);
            n += g;
            __syncwarp();
            if (n == cap) break;
            const uint32_t hi = s_seg[n - 1];
            if (hi >= mx) break;
            const float need = __fdividef((float)(mx - hi) * (float)n, (float)max(hi - s_seg[0], 1u));
            if (need > (float)(cap - n)) break;
            // the estimate, with a margin, in one more step
            g = min(cap - n, ((uint32_t)(need * 1.25f) + 32u) & ~31u);
        }
        win.A = A;
        win.n = n;
        win.cur = 0;
    }
    const bool to_end = win.A + win.n == c.pend;
    const uint32_t last = win.n > 0 ? s_seg[win.n - 1] : 0u;
    const uint32_t off = (uint32_t)(A - win.A);   // entries below A are all < mn
    if ((to_end || mx <= last) &&
        !(off + N2V_SCAN < win.n && s_seg[off + N2V_SCAN] <= mx)) {
        // All of N(prev) within [mn, mx] is staged, at most N2V_SCAN entries
        // from off (a hub after a low-degree vertex, say): each lane compares
        // its ids with every entry (a merge step) instead of searching.
        uint32_t hit = 0u;   // bit j: uu[j] is in N(prev)
        uint32_t i = off;
        for (; i < win.n; ++i) {
            const uint32_t y = s_seg[i];
            if (y > mx) break;
            hit |= (uu[0] == y ? 1u : 0u) | (uu[1] == y ? 2u : 0u) | (uu[2] == y ? 4u : 0u) |
                   (uu[3] == y ? 8u : 0u);
        }
        win.cur = i;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (valid[j]) b[j] *= uu[j] == c.prev ? p.m0 : ((hit >> j) & 1u) ? p.m1 : p.m2;
        return;
    }
    win.cur = off;
    // One id per iteration, rotating uu/b/valid so that the body (and its
    // searches) is emitted once: the kernel's code has to fit the
    // instruction cache.  A lane's ids ascend, so after a binary search for
    // its first id each later search gallops on from where the last ended.
    uint32_t pos = ~0u;   // none yet
    uint32_t vm = (valid[0] ? 1u : 0u) | (valid[1] ? 2u : 0u) | (valid[2] ? 4u : 0u) | (valid[3] ? 8u : 0u);
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
        const uint32_t u = uu[0];
        if (vm & 1u) {
            uint32_t m;
            if (u == c.prev) {
                m = p.m0;
            } else {
                bool in;
                if (to_end || u <= last) {
                    uint32_t lo = off, hi = win.n;
                    if (pos != ~0u) {
                        lo = pos;
                        uint32_t bound = 1;
                        while (lo + bound - 1 < win.n && s_seg[lo + bound - 1] < u) { lo += bound; bound <<= 1; }
                        hi = min(lo + bound - 1, win.n);
                    }
                    const uint32_t at = lo + lower_bound_smem(s_seg + lo, hi - lo, u);
                    in = at < win.n && s_seg[at] == u;
                    pos = at;
                } else {
                    const uint64_t at = lower_bound_col(p.col, win.A + win.n, c.pend, u);
                    in = at < c.pend && __ldg(p.col + at) == u;
                }
                m = in ? p.m1 : p.m2;
            }
            b[0] *= m;
        }
        uu[0] = uu[1]; uu[1] = uu[2]; uu[2] = uu[3];
        const uint32_t t = b[0]; b[0] = b[1]; b[1] = b[2]; b[2] = b[3]; b[3] = t;
        vm >>= 1;
    }
}

// Sum type of a lane's sixteen biases in one round and of a round's total:
// 32 bits when max bias * ROUND < 2^32 (NARROW), else 64 bits.
template <bool WIDE>
struct Acc;
template <>
struct Acc<false> {
    using T = uint32_t;
    static __device__ __forceinline__ uint32_t warp_sum(uint32_t x) { return __reduce_add_sync(CSAW_FULL_MASK, x); }
    static __device__ __forceinline__ uint32_t scan(uint32_t x, int lane)
    {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(CSAW_FULL_MASK, x, o);
            if (lane >= o) x += y;
        }
        return x;
    }
};
template <>
struct Acc<true> {
    using T = uint64_t;
    static __device__ __forceinline__ uint64_t warp_sum(uint64_t x) { return warp_sum_u64(x); }
    static __device__ __forceinline__ uint64_t scan(uint64_t x, int lane) { return warp_inclusive_scan_u64(x, lane); }
};

// ---------------------------------------------------------------------------
// node2vec step from the intersection (when the weights' cumulative array is
// cached, or all weights are one).  With W the row's weight prefix sums, J the
// positions j of N(cur) whose id is in N(prev) (other than prev), and p the
// position of prev in N(cur):
//   S[i] = m2*W[i] + (m1-m2)*sum_{j in J, j<=i} w_j + (m0-m2)*w_p*[p <= i],
// the same prefix sums the streaming pass forms (computed in wrapping 64-bit
// arithmetic, exact because every true value fits).  J comes from binary
// searches of the shorter list's ids in the longer list, so a hub row after a
// low-degree previous vertex costs O(d_prev log d_cur) instead of O(d_cur);
// the pick is a 32-way warp search over S.
constexpr uint32_t JCAP = 256;

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* __restrict__ a, uint32_t n, uint32_t u)
{
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < u) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t ceil_log2(uint32_t x)
{
    return x <= 1 ? 0u : 32u - __clz(x - 1);
}

// Whether the intersection path is expected to beat streaming the row.
__device__ __forceinline__ bool n2v_fast_pays(uint32_t da, uint32_t db)
{
    const uint32_t mn = min(da, db), mx = max(da, db);
    if (mn > JCAP) return false;
    const uint32_t fast = ((mn + 31) / 32) * (ceil_log2(mx) + 2) + 2 * ceil_log2(da) + 24;
    const uint32_t stream = 3 * ((da + TILE - 1) / TILE) + 6;
    return fast < stream;
}

__device__ __forceinline__ bool n2v_fast_pick(const WalkParams& p, const Row& row, const PrevCtx& c,
                                              uint64_t r, int lane, uint32_t* s_jpos, uint64_t* s_jw,
                                              uint32_t* idx)
{
    const uint32_t da = row.d;
    const uint32_t db = (uint32_t)(c.pend - c.pbeg);
    const uint32_t* A = p.col + row.beg;
    const uint32_t* B = p.col + c.pbeg;
    const uint64_t* W = p.cdfw ? p.cdfw + row.beg : nullptr;
    auto Wat = [&](uint32_t i) -> uint64_t { return W ? __ldg(W + i) : (uint64_t)i + 1; };
    auto wof = [&](uint32_t i) -> uint64_t { return Wat(i) - (i ? Wat(i - 1) : 0); };
    const uint32_t lt = lanemask_lt();
    // J in ascending position order
    uint32_t nj = 0;
    if (db <= da) {
        for (uint32_t t0 = 0; t0 < db; t0 += 32) {
            const uint32_t j = t0 + lane;
            int pos = -1;
            if (j < db) {
                const uint32_t u = __ldg(B + j);
                if (u != c.prev) {
                    const uint32_t k = lower_bound_u32(A, da, u);
                    if (k < da && __ldg(A + k) == u) pos = (int)k;
                }
            }
            const uint32_t bal = __ballot_sync(CSAW_FULL_MASK, pos >= 0);
            if (pos >= 0) s_jpos[nj + __popc(bal & lt)] = (uint32_t)pos;
            nj += __popc(bal);
        }
    } else {
        for (uint32_t t0 = 0; t0 < da; t0 += 32) {
            const uint32_t j = t0 + lane;
            bool in = false;
            if (j < da) {
                const uint32_t u = __ldg(A + j);
                if (u != c.prev) {
                    const uint32_t k = lower_bound_u32(B, db, u);
                    in = k < db && __ldg(B + k) == u;
                }
            }
            const uint32_t bal = __ballot_sync(CSAW_FULL_MASK, in);
            if (in) s_jpos[nj + __popc(bal & lt)] = j;
            nj += __popc(bal);
        }
    }
    __syncwarp();
    // cumulative weights of the J entries
    uint64_t sum_j = 0;
    for (uint32_t t0 = 0; t0 < nj; t0 += 32) {
        const uint32_t j = t0 + lane;
        const uint64_t wj = j < nj ? wof(s_jpos[j]) : 0;
        const uint64_t incl = warp_inclusive_scan_u64(wj, lane) + sum_j;
        if (j < nj) s_jw[j] = incl;
        sum_j = __shfl_sync(CSAW_FULL_MASK, incl, 31);
    }
    // position and weight of prev in N(cur)
    uint32_t pp = 0;
    if (lane == 0) pp = lower_bound_u32(A, da, c.prev);
    pp = __shfl_sync(CSAW_FULL_MASK, pp, 0);
    const bool has_p = pp < da && __ldg(A + pp) == c.prev;
    const uint64_t wp = has_p ? wof(pp) : 0;
    __syncwarp();
    const uint64_t m2 = p.m2;
    const uint64_t dm1 = (uint64_t)p.m1 - m2;   // wrapping differences
    const uint64_t dm0 = (uint64_t)p.m0 - m2;
    auto S = [&](uint32_t i) -> uint64_t {
        // J entries at positions <= i
        uint32_t lo = 0, hi = nj;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_jpos[mid] <= i) lo = mid + 1; else hi = mid;
        }
        const uint64_t ij = lo ? s_jw[lo - 1] : 0;
        return m2 * Wat(i) + dm1 * ij + ((has_p && pp <= i) ? dm0 * wp : 0);
    };
    const uint64_t T = m2 * Wat(da - 1) + dm1 * sum_j + (has_p ? dm0 * wp : 0);
    if (T == 0) return false;
    const uint64_t x = scale_draw(r, T);
    // smallest i with S(i) > x; S(da-1) = T > x
    uint32_t lo = 0, hi = da - 1;
    while (hi - lo >= 32) {
        const uint32_t pk = lo + (uint32_t)(((uint64_t)(hi - lo) * (lane + 1)) / 32);
        const uint32_t hit = __ballot_sync(CSAW_FULL_MASK, S(pk) > x);
        const int k = __ffs(hit) - 1;   // lane 31's pivot is hi, so some lane hits
        const uint32_t pk_hit = __shfl_sync(CSAW_FULL_MASK, pk, k);
        const uint32_t pk_prev = __shfl_sync(CSAW_FULL_MASK, pk, k > 0 ? k - 1 : 0);
        lo = k > 0 ? pk_prev + 1 : lo;
        hi = pk_hit;
    }
    const uint32_t i = lo + lane;
    const uint32_t hit = __ballot_sync(CSAW_FULL_MASK, i <= hi && S(i) > x);
    *idx = lo + (__ffs(hit) - 1);
    return true;
}

// Biases of round `rd` (tiles rd*U .. rd*U+U-1) into b[u][j].  node2vec
// tiles are formed in a rolled loop (one emitted copy of the tile code) and
// pass through s_round (ROUND words of this warp's shared memory, each lane
// reading back only what it wrote) so that b is not live across it.
template <int KIND>
__device__ __forceinline__ void load_round(const WalkParams& p, const Row& r, uint32_t rd,
                                           const PrevCtx& c, int lane, uint32_t* s_seg, N2vWin& win,
                                           uint32_t* s_round, uint32_t (&b)[U][4])
{
    if constexpr (KIND == CSAW_BIAS_NODE2VEC) {
        uint4* s4 = reinterpret_cast<uint4*>(s_round);
#pragma unroll 1
        for (int u = 0; u < U; ++u) {
            uint32_t t[4] = {0u, 0u, 0u, 0u};
            if (rd * ROUND + u * TILE < r.span)   // warp-uniform: tiles past the row are empty
                n2v_tile_bias(p, r, rd * ROUND + u * TILE, c, lane, s_seg, win, t);
            s4[u * 32 + lane] = make_uint4(t[0], t[1], t[2], t[3]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint4 v = s4[u * 32 + lane];
            b[u][0] = v.x; b[u][1] = v.y; b[u][2] = v.z; b[u][3] = v.w;
        }
    } else {
#pragma unroll
        for (int u = 0; u < U; ++u) group_bias<KIND>(p, r, rd * ROUND + u * TILE + 4u * lane, c, b[u]);
    }
}

// Within round `rd` whose biases are b and which starts at prefix `before`,
// find the neighbour whose interval holds x (x is known to lie in this
// round).  Returns its index relative to beg.
template <bool WIDE>
__device__ __forceinline__ uint32_t locate_in_round(const Row& r, uint32_t rd, const uint32_t (&b)[U][4],
                                                    uint64_t before, uint64_t x, int lane)
{
    using A = Acc<WIDE>;
    using T = typename A::T;
    // tile holding x: the first whose inclusive prefix exceeds x (selected
    // without dynamic indexing so the biases stay in registers)
    T st[U];
    int ut = -1;
    uint64_t bt = 0, acc = before;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        st[u] = (T)b[u][0] + b[u][1] + b[u][2] + b[u][3];
        const uint64_t tt = A::warp_sum(st[u]);
        if (ut < 0 && acc + tt > x) { ut = u; bt = acc; }
        acc += tt;
    }
    T sl = 0;
    uint32_t b0 = 0, b1 = 0, b2 = 0;
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (u == ut) { sl = st[u]; b0 = b[u][0]; b1 = b[u][1]; b2 = b[u][2]; }
    const T incl = A::scan(sl, lane);
    const uint32_t hit = __ballot_sync(CSAW_FULL_MASK, bt + incl > x);
    const int L = __ffs(hit) - 1;
    // inside the hit lane's four neighbours: the first whose inclusive prefix exceeds x
    const uint64_t e0 = bt + incl - sl + b0;
    const uint64_t e1 = e0 + b1;
    const uint64_t e2 = e1 + b2;
    uint32_t j = e0 > x ? 0u : (e1 > x ? 1u : (e2 > x ? 2u : 3u));
    j = __shfl_sync(CSAW_FULL_MASK, j, L);
    return rd * ROUND + (uint32_t)ut * TILE + 4u * L + j - r.lo;
}

// Sum of the biases of an interior round rd (all of its groups inside the
// row: rd >= 1 and (rd + 1) * ROUND <= span): no bounds checks or masks.
template <int KIND, bool WIDE>
__device__ __forceinline__ typename Acc<WIDE>::T sum_interior_round(const WalkParams& p, const Row& r,
                                                                    uint32_t rd, int lane)
{
    using T = typename Acc<WIDE>::T;
    T s = 0;
    if constexpr (KIND == CSAW_BIAS_EDGE_WEIGHT) {
        const uint4* base = reinterpret_cast<const uint4*>(p.w + r.abeg) + (rd * ROUND) / 4 + lane;
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = __ldg(base + u * (TILE / 4));
#pragma unroll
        for (int u = 0; u < U; ++u) s += (T)v[u].x + v[u].y + v[u].z + v[u].w;
    } else {
        const uint4* base = reinterpret_cast<const uint4*>(p.col + r.abeg) + (rd * ROUND) / 4 + lane;
        uint4 c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) c[u] = __ldg(base + u * (TILE / 4));
#pragma unroll
        for (int u = 0; u < U; ++u)
            s += (T)__ldg(p.deg + c[u].x) + __ldg(p.deg + c[u].y) + __ldg(p.deg + c[u].z) + __ldg(p.deg + c[u].w);
    }
    return s;
}

// Biases of an interior round (no bounds checks or masks), for the locate step.
template <int KIND>
__device__ __forceinline__ void load_interior_round(const WalkParams& p, const Row& r, uint32_t rd,
                                                    int lane, uint32_t (&b)[U][4])
{
    if constexpr (KIND == CSAW_BIAS_EDGE_WEIGHT) {
        const uint4* base = reinterpret_cast<const uint4*>(p.w + r.abeg) + (rd * ROUND) / 4 + lane;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint4 v = __ldg(base + u * (TILE / 4));
            b[u][0] = v.x; b[u][1] = v.y; b[u][2] = v.z; b[u][3] = v.w;
        }
    } else {
        const uint4* base = reinterpret_cast<const uint4*>(p.col + r.abeg) + (rd * ROUND) / 4 + lane;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint4 c = __ldg(base + u * (TILE / 4));
            b[u][0] = __ldg(p.deg + c.x); b[u][1] = __ldg(p.deg + c.y);
            b[u][2] = __ldg(p.deg + c.z); b[u][3] = __ldg(p.deg + c.w);
        }
    }
}

// One walk step: the inverse transform pick for draw r over row `row`.
// Returns false at a dead end (T == 0).
template <int KIND, bool WIDE>
__device__ __forceinline__ bool walk_pick(const WalkParams& p, const Row& row, const PrevCtx& c,
                                          uint64_t r, uint64_t* s_chunk, uint32_t* s_seg, uint32_t* s_jpos,
                                          uint64_t* s_jw, int lane, uint32_t* idx)
{
    using A = Acc<WIDE>;
    using T = typename A::T;
    if (row.d == 0) return false;
    if constexpr (KIND == CSAW_BIAS_NODE2VEC) {
        __syncwarp();   // the last step's reads of the overlaid buffers are done
        if (c.prev != CSAW_NONE && (p.cdfw != nullptr || p.w == nullptr) &&
            n2v_fast_pays(row.d, (uint32_t)(c.pend - c.pbeg)))
            return n2v_fast_pick(p, row, c, r, lane, s_jpos, s_jw, idx);
    }
    if constexpr (KIND == CSAW_BIAS_UNIFORM) {
        *idx = (uint32_t)scale_draw(r, row.d);   // b = 1: S[i] = i + 1, the pick is x itself
        return true;
    }
    if constexpr (KIND != CSAW_BIAS_NODE2VEC) {
        if (row.span <= TILE) {
            // One tile: lane l holds positions 4l .. 4l+3; its inclusive
            // prefix over lanes gives S at 4l+3, the total is lane 31's.
            uint32_t b[4];
            group_bias<KIND>(p, row, 4u * lane, c, b);
            const T sl = (T)b[0] + b[1] + b[2] + b[3];
            const T incl = A::scan(sl, lane);
            const uint64_t total = (uint64_t)__shfl_sync(CSAW_FULL_MASK, incl, 31);
            if (total == 0) return false;
            const uint64_t x = scale_draw(r, total);
            const uint32_t hit = __ballot_sync(CSAW_FULL_MASK, (uint64_t)incl > x);
            const int L = __ffs(hit) - 1;
            const uint64_t e0 = (uint64_t)(incl - sl) + b[0];
            const uint64_t e1 = e0 + b[1];
            const uint64_t e2 = e1 + b[2];
            uint32_t j = e0 > x ? 0u : (e1 > x ? 1u : (e2 > x ? 2u : 3u));
            j = __shfl_sync(CSAW_FULL_MASK, j, L);
            *idx = 4u * (uint32_t)L + j - row.lo;
            return true;
        }
    }
    N2vWin win = {c.pbeg, 0, 0};
    // node2vec round biases pass through the chunk table's space: it is free
    // in a one-round step, and in pass 2 once the chunk has been found
    static_assert(ROUND <= 2 * CHUNK_SLOTS, "a round must fit the chunk table");
    uint32_t* s_round = reinterpret_cast<uint32_t*>(s_chunk);
    const uint32_t nrounds = (row.span + ROUND - 1) / ROUND;
    if (nrounds == 1) {
        uint32_t b[U][4];
        load_round<KIND>(p, row, 0, c, lane, s_seg, win, s_round, b);
        T s = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) s += (T)b[u][0] + b[u][1] + b[u][2] + b[u][3];
        const uint64_t total = A::warp_sum(s);
        if (total == 0) return false;
        *idx = locate_in_round<WIDE>(row, 0, b, 0, scale_draw(r, total), lane);
        return true;
    }
    // Pass 1: total, with the running prefix stored after every chunk of G rounds.
    const uint32_t G = (nrounds + CHUNK_SLOTS - 1) / CHUNK_SLOTS;
    const uint32_t nchunks = (nrounds + G - 1) / G;
    uint64_t running = 0;
    for (uint32_t ch = 0; ch < nchunks; ++ch) {
        const uint32_t r_end = min(nrounds, (ch + 1) * G);
#pragma unroll PASS1_UNROLL
        for (uint32_t rd = ch * G; rd < r_end; ++rd) {
            T s = 0;
            if constexpr (KIND == CSAW_BIAS_NODE2VEC) {
                // only the round's sum is needed: tiles in a rolled loop
#pragma unroll 1
                for (int u = 0; u < U; ++u) {
                    uint32_t t[4];
                    n2v_tile_bias(p, row, rd * ROUND + u * TILE, c, lane, s_seg, win, t);
                    s += (T)t[0] + t[1] + t[2] + t[3];
                }
            } else if (rd >= 1 && (rd + 1) * ROUND <= row.span) {
                s = sum_interior_round<KIND, WIDE>(p, row, rd, lane);
            } else {
                uint32_t b[U][4];
                load_round<KIND>(p, row, rd, c, lane, s_seg, win, s_round, b);
#pragma unroll
                for (int u = 0; u < U; ++u) s += (T)b[u][0] + b[u][1] + b[u][2] + b[u][3];
            }
            running += A::warp_sum(s);
        }
        if (lane == 0) s_chunk[ch] = running;
    }
    __syncwarp();
    const uint64_t total = running;
    if (total == 0) return false;
    const uint64_t x = scale_draw(r, total);
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
    win = {c.pbeg, 0, 0};   // pass 2 restarts the node2vec window at the chunk's first tile
    // Pass 2: rescan that chunk's rounds.
    const uint32_t r_end = min(nrounds, (ch + 1) * G);
    for (uint32_t rd = ch * G; rd < r_end; ++rd) {
        uint32_t b[U][4];
        if (KIND != CSAW_BIAS_NODE2VEC && rd >= 1 && (rd + 1) * ROUND <= row.span)
            load_interior_round<KIND == CSAW_BIAS_NODE2VEC ? CSAW_BIAS_EDGE_WEIGHT : KIND>(p, row, rd, lane, b);
        else
            load_round<KIND>(p, row, rd, c, lane, s_seg, win, s_round, b);
        T s = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) s += (T)b[u][0] + b[u][1] + b[u][2] + b[u][3];
        const uint64_t rt = A::warp_sum(s);
        if (before + rt > x) {
            *idx = locate_in_round<WIDE>(row, rd, b, before, x, lane);
            return true;
        }
        before += rt;
    }
    *idx = row.d - 1;   // not reached: x < total lies in some round
    return true;
}

// Resident blocks per SM the register budget is set for (the kernel is
// latency-bound, so residency beats a few spilled registers): edge weight 6
// (40 registers), neighbour degree 4 (64), node2vec's windows 3 (80).
#ifndef CSAW_WALK_EW_BLOCKS
#define CSAW_WALK_EW_BLOCKS 6   // edge-weight, 32-bit sums (swept: 5 -> 42.9 ms, 6 -> 39.9 ms, 7 -> 43.8 ms at s20)
#endif

#ifndef CSAW_WALK_N2V_BLOCKS
#define CSAW_WALK_N2V_BLOCKS 4   // node2vec, plain walks (64 registers; 3 blocks: 80 registers)
#endif

template <int KIND, bool WIDE, bool TELE, bool BATCH>
constexpr int walk_min_blocks()
{
    return KIND == CSAW_BIAS_UNIFORM ? 5
           : (KIND == CSAW_BIAS_EDGE_WEIGHT && !WIDE) ? CSAW_WALK_EW_BLOCKS
           : KIND == CSAW_BIAS_NODE2VEC ? (TELE || BATCH ? 3 : CSAW_WALK_N2V_BLOCKS) : 4;
}

// TELE: random walk with restart or with jump (Sec. II-A; an Update, Eq. 4,
// that returns a vertex other than the sampled neighbour).  Each step first
// draws attempt 1; if its upper 32 bits are below tele_q32 the walker goes to
// its start (restart) or to vertex floor(r2 * V / 2^64), r2 the draw of
// attempt 2 (jump), instead of to a neighbour; a dead end teleports the same
// way instead of stopping, and node2vec's next step has no previous vertex.
// BATCH: walkers of several requests (WalkSegments), each with its own
// seed, walker index and length; the draws are those of its request alone.
template <int KIND, bool WIDE, bool TELE, bool BATCH = false>
__global__ void __launch_bounds__(WALK_THREADS, (walk_min_blocks<KIND, WIDE, TELE, BATCH>())) walk_kernel(WalkParams p)
{
    static_assert(!(TELE && BATCH), "teleporting walks are not batched");
    // Per warp: the chunk prefix table, then (node2vec) the N(prev) window.
    // The intersection path's buffers overlay them: a step uses one or the other.
    constexpr uint32_t WARP_WORDS = CHUNK_SLOTS + (KIND == CSAW_BIAS_NODE2VEC ? SEG_SMEM / 2 : 0);
    static_assert(KIND != CSAW_BIAS_NODE2VEC || JCAP * 12 <= WARP_WORDS * 8, "intersection buffers overflow");
    __shared__ __align__(16) uint64_t s_warp_all[WALK_WARPS][WARP_WORDS];
    const int lane = threadIdx.x & 31;
    uint64_t* s_chunk = s_warp_all[threadIdx.x >> 5];
    uint32_t* s_seg = reinterpret_cast<uint32_t*>(s_chunk + (KIND == CSAW_BIAS_NODE2VEC ? CHUNK_SLOTS : 0));
    uint64_t* s_jw = s_chunk;
    uint32_t* s_jpos = reinterpret_cast<uint32_t*>(s_chunk + JCAP);
    for (uint32_t taken = 0;; ++taken) {
        if constexpr (BATCH) {
            if (p.seg.warp_budget && taken >= p.seg.warp_budget) break;
        }
        unsigned long long wk = 0;
        if (lane == 0) wk = atomicAdd(p.next_walker, 1ull);
        wk = __shfl_sync(CSAW_FULL_MASK, wk, 0);
        if (wk >= p.n) break;
        uint32_t L = p.L;
        uint32_t* out;
        WalkerSlot ws;
        if constexpr (BATCH) {
            ws = walker_slot(p.seg, wk);
            L = ws.L;
            out = p.path + ws.row0;
        } else {
            out = p.path + wk * ((uint64_t)p.L + 1);
        }
        const uint64_t row_len = (uint64_t)L + 1;
        uint32_t cur = __ldg(p.starts + wk);
        if (cur >= p.V) {
            for (uint64_t t = lane; t < row_len; t += 32) out[t] = CSAW_NONE;
            continue;
        }
        PrevCtx c;
        c.prev = CSAW_NONE;
        c.pbeg = c.pend = 0;
        uint32_t buf = lane == 0 ? cur : CSAW_NONE;   // entries of the current 32-block
        uint64_t flushed = 0;                         // entries [0, flushed) are in memory
        for (uint32_t s = 0; s < L; ++s) {
            uint32_t nxt = 0;
            bool jump = false;   // warp-uniform: every lane draws the same
            if constexpr (TELE)
                jump = (uint32_t)(philox_draw(p.keys, 1u, cur, s, (uint32_t)wk) >> 32) < p.tele_q32;
            if (!jump) {
                Row row;
                row.beg = __ldg(p.off + cur);
                row.end = __ldg(p.off + cur + 1);
                row.abeg = row.beg & ~3ull;
                row.d = (uint32_t)(row.end - row.beg);
                row.span = (uint32_t)(row.end - row.abeg);
                row.lo = (uint32_t)(row.beg - row.abeg);
                uint64_t r;
                if constexpr (BATCH) r = philox_draw(ws.k0, ws.k1, 0u, cur, s, ws.id);
                else r = philox_draw(p.keys, 0u, cur, s, (uint32_t)wk);
                uint32_t idx;
                if (walk_pick<KIND, WIDE>(p, row, c, r, s_chunk, s_seg, s_jpos, s_jw, lane, &idx)) {
                    nxt = __ldg(p.col + row.beg + idx);
                    if constexpr (KIND == CSAW_BIAS_NODE2VEC) {
                        c.prev = cur;
                        c.pbeg = row.beg;
                        c.pend = row.end;
                    }
                } else {
                    if constexpr (!TELE) break;
                    jump = true;   // a dead end teleports
                }
            }
            if constexpr (TELE) {
                if (jump) {
                    nxt = p.tele == CSAW_TELEPORT_RESTART
                              ? __ldg(p.starts + wk)
                              : (uint32_t)scale_draw(philox_draw(p.keys, 2u, cur, s, (uint32_t)wk), p.V);
                    if constexpr (KIND == CSAW_BIAS_NODE2VEC) {
                        c.prev = CSAW_NONE;
                        c.pbeg = c.pend = 0;
                    }
                }
            }
            cur = nxt;
            const uint64_t t = (uint64_t)s + 1;
            if ((uint32_t)(t & 31) == (uint32_t)lane) buf = cur;
            if ((t & 31) == 31) {
                out[t - 31 + lane] = buf;
                buf = CSAW_NONE;
                flushed = t + 1;
            }
        }
        // Remaining entries: the buffered block, then CSAW_NONE to the end of the row.
        for (uint64_t t = flushed + lane; t < row_len; t += 32)
            out[t] = (t < flushed + 32) ? buf : CSAW_NONE;
    }
}

template <int KIND, bool WIDE, bool TELE, bool BATCH = false>
static csaw_status launch_walk_kwt(const WalkParams& p, int sm_count, cudaStream_t s)
{
    // resident blocks per SM, looked up once (calls may come from several threads)
    static std::atomic<int> cached{0};
    int per_sm = cached.load(std::memory_order_acquire);
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_kernel<KIND, WIDE, TELE, BATCH>,
                                                                      WALK_THREADS, 0);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy(walk)");
        if (per_sm < 1) per_sm = 1;
        cached.store(per_sm, std::memory_order_release);
    }
    uint64_t blocks = (uint64_t)sm_count * per_sm;
    if (BATCH && p.seg.warp_budget) {
        // enough warps that each takes at most warp_budget walkers
        const uint64_t per_block = (uint64_t)WALK_WARPS * p.seg.warp_budget;
        blocks = (p.n + per_block - 1) / per_block;
        if (blocks < 1) blocks = 1;
    }
    walk_kernel<KIND, WIDE, TELE, BATCH><<<(unsigned)blocks, WALK_THREADS, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "walk_kernel launch");
    return CSAW_OK;
}

template <int KIND, bool WIDE>
static csaw_status launch_walk_kw(const WalkParams& p, int sm_count, cudaStream_t s)
{
    return p.tele ? launch_walk_kwt<KIND, WIDE, true>(p, sm_count, s)
                  : launch_walk_kwt<KIND, WIDE, false>(p, sm_count, s);
}

// max_bias: an upper bound of any bias of this call; 32-bit round sums when
// a round of ROUND neighbours cannot reach 2^32.
static csaw_status launch_walk(int kind, uint64_t max_bias, const WalkParams& p, int sm_count,
                               cudaStream_t s)
{
    const bool wide = max_bias * ROUND >= (1ull << 32);
    switch (kind) {
    case CSAW_BIAS_UNIFORM: return launch_walk_kw<CSAW_BIAS_UNIFORM, false>(p, sm_count, s);
    case CSAW_BIAS_EDGE_WEIGHT:
        return wide ? launch_walk_kw<CSAW_BIAS_EDGE_WEIGHT, true>(p, sm_count, s)
                    : launch_walk_kw<CSAW_BIAS_EDGE_WEIGHT, false>(p, sm_count, s);
    case CSAW_BIAS_NEIGHBOR_DEGREE:
        return wide ? launch_walk_kw<CSAW_BIAS_NEIGHBOR_DEGREE, true>(p, sm_count, s)
                    : launch_walk_kw<CSAW_BIAS_NEIGHBOR_DEGREE, false>(p, sm_count, s);
    case CSAW_BIAS_NODE2VEC:
        return wide ? launch_walk_kw<CSAW_BIAS_NODE2VEC, true>(p, sm_count, s)
                    : launch_walk_kw<CSAW_BIAS_NODE2VEC, false>(p, sm_count, s);
    default:
        return fail(CSAW_ERR_INVALID, "unknown bias kind %d", kind);
    }
}

// launch_walk for a batch of requests (p.seg set, no teleports).
static csaw_status launch_walk_batch(int kind, uint64_t max_bias, const WalkParams& p, int sm_count,
                                     cudaStream_t s)
{
    const bool wide = max_bias * ROUND >= (1ull << 32);
    switch (kind) {
    case CSAW_BIAS_UNIFORM: return launch_walk_kwt<CSAW_BIAS_UNIFORM, false, false, true>(p, sm_count, s);
    case CSAW_BIAS_EDGE_WEIGHT:
        return wide ? launch_walk_kwt<CSAW_BIAS_EDGE_WEIGHT, true, false, true>(p, sm_count, s)
                    : launch_walk_kwt<CSAW_BIAS_EDGE_WEIGHT, false, false, true>(p, sm_count, s);
    case CSAW_BIAS_NEIGHBOR_DEGREE:
        return wide ? launch_walk_kwt<CSAW_BIAS_NEIGHBOR_DEGREE, true, false, true>(p, sm_count, s)
                    : launch_walk_kwt<CSAW_BIAS_NEIGHBOR_DEGREE, false, false, true>(p, sm_count, s);
    case CSAW_BIAS_NODE2VEC:
        return wide ? launch_walk_kwt<CSAW_BIAS_NODE2VEC, true, false, true>(p, sm_count, s)
                    : launch_walk_kwt<CSAW_BIAS_NODE2VEC, false, false, true>(p, sm_count, s);
    default:
        return fail(CSAW_ERR_INVALID, "unknown bias kind %d", kind);
    }
}


csaw_status walk_batch(const csaw_graph* g, const csaw_bias* bias, const uint32_t* d_starts, uint64_t n,
                       const WalkSegments& seg, uint32_t max_len, uint32_t* d_path, cudaStream_t s)
{
    int kind;
    CSAW_TRY(check_bias(g, bias, true, &kind));
    if (n == 0) return CSAW_OK;
    if (kind != CSAW_BIAS_NODE2VEC && cached_cdf_usable(g, kind))
        return walk_batch_cached(g, kind, d_starts, n, seg, max_len, d_path, s);
    void* counter = nullptr;
    CSAW_TRY(dalloc(&counter, sizeof(unsigned long long), s));
    csaw_status st = CSAW_OK;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) st = cuda_fail(e, "memset counter");
    if (st == CSAW_OK) {
        WalkParams p;
        p.off = g->off; p.col = g->col; p.w = g->w; p.deg = g->deg; p.V = g->V;
        p.starts = d_starts; p.n = n; p.L = max_len; p.path = d_path;
        p.keys = philox_round_keys(0);
        p.m0 = bias->n2v_mult[0]; p.m1 = bias->n2v_mult[1]; p.m2 = bias->n2v_mult[2];
        p.tele = CSAW_TELEPORT_NONE;
        p.tele_q32 = 0;
        p.next_walker = (unsigned long long*)counter;
        p.cdfw = g->cdf[CSAW_BIAS_EDGE_WEIGHT];
        p.seg = seg;
        uint64_t max_bias = 1;
        if (kind == CSAW_BIAS_EDGE_WEIGHT) max_bias = g->max_weight;
        else if (kind == CSAW_BIAS_NEIGHBOR_DEGREE) max_bias = g->max_degree;
        else if (kind == CSAW_BIAS_NODE2VEC) {
            uint64_t m = 1;
            for (int i = 0; i < 3; ++i) m = bias->n2v_mult[i] > m ? bias->n2v_mult[i] : m;
            max_bias = (uint64_t)g->max_weight * m;
        }
        st = launch_walk_batch(kind, max_bias, p, g->sm_count, s);
    }
    dfree(counter, s);
    return st;
}

// CUDA events around a call's phases, when the caller asks for their times:
// [0] before the array's construction, [1] before the walk, [2] after it.
struct PhaseTimer {
    float* out = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    bool ok = true;
    PhaseTimer(float* o, cudaStream_t s) : out(o)
    {
        for (int i = 0; out && ok && i < 3; ++i) ok = cudaEventCreate(&ev[i]) == cudaSuccess;
        mark(0, s);
    }
    void mark(int i, cudaStream_t s)
    {
        if (out && ok) ok = cudaEventRecord(ev[i], s) == cudaSuccess;
    }
    // Waits for the last mark and stores the two phase times.
    csaw_status finish()
    {
        if (!out) return CSAW_OK;
        cudaError_t e = ok ? cudaEventSynchronize(ev[2]) : cudaErrorUnknown;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&out[0], ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&out[1], ev[1], ev[2]);
        return e == cudaSuccess ? CSAW_OK : cuda_fail(e, "phase times");
    }
    ~PhaseTimer()
    {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

}  // namespace csaw

using namespace csaw;

extern "C" csaw_status csaw_walk_ex(csaw_graph* g, const uint32_t* starts, uint64_t n_walkers,
                                    uint32_t length, const csaw_bias* bias, uint64_t rng_seed,
                                    uint32_t* path, int mem_kind, void* stream, const csaw_walk_opts* opts)
{
    clear_error();
    if (!g) return fail(CSAW_ERR_INVALID, "graph is NULL");
    AllocScope alloc_scope(g);
    int kind;
    CSAW_TRY(check_bias(g, bias, true, &kind));
    const uint32_t tele = opts ? (uint32_t)opts->teleport : CSAW_TELEPORT_NONE;
    if (tele != CSAW_TELEPORT_NONE && tele != CSAW_TELEPORT_RESTART && tele != CSAW_TELEPORT_JUMP)
        return fail(CSAW_ERR_INVALID, "unknown teleport mode %d", opts->teleport);
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
    // static bias with a positive cumulative array: the graph's cached one,
    // or (build_cdf) one built for this call into a stream-ordered temporary
    const bool cached = cached_cdf_usable(g, kind);
    const bool build = !cached && opts && opts->build_cdf && cdf_kind_positive(g, kind);
    const bool over_array = tele == CSAW_TELEPORT_NONE && kind != CSAW_BIAS_NODE2VEC && (cached || build);
    if (mem_kind == CSAW_MEM_HOST) {
        // (over the array, the host starts are checked while the walk runs:
        // the kernels stop a walker whose start is not a vertex)
        for (uint64_t i = 0; !over_array && i < n_walkers; ++i)
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
    PhaseTimer timer(opts ? opts->phase_ms : nullptr, s);
    if (over_array) {
        const uint64_t* cdf = kind == CSAW_BIAS_UNIFORM ? nullptr : g->cdf[kind];
        void* tmp = nullptr;
        csaw_status st = CSAW_OK;
        // built for the call: edge weights keep only the summaries and
        // records (the leaf level is formed from the weights); neighbour
        // degree keeps the whole array (its biases are gathers)
        const bool leaf = !(build && kind == CSAW_BIAS_EDGE_WEIGHT);
        if (build) {
            const uint64_t words = leaf ? cdf_words(g->E, g->V) : wsum_layout(g->E, g->V).words;
            st = dalloc(&tmp, sizeof(uint64_t) * words, s);
            if (st == CSAW_OK && leaf) st = enqueue_cdf_build(g, kind, (uint64_t*)tmp, s);
            if (st == CSAW_OK && !leaf) {
                const CdfView c = wsum_view((const uint64_t*)tmp, g->E, g->V);
                st = enqueue_cdf_build_raw(g->off, g->col, g->w, g->deg, g->V, g->E, g->sm_count, kind, nullptr,
                                           (uint64_t*)c.s1, (uint64_t*)c.s2, (uint64_t*)c.rec, s);
            }
            cdf = (const uint64_t*)tmp;
        }
        timer.mark(1, s);
        // thread per walker; host paths come back chunk by chunk while the
        // next chunk walks
        if (st == CSAW_OK) {
            if (mem_kind == CSAW_MEM_HOST) {
                st = walk_cached_to_host(g, kind, cdf, leaf, starts, d_starts, n_walkers, length, rng_seed, d_path,
                                         path, s, timer.out && timer.ok ? timer.ev[2] : nullptr);
            } else {
                st = launch_walk_cached(g, kind, cdf, leaf, d_starts, 0, n_walkers, length, rng_seed, d_path, s);
                timer.mark(2, s);
            }
        }
        if (st == CSAW_OK) st = timer.finish();
        dfree(tmp, s);
        if (mem_kind == CSAW_MEM_HOST) {
            if (st != CSAW_OK) cudaStreamSynchronize(s);
            dfree((void*)d_starts, s);
            dfree(d_path, s);
        }
        return st;
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
        p.keys = philox_round_keys(rng_seed);
        p.m0 = bias->n2v_mult[0]; p.m1 = bias->n2v_mult[1]; p.m2 = bias->n2v_mult[2];
        p.tele = tele;
        p.tele_q32 = tele != CSAW_TELEPORT_NONE ? opts->teleport_q32 : 0u;
        p.next_walker = (unsigned long long*)counter;
        p.cdfw = g->cdf[CSAW_BIAS_EDGE_WEIGHT];
        p.seg = WalkSegments{};
        uint64_t max_bias = 1;
        if (kind == CSAW_BIAS_EDGE_WEIGHT) max_bias = g->max_weight;
        else if (kind == CSAW_BIAS_NEIGHBOR_DEGREE) max_bias = g->max_degree;
        else if (kind == CSAW_BIAS_NODE2VEC) {
            uint64_t m = 1;
            for (int i = 0; i < 3; ++i) m = bias->n2v_mult[i] > m ? bias->n2v_mult[i] : m;
            max_bias = (uint64_t)g->max_weight * m;
        }
        timer.mark(1, s);
        st = launch_walk(kind, max_bias, p, g->sm_count, s);
        timer.mark(2, s);
    }
    dfree(counter, s);
    if (st == CSAW_OK) st = timer.finish();
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

extern "C" csaw_status csaw_walk(csaw_graph* g, const uint32_t* starts, uint64_t n_walkers,
                                 uint32_t length, const csaw_bias* bias, uint64_t rng_seed,
                                 uint32_t* path, int mem_kind, void* stream)
{
    return csaw_walk_ex(g, starts, n_walkers, length, bias, rng_seed, path, mem_kind, stream, nullptr);
}
