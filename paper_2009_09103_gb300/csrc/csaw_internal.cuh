// csaw_internal.cuh -- shared pieces of libcsaw's CUDA translation units.
//
// Device-side random numbers, integer draw mapping, warp collectives, the
// graph object and error plumbing.  Everything here is written for sm_103a.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "csaw.h"

#define CSAW_FULL_MASK 0xFFFFFFFFu
#define CSAW_EDGE_PAD 16   // zeroed uint32 entries after col[] and w[]

// The caller's device allocator (csaw_graph_set_allocator), or none.
struct DevAllocator {
    csaw_alloc_fn alloc = nullptr;
    csaw_free_fn free = nullptr;
    void* ctx = nullptr;
};

// ---------------------------------------------------------------------------
// Graph: CSR resident in HBM (uint64 offsets, uint32 columns and weights) and
// the derived uint32 degree array used by the neighbour-degree bias.
struct csaw_graph {
    uint32_t V = 0;
    uint64_t E = 0;
    uint64_t* off = nullptr;   // [V+1]
    uint32_t* col = nullptr;   // [E], rows strictly ascending
    uint32_t* w = nullptr;     // [E] or nullptr (all ones)
    uint32_t* deg = nullptr;   // [V]
    uint32_t max_degree = 0;
    uint32_t max_weight = 1;
    uint32_t min_weight = 1;            // 0 if some edge weight is zero
    bool zero_degree_target = false;    // some edge points at a vertex without neighbours
    uint64_t device_bytes = 0;
    int device = 0;
    int sm_count = 0;
    // cached per-edge inclusive prefix sums of a static bias kind (or null):
    // cdf[kind][e] = b(row start) + ... + b(e) within e's row
    uint64_t* cdf[4] = {nullptr, nullptr, nullptr, nullptr};
    // selection launch shape per bias kind (0 = default): warp-item degree
    // threshold and resident blocks per SM
    uint32_t tune_theta_w[4] = {0, 0, 0, 0};
    uint32_t tune_blocks_per_sm[4] = {0, 0, 0, 0};
    DevAllocator allocator;             // device memory of calls on this graph
    DevAllocator cdf_alloc[4];          // the allocator each cached array came from
};

// ---------------------------------------------------------------------------
// Errors: every entry point returns a csaw_status and leaves a message in a
// thread-local buffer.
namespace csaw {

csaw_status fail(csaw_status st, const char* fmt, ...);
csaw_status cuda_fail(cudaError_t err, const char* what);
void clear_error();

#define CSAW_CUDA(call)                                                   \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) return ::csaw::cuda_fail(_e, #call);       \
    } while (0)

#define CSAW_TRY(expr)                                                    \
    do {                                                                  \
        csaw_status _s = (expr);                                          \
        if (_s != CSAW_OK) return _s;                                     \
    } while (0)

// Stream-ordered device allocation: the caller's allocator of the graph
// whose call is running on this thread (AllocScope), else CUDA's pool.
csaw_status dalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);

// The allocator dalloc/dfree use on this thread while an entry point on a
// graph runs; nested scopes restore the outer one.
const DevAllocator* current_allocator();
struct AllocScope {
    const DevAllocator* prev;
    explicit AllocScope(const csaw_graph* g);
    ~AllocScope();
};

// Allocation and release through an explicit allocator (null or empty:
// cudaMalloc / cudaFree), for memory that outlives the call that made it.
csaw_status alloc_with(const DevAllocator* a, void** p, size_t bytes, cudaStream_t s);
void free_with(const DevAllocator& a, void* p, cudaStream_t s);

// Device-wide exclusive scan of n uint32 (n read from *n_dev, n <= n_max):
// out[i] = in[0] + ... + in[i-1] for i <= n; *total_out (device, optional)
// receives out[n].  scratch: scan_scratch_bytes(n_max).
size_t scan_scratch_bytes(uint64_t n_max);
csaw_status scan_u32(const uint32_t* in, uint64_t* out, const uint64_t* n_dev, uint64_t n_max,
                     void* scratch, uint64_t* total_out, cudaStream_t s);

// Stable LSD radix sort of n uint64 keys on their low `bits` bits (n read
// from *n_dev, n <= n_max < 2^32).  keys and alt hold n_max keys; *result is
// the one holding the sorted keys.  scratch: sort_scratch_bytes(n_max).
size_t sort_scratch_bytes(uint64_t n_max);
csaw_status radix_sort_u64(uint64_t* keys, uint64_t* alt, const uint64_t* n_dev, uint64_t n_max,
                           int bits, int sm_count, void* scratch, cudaStream_t s, uint64_t** result);

// Several walk requests in one launch (the request server's batches):
// walker w belongs to request r with start[r] <= w < start[r + 1]; its draws
// use that request's key and its index w - start[r] (the instance word), and
// its row of len[r] + 1 entries starts at path + row0[r] + (w - start[r]) *
// (len[r] + 1).  Device arrays.
struct WalkSegments {
    const uint64_t* __restrict__ start;   // [n + 1]
    const uint32_t* __restrict__ len;     // [n]
    const uint32_t* __restrict__ key;     // [2 n]
    const uint64_t* __restrict__ row0;    // [n]
    uint32_t n;
    // walkers a warp takes before its block exits (0: until all are done).
    // Short-lived blocks let the kernels of a request that arrives later
    // (on a higher-priority stream) start without waiting for this launch.
    uint32_t warp_budget;
};

// Which segment walker w is in, and its place there.
struct WalkerSlot {
    uint32_t k0, k1, id, L;
    uint64_t row0;
};

__device__ __forceinline__ WalkerSlot walker_slot(const WalkSegments& sg, uint64_t w)
{
    uint32_t lo = 0, hi = sg.n;   // last r with start[r] <= w
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(sg.start + mid) <= w) lo = mid; else hi = mid;
    }
    WalkerSlot ws;
    ws.id = (uint32_t)(w - __ldg(sg.start + lo));
    ws.L = __ldg(sg.len + lo);
    ws.k0 = __ldg(sg.key + 2 * lo);
    ws.k1 = __ldg(sg.key + 2 * lo + 1);
    ws.row0 = __ldg(sg.row0 + lo) + (uint64_t)ws.id * ((uint64_t)ws.L + 1);
    return ws;
}

// The walks of a batch of requests (same bias) in one launch: d_starts holds
// the n walkers of all requests in segment order, max_len is the longest
// length.  Results are those of csaw_walk for each request alone.  Defined
// in csaw_walk.cu.
csaw_status walk_batch(const csaw_graph* g, const csaw_bias* bias, const uint32_t* d_starts, uint64_t n,
                       const WalkSegments& seg, uint32_t max_len, uint32_t* d_path, cudaStream_t s);

// Checks a partition of a host CSR once it is on the device, so that the
// out-of-memory calls need no pass over every edge on the host: a column that
// is not a vertex is flagged (bit 1) and replaced by 0, a zero weight (when w
// is given) flagged (bit 2) and replaced by 1, and an edge into a vertex of
// degree 0 (when deg is given) flagged (bit 4).  The call then fails with
// CSAW_ERR_INVALID; the replacements only keep the kernels in bounds.
// Defined in csaw_oom.cu.
// Page-locks a caller's host range for the duration of a call (read-only
// registration where the device supports it, else ordinary); false if
// refused, with the CUDA error cleared.  Defined in csaw_oom.cu.
bool host_register(void* p, size_t bytes);

void launch_partition_check(uint32_t* col, uint32_t* w, uint64_t ne, uint32_t V, const uint32_t* deg,
                            uint32_t* err, cudaStream_t s);

// Walks that read a cached cumulative array (or, for uniform bias, none):
// one thread per walker.  Defined in csaw_walk.cu.
// cdf: the kind's cumulative array (cdf_words(E, V) words; ignored for
// uniform); leaf = false: summaries and records only, the leaf level formed
// from the edge weights (edge-weight bias).  Walkers w0 .. w0+n-1 of the
// call: starts and path point at walker w0's entries, and walker w0 + i
// draws as walker w0 + i.  Defined in csaw_walk_cdf.cu.
csaw_status launch_walk_cached(const csaw_graph* g, int kind, const uint64_t* cdf, bool leaf,
                               const uint32_t* starts, uint64_t w0, uint64_t n, uint32_t length, uint64_t rng_seed,
                               uint32_t* path, cudaStream_t s);
// The same walks with the path matrix copied to host memory h_path: the
// walkers run in a few chunks on s, and each chunk's rows are copied out on
// a second stream while the next chunk walks.  Returns after the copies.
// The host starts h_starts (the source of d_starts) are checked while the
// walks run: CSAW_ERR_INVALID for a start that is not a vertex.
// walked (or null) is recorded on s after the last walk kernel.
csaw_status walk_cached_to_host(const csaw_graph* g, int kind, const uint64_t* cdf, bool leaf,
                                const uint32_t* h_starts, const uint32_t* d_starts, uint64_t n, uint32_t length,
                                uint64_t rng_seed, uint32_t* d_path, uint32_t* h_path, cudaStream_t s,
                                cudaEvent_t walked);
// Walks over CSR arrays in host memory, read in place (coherent access to
// host memory): off, col and w (null: uniform) are host arrays, c holds
// device summaries and records of the weights (no leaf level).
struct CdfView;
csaw_status launch_walk_host(const CdfView& c, const uint64_t* off, const uint32_t* col, const uint32_t* w,
                             uint32_t V, uint64_t E, int sm_count, const uint32_t* starts, uint64_t n,
                             uint32_t length, uint64_t rng_seed, uint32_t* path, cudaStream_t s);
// The batched form (several requests, WalkSegments) over the graph's cached array.
csaw_status walk_batch_cached(const csaw_graph* g, int kind, const uint32_t* d_starts, uint64_t n,
                              const WalkSegments& seg, uint32_t max_len, uint32_t* d_path, cudaStream_t s);

// Whether selection/walks of this kind can use a cached cumulative array:
// uniform always (implicit), edge weight / neighbour degree when built and
// no bias of the kind is zero.
bool cached_cdf_usable(const csaw_graph* g, int kind);

// Whether every bias of a static kind is positive (the condition for walking
// or selecting over its cumulative array).
bool cdf_kind_positive(const csaw_graph* g, int kind);

// The cumulative array of a static kind and its search aids, in one
// allocation of cdf_layout(E, V).words words (each part 64-byte aligned):
//   cdf[E + pad]        inclusive row prefix sums, cdf[e] = b(row start) + ... + b(e)
//   s1[(E+7)/8 + 8]     s1[g] = cdf[8g + 7]      for 8g + 7 < E
//   s2[(E+63)/64 + 8]   s2[h] = cdf[64h + 63]    for 64h + 63 < E
//   rec[V][4]           rec[v] = {off[v], off[v+1], row total, 0}: one 32-byte sector
struct CdfLayout {
    uint64_t s1, s2, rec, words;   // word offsets and the total
};
__host__ __device__ inline CdfLayout cdf_layout(uint64_t E, uint64_t V)
{
    CdfLayout L;
    L.s1 = (E + CSAW_EDGE_PAD + 7) & ~7ull;
    L.s2 = (L.s1 + (E + 7) / 8 + 8 + 7) & ~7ull;
    L.rec = (L.s2 + (E + 63) / 64 + 8 + 7) & ~7ull;
    L.words = L.rec + 4 * V;
    return L;
}
// A summary-only array (edge weights: the leaf level is formed from the
// weights by w_search) has the same layout with cdf unused.
struct CdfView {
    const uint64_t* cdf = nullptr;
    const uint64_t* s1 = nullptr;
    const uint64_t* s2 = nullptr;
    const uint64_t* rec = nullptr;
};
__host__ __device__ inline CdfView cdf_view(const uint64_t* base, uint64_t E, uint64_t V)
{
    CdfView c;
    if (!base) return c;
    const CdfLayout L = cdf_layout(E, V);
    c.cdf = base;
    c.s1 = base + L.s1;
    c.s2 = base + L.s2;
    c.rec = base + L.rec;
    return c;
}
uint64_t cdf_words(uint64_t E, uint64_t V);

// Summaries and records alone (edge weights, no leaf level), in one
// allocation of wsum_layout(E, V).words words with s1 at word 0.
__host__ __device__ inline CdfLayout wsum_layout(uint64_t E, uint64_t V)
{
    CdfLayout L;
    L.s1 = 0;
    L.s2 = ((E + 7) / 8 + 8 + 7) & ~7ull;
    L.rec = (L.s2 + (E + 63) / 64 + 8 + 7) & ~7ull;
    L.words = L.rec + 4 * V;
    return L;
}
__host__ __device__ inline CdfView wsum_view(const uint64_t* base, uint64_t E, uint64_t V)
{
    CdfView c;
    if (!base) return c;
    const CdfLayout L = wsum_layout(E, V);
    c.s1 = base + L.s1;
    c.s2 = base + L.s2;
    c.rec = base + L.rec;
    return c;
}

// Enqueues the build of the cumulative array of a static kind and its
// search aids into cdf (cdf_words(E, V) words) on s; temporaries are
// stream-ordered.
csaw_status enqueue_cdf_build(const csaw_graph* g, int kind, uint64_t* cdf, cudaStream_t s);
// The same from raw CSR pointers (device, or host arrays read in place, with
// w 16-byte aligned), writing the leaf level to leaf (or, when leaf is null,
// only the summaries and records: edge weights) and the search aids to
// s1, s2, rec.
csaw_status enqueue_cdf_build_raw(const uint64_t* off, const uint32_t* col, const uint32_t* w, const uint32_t* deg,
                                  uint32_t V, uint64_t E, int sm_count, int kind, uint64_t* leaf, uint64_t* s1,
                                  uint64_t* s2, uint64_t* rec, cudaStream_t s);

// Releases a result made by the request server (tagged "CSRV").
void free_server_result(void* result);

// Several sampling requests in one multi-instance run (the request server's
// batches).  Device tables: each instance's Philox key (two words), its index
// within its request (the instance word of its draws) and its fanout at every
// layer ([depth][n_inst], 0 past its request's depth).  fan_max[l] (host) is
// the largest fanout of layer l.  The result has csaw_sample's layout over
// the batch's instances; each request's instances keep their own draws.
struct SampleTables {
    const uint32_t* inst_key;
    const uint32_t* inst_id;
    const uint32_t* inst_fan;
};
csaw_status sample_batch(csaw_graph* g, const uint32_t* d_seeds, const uint64_t* d_inst_off, uint32_t n_inst,
                         uint64_t n_seeds, uint32_t depth, const uint32_t* fan_max, const SampleTables& t,
                         int kind, cudaStream_t s, csaw_sample_result** out);

// Frees a result of sample_batch: its device edges stream-ordered on s (no
// device-wide synchronisation, unlike csaw_result_free, whose caller's stream
// may be gone), then the result.  For callers that own s.
void free_sample_result_on(csaw_sample_result* R, cudaStream_t s);

// Validation of a bias argument against a graph; fills the effective kind
// (EDGE_WEIGHT on a graph without weights is UNIFORM).
csaw_status check_bias(const csaw_graph* g, const csaw_bias* bias, bool allow_node2vec,
                       int* kind_out);

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC11): ten rounds, each two
// 32x32 -> 64-bit products of counter words 0 and 2 with the round
// multipliers, the high halves xored with the other counter words and the
// key; the key advances by the Weyl increments between rounds.
// Key = {lo32(seed), hi32(seed)}; counter = {attempt, vertex, layer, instance};
// the 64-bit draw is out1 << 32 | out0.
__device__ __forceinline__ uint64_t philox_draw(uint32_t k0, uint32_t k1, uint32_t attempt,
                                                uint32_t vertex, uint32_t layer,
                                                uint32_t instance)
{
    uint32_t c0 = attempt, c1 = vertex, c2 = layer, c3 = instance;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;   // one wide multiply: both halves
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        c0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        c1 = (uint32_t)p1;
        c2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c3 = (uint32_t)p0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return ((uint64_t)c1 << 32) | (uint64_t)c0;
}

// The ten round keys of one seed, computed once on the host: round r uses
// (k0 + r * 0x9E3779B9, k1 + r * 0xBB67AE85) mod 2^32.  Passed in a kernel's
// parameters, each is a constant operand of its round.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

inline PhiloxKeys philox_round_keys(uint64_t seed)
{
    PhiloxKeys K;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = k0;
        K.k1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return K;
}

// philox_draw with precomputed round keys (same output).
__device__ __forceinline__ uint64_t philox_draw(const PhiloxKeys& K, uint32_t attempt, uint32_t vertex,
                                                uint32_t layer, uint32_t instance)
{
    uint32_t c0 = attempt, c1 = vertex, c2 = layer, c3 = instance;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        c0 = (uint32_t)(p1 >> 32) ^ c1 ^ K.k0[r];
        c1 = (uint32_t)p1;
        c2 = (uint32_t)(p0 >> 32) ^ c3 ^ K.k1[r];
        c3 = (uint32_t)p0;
    }
    return ((uint64_t)c1 << 32) | (uint64_t)c0;
}

// x = floor(r * T / 2^64), the draw placed in [0, T).
__device__ __forceinline__ uint64_t scale_draw(uint64_t r, uint64_t total)
{
    return __umul64hi(r, total);
}

// ---------------------------------------------------------------------------
// Warp collectives on 64-bit values.
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(CSAW_FULL_MASK, x, o);
    return x;
}

__device__ __forceinline__ uint64_t warp_inclusive_scan_u64(uint64_t x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(CSAW_FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Membership of u in the sorted neighbour list col[beg, end) (node2vec's
// "is u adjacent to the previous vertex").
__device__ __forceinline__ bool sorted_contains(const uint32_t* __restrict__ col, uint64_t beg,
                                                uint64_t end, uint32_t u)
{
    const uint64_t row_end = end;
    while (beg < end) {
        const uint64_t mid = beg + ((end - beg) >> 1);
        const uint32_t c = __ldg(col + mid);
        if (c < u) beg = mid + 1; else end = mid;
    }
    return beg < row_end && __ldg(col + beg) == u;
}

// First i in [lo, hi) with a[i] > x (hi if none), where [lo, hi) lies in
// one aligned run a[8q .. 8q+7] and a does not decrease over [lo, hi):
// the run is read as two 32-byte halves, the second only when every entry
// of [lo, hi) in the first is <= x.  Reads a[8q .. 8q+7].  STREAM: loads
// marked evict-first (lines unlikely to be read again soon).
template <bool STREAM = false>
__device__ __forceinline__ ulonglong2 ld_pair(const ulonglong2* p)
{
    if constexpr (STREAM) return __ldcs(p);
    else return __ldg(p);
}

template <bool STREAM = false>
__device__ __forceinline__ uint64_t first_above8(const uint64_t* __restrict__ a, uint64_t lo, uint64_t hi,
                                                 uint64_t x)
{
    if (lo >= hi) return hi;
    const uint64_t q = lo & ~7ull, mid = q + 4;
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(a + q);
    if (lo < mid) {
        const ulonglong2 u0 = ld_pair<STREAM>(p), u1 = ld_pair<STREAM>(p + 1);
        const uint64_t v[4] = {u0.x, u0.y, u1.x, u1.y};
        const uint64_t h = hi < mid ? hi : mid;
        uint32_t le = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) le += q + j >= lo && q + j < h && v[j] <= x;
        if (lo + le < h || hi <= mid) return lo + le;
        lo = mid;
    }
    const ulonglong2 u2 = ld_pair<STREAM>(p + 2), u3 = ld_pair<STREAM>(p + 3);
    const uint64_t v[4] = {u2.x, u2.y, u3.x, u3.y};
    uint32_t le = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) le += mid + j >= lo && mid + j < hi && v[j] <= x;
    return lo + le;
}

// The 8-edge group of the hit: the group g of the smallest e in [beg, end)
// with cdf[e] > x, for x below the row total (a row of the cumulative array
// of c).  Every s2[h] with beg/64 <= h < (end-1)/64, and every s1[g] with
// beg/8 <= g < (end-1)/8, is a prefix sum of this row.  Bisecting the row's
// s2 entries finds the 64-edge block of the hit (the row's last block when
// none exceeds x); that block's s1 entries in the row (at most 7, one
// aligned run) give its group.  Reads stay inside s1, s2 and their padding.
__device__ __forceinline__ uint64_t cdf_group(const CdfView& c, uint64_t beg, uint64_t end, uint64_t x)
{
    uint64_t lo = beg >> 6, hi = (end - 1) >> 6;
    while (lo < hi) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(c.s2 + mid) > x) hi = mid; else lo = mid + 1;
    }
    const uint64_t g_lo = (lo << 3) > (beg >> 3) ? (lo << 3) : (beg >> 3);
    const uint64_t g_end = (end - 1) >> 3;
    const uint64_t g_hi = (lo << 3) + 7 < g_end ? (lo << 3) + 7 : g_end;
    return first_above8(c.s1, g_lo, g_hi, x);
}

// Smallest e in [beg, end) with cdf[e] > x: the group's entries in the row
// (one or two 32-byte sectors of the array).  STREAM_LEAF: the array's own
// sectors are read evict-first, so that they do not push the summaries out
// of L2.
template <bool STREAM_LEAF = false>
__device__ __forceinline__ uint64_t cdf_search(const CdfView& c, uint64_t beg, uint64_t end, uint64_t x)
{
    const uint64_t g = cdf_group(c, beg, end, x);
    const uint64_t e_lo = (g << 3) > beg ? (g << 3) : beg;
    const uint64_t e_hi = (g << 3) + 8 < end ? (g << 3) + 8 : end;
    return first_above8<STREAM_LEAF>(c.cdf, e_lo, e_hi, x);
}

// The same search without the array's leaf level (summaries and records
// only): the group's sums are formed from its biases w[8g .. 8g+7] (one
// 32-byte sector), starting from the previous summary entry s1[g-1] =
// cdf[8g-1] when that edge is in the row (else from 0 at the row start).
// PADDED: w is a graph array, 16-byte aligned and readable to E + 7, read
// as two 16-byte loads (evict-first); otherwise (arrays in host memory) the
// group is read entry by entry below E.
template <bool PADDED>
__device__ __forceinline__ uint64_t w_search(const CdfView& c, const uint32_t* __restrict__ w, uint64_t E,
                                             uint64_t beg, uint64_t end, uint64_t x)
{
    const uint64_t g = cdf_group(c, beg, end, x);
    const uint64_t gb = g << 3;
    const uint64_t e_lo = gb > beg ? gb : beg;
    const uint64_t e_hi = gb + 8 < end ? gb + 8 : end;
    uint64_t acc = gb > beg ? __ldg(c.s1 + g - 1) : 0ull;
    uint32_t v[8];
    if constexpr (PADDED) {
        const uint4 a = __ldcs(reinterpret_cast<const uint4*>(w + gb));
        const uint4 b = __ldcs(reinterpret_cast<const uint4*>(w + gb) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = gb + j < E ? w[gb + j] : 0u;
    }
    uint64_t hit = e_hi - 1;
    bool found = false;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint64_t pos = gb + j;
        const bool in = pos >= e_lo && pos < e_hi;
        if (in) acc += v[j];
        if (in && !found && acc > x) {
            hit = pos;
            found = true;
        }
    }
    return hit;
}

}  // namespace csaw
