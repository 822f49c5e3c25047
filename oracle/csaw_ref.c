/*
 * csaw_ref.c -- the oracle for C-SAW biased neighbour selection.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded C
 * statement of what the selection path computes.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or helper with the CUDA library; the CUDA library
 * never loads it.
 *
 * What it follows (Pandey et al., "C-SAW: A Framework for Graph Sampling and
 * Random Walk on GPUs", SC20):
 *   - Theorem 1 (Sec. II-B): a candidate is chosen with probability b_k / sum b.
 *   - Inverse transform sampling (Sec. II-B, Eq. 1): prefix sum S of the
 *     biases, a uniform draw, a binary search of the draw over S.  Here S is
 *     kept in integers: S[i] is the inclusive uint64 sum b[0] + ... + b[i],
 *     candidate i owns [S[i-1], S[i]), and a 64-bit draw r is mapped to
 *     x = floor(r * T / 2^64) in [0, T) with T = S[d-1].
 *   - Repeated sampling (Sec. IV-B, "Naive Solutions"): without replacement,
 *     redraw until an unselected candidate is hit; the first k distinct hits
 *     in draw order are the selection.
 *   - Updated sampling (Sec. IV-B, Fig. 5(b)): recompute the prefix sum with
 *     the selected candidates removed and search the draw there.  The oracle
 *     switches to this after a fixed number of attempts so that selection
 *     always ends (the paper notes that redrawing can need very many rounds
 *     on skewed biases).
 *   - EdgeBias (Sec. III-C, Eq. 3) with four fixed kinds: uniform, edge weight,
 *     neighbour degree, and node2vec's second-order bias (Sec. II-A): weight
 *     times m0 if the neighbour is the previous vertex, m1 if it is adjacent
 *     to the previous vertex, m2 otherwise.
 *   - The framework loop (Sec. III-B, Fig. 2(b)) for layered sampling, with
 *     Update (Eq. 4) filtering already visited vertices out of the next
 *     frontier (Sec. II-A: traversal sampling never samples a vertex twice).
 *   - Random walk (Sec. II-A): one neighbour per step, repeats allowed.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC11), written here from that definition.
 * Key = (low 32 bits of seed, high 32 bits of seed); counter =
 * (attempt, vertex, layer or step, instance); r = (out[1] << 32) | out[0].
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define REF_NONE 0xFFFFFFFFu
#define REF_FANOUT_ALL 0xFFFFFFFFu

enum { REF_OK = 0, REF_ERR_INVALID = 1, REF_ERR_NOMEM = 2, REF_ERR_OVERFLOW = 4 };
enum { REF_BIAS_UNIFORM = 0, REF_BIAS_EDGE_WEIGHT = 1, REF_BIAS_NEIGHBOR_DEGREE = 2,
       REF_BIAS_NODE2VEC = 3 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC11): ten rounds of two 32x32->64 products,
 * the key bumped by the Weyl constants between rounds.                       */

void ref_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The 64-bit draw for one attempt. */
uint64_t ref_draw(uint64_t seed, uint32_t attempt, uint32_t vertex, uint32_t layer,
                  uint32_t instance)
{
    uint32_t ctr[4] = { attempt, vertex, layer, instance };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    ref_philox4x32_10(ctr, key, out);
    return ((uint64_t)out[1] << 32) | (uint64_t)out[0];
}

/* x = floor(r * T / 2^64): a draw r in [0, 2^64) scaled to [0, T). */
uint64_t ref_scale(uint64_t r, uint64_t total)
{
    unsigned __int128 p = (unsigned __int128)r * (unsigned __int128)total;
    return (uint64_t)(p >> 64);
}

/* Index of the candidate whose interval [S[i-1], S[i]) holds x, i.e. the
 * smallest i with S[i] > x (S inclusive, x < S[d-1]).  Plain binary search. */
static uint32_t upper_bound_u64(const uint64_t* S, uint32_t d, uint64_t x)
{
    uint32_t lo = 0, hi = d;
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (S[mid] > x) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* ------------------------------------------------------------------------ */
/* Selection on an explicit bias array b[0..d-1].
 *
 * draw(ctx, a, &r) supplies the 64-bit draw r of attempt a and returns 0, or
 * returns nonzero when it has no draw for that attempt.
 *
 * Returns the number of picks written to out_idx (candidate indices, in the
 * order they were picked), -1 if the draws ran out first, -2 on allocation
 * failure.  k == REF_FANOUT_ALL takes every candidate of positive bias.
 * attempt_cap is the number of repeated-sampling attempts before the switch
 * to updated sampling.                                                       */
typedef int (*ref_draw_fn)(void* ctx, uint32_t attempt, uint64_t* r);

/* Counts kept for the attempts-per-pick measurement (Sec. VI reports
 * iterations per pick): the draws the selections consumed, and the picks of
 * the selections that drew (take-all selections draw nothing).  Counting
 * does not change any result; not thread-safe (the oracle is
 * single-threaded). */
static uint64_t g_attempts = 0, g_drawn_picks = 0;

void ref_stats(uint64_t out[2], int reset)
{
    out[0] = g_attempts;
    out[1] = g_drawn_picks;
    if (reset) g_attempts = g_drawn_picks = 0;
}

static int64_t select_core(const uint32_t* b, uint32_t d, uint32_t k, uint32_t attempt_cap,
                           ref_draw_fn draw, void* ctx, uint32_t* out_idx)
{
    if (d == 0 || k == 0) return 0;
    uint64_t* S = (uint64_t*)malloc(sizeof(uint64_t) * d);
    if (!S) return -2;
    uint64_t run = 0;
    uint32_t npos = 0;
    for (uint32_t i = 0; i < d; ++i) {
        run += b[i];
        S[i] = run;
        if (b[i] > 0) ++npos;
    }
    uint64_t T = run;
    if (T == 0) { free(S); return 0; }

    /* Not more positive candidates than asked for: take them all, CSR order. */
    if (k == REF_FANOUT_ALL || npos <= k) {
        uint32_t n = 0;
        for (uint32_t i = 0; i < d; ++i) if (b[i] > 0) out_idx[n++] = i;
        free(S);
        return n;
    }

    unsigned char* chosen = (unsigned char*)calloc(d, 1);
    uint64_t* S2 = (uint64_t*)malloc(sizeof(uint64_t) * d);
    if (!chosen || !S2) { free(S); free(chosen); free(S2); return -2; }

    int64_t have = 0;
    uint32_t a = 0;
    for (; have < (int64_t)k; ++a) {
        uint64_t r;
        if (draw(ctx, a, &r) != 0) { have = -1; break; }
        if (a < attempt_cap) {
            /* Repeated sampling: search the original prefix sums. */
            uint32_t i = upper_bound_u64(S, d, ref_scale(r, T));
            if (!chosen[i]) { chosen[i] = 1; out_idx[have++] = i; }
        } else {
            /* Updated sampling: prefix sums with the picked candidates removed. */
            uint64_t run2 = 0;
            for (uint32_t i = 0; i < d; ++i) {
                if (!chosen[i]) run2 += b[i];
                S2[i] = run2;
            }
            uint32_t i = upper_bound_u64(S2, d, ref_scale(r, run2));
            chosen[i] = 1;
            out_idx[have++] = i;
        }
    }
    if (have > 0) {
        g_attempts += a;
        g_drawn_picks += (uint64_t)have;
    }
    free(S); free(S2); free(chosen);
    return have;
}

/* Test hook: selection with the draws given as an array (draws[a] for
 * attempt a). */
typedef struct { const uint64_t* r; uint32_t n; } array_draws;

static int draw_from_array(void* ctx, uint32_t attempt, uint64_t* r)
{
    const array_draws* A = (const array_draws*)ctx;
    if (attempt >= A->n) return 1;
    *r = A->r[attempt];
    return 0;
}

int64_t ref_select_given_draws(const uint32_t* b, uint32_t d, uint32_t k, uint32_t attempt_cap,
                               const uint64_t* draws, uint32_t n_draws, uint32_t* out_idx)
{
    array_draws A = { draws, n_draws };
    return select_core(b, d, k, attempt_cap, draw_from_array, &A, out_idx);
}

/* ------------------------------------------------------------------------ */
/* Graph and EdgeBias (Eq. 3). */

typedef struct {
    const uint64_t* off;   /* [V+1] */
    const uint32_t* col;   /* [E], ascending within each row */
    const uint32_t* w;     /* [E] or NULL (all ones) */
    uint32_t V;
} ref_graph;

static int is_neighbour(const ref_graph* g, uint32_t t, uint32_t u)
{
    /* Binary search for u in t's sorted neighbour list. */
    uint64_t lo = g->off[t], hi = g->off[t + 1];
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (g->col[mid] < u) lo = mid + 1; else hi = mid;
    }
    return lo < g->off[t + 1] && g->col[lo] == u;
}

/* Biases of all neighbours of v into b[0..d-1]. */
static int edge_biases(const ref_graph* g, uint32_t v, int kind, const uint32_t mult[3],
                       uint32_t prev, uint32_t* b)
{
    uint64_t beg = g->off[v], end = g->off[v + 1];
    for (uint64_t e = beg; e < end; ++e) {
        uint32_t u = g->col[e];
        uint32_t w = g->w ? g->w[e] : 1u;
        uint64_t val;
        switch (kind) {
        case REF_BIAS_UNIFORM: val = 1; break;
        case REF_BIAS_EDGE_WEIGHT: val = w; break;
        case REF_BIAS_NEIGHBOR_DEGREE: val = g->off[u + 1] - g->off[u]; break;
        case REF_BIAS_NODE2VEC:
            if (prev == REF_NONE) val = w;
            else if (u == prev) val = (uint64_t)w * mult[0];
            else if (is_neighbour(g, prev, u)) val = (uint64_t)w * mult[1];
            else val = (uint64_t)w * mult[2];
            break;
        default: return REF_ERR_INVALID;
        }
        if (val > 0xFFFFFFFFull) return REF_ERR_OVERFLOW;
        b[e - beg] = (uint32_t)val;
    }
    return REF_OK;
}

typedef struct { uint64_t seed; uint32_t vertex, layer, instance; } key_draws;

static int draw_from_key(void* ctx, uint32_t attempt, uint64_t* r)
{
    const key_draws* K = (const key_draws*)ctx;
    *r = ref_draw(K->seed, attempt, K->vertex, K->layer, K->instance);
    return 0;
}

/* Biased selection of up to k neighbours of v without replacement.  Writes
 * neighbour vertex ids (not indices) to out, returns the count or a negative
 * error. */
int64_t ref_select(const uint64_t* off, const uint32_t* col, const uint32_t* w, uint32_t V,
                   uint32_t v, uint32_t k, int kind, const uint32_t mult[3], uint32_t prev,
                   uint64_t seed, uint32_t layer, uint32_t instance, uint32_t attempt_cap,
                   uint32_t* out)
{
    ref_graph g = { off, col, w, V };
    uint32_t d = (uint32_t)(off[v + 1] - off[v]);
    if (d == 0) return 0;
    uint32_t* b = (uint32_t*)malloc(sizeof(uint32_t) * d);
    uint32_t* idx = (uint32_t*)malloc(sizeof(uint32_t) * d);
    if (!b || !idx) { free(b); free(idx); return -2; }
    int rc = edge_biases(&g, v, kind, mult, prev, b);
    if (rc != REF_OK) { free(b); free(idx); return -(int64_t)rc - 10; }
    key_draws K = { seed, v, layer, instance };
    int64_t n = select_core(b, d, k, attempt_cap, draw_from_key, &K, idx);
    for (int64_t j = 0; j < n; ++j) out[j] = col[off[v] + idx[j]];
    free(b); free(idx);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Random walk (Sec. II-A; node2vec's second-order bias when kind is
 * NODE2VEC).  path is [n][L+1] row-major; path[w][0] = start.  The draw of
 * walker w at step s is attempt 0, vertex = current vertex, layer = s,
 * instance = walker_ids ? walker_ids[w] : w.  A walker at a vertex with no
 * neighbour of positive bias stops; the rest of its row is REF_NONE.
 *
 * Random walk with restart or with jump (Sec. II-A; the Update of Eq. 4 that
 * returns a vertex other than the sampled neighbour): when tele is
 * REF_TELE_RESTART or REF_TELE_JUMP, each step first draws attempt 1 (same
 * vertex, layer and instance); if its upper 32 bits are below tele_q32 the
 * step teleports instead of moving to a neighbour: to the walker's start
 * (restart) or to vertex floor(r2 * V / 2^64) with r2 the draw of attempt 2
 * (jump).  A walker at a vertex with no neighbour of positive bias teleports
 * the same way instead of stopping.  After a teleport the walk has no
 * previous vertex (node2vec's next step uses the weights alone).           */
#define REF_TELE_NONE 0
#define REF_TELE_RESTART 1
#define REF_TELE_JUMP 2

static uint32_t teleport_target(int tele, uint32_t start, uint32_t V, uint64_t seed, uint32_t cur,
                                uint32_t s, uint32_t inst)
{
    if (tele == REF_TELE_RESTART) return start;
    return (uint32_t)ref_scale(ref_draw(seed, 2, cur, s, inst), V);
}

int ref_walk_tele(const uint64_t* off, const uint32_t* col, const uint32_t* w, uint32_t V,
                  const uint32_t* starts, const uint64_t* walker_ids, uint64_t n, uint32_t L,
                  int kind, const uint32_t mult[3], uint64_t seed, int tele, uint32_t tele_q32,
                  uint32_t* path)
{
    if (tele != REF_TELE_NONE && tele != REF_TELE_RESTART && tele != REF_TELE_JUMP)
        return REF_ERR_INVALID;
    ref_graph g = { off, col, w, V };
    uint32_t maxd = 0;
    for (uint32_t v = 0; v < V; ++v) {
        uint64_t d = off[v + 1] - off[v];
        if (d > maxd) maxd = (uint32_t)d;
    }
    uint32_t* b = (uint32_t*)malloc(sizeof(uint32_t) * (maxd ? maxd : 1));
    uint64_t* S = (uint64_t*)malloc(sizeof(uint64_t) * (maxd ? maxd : 1));
    if (!b || !S) { free(b); free(S); return REF_ERR_NOMEM; }
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t* row = path + i * (uint64_t)(L + 1);
        uint32_t inst = walker_ids ? (uint32_t)walker_ids[i] : (uint32_t)i;
        uint32_t cur = starts[i], prev = REF_NONE;
        if (cur >= V) { free(b); free(S); return REF_ERR_INVALID; }
        row[0] = cur;
        uint32_t s = 0;
        for (; s < L; ++s) {
            if (tele != REF_TELE_NONE && (uint32_t)(ref_draw(seed, 1, cur, s, inst) >> 32) < tele_q32) {
                cur = teleport_target(tele, starts[i], V, seed, cur, s, inst);
                prev = REF_NONE;
                row[s + 1] = cur;
                continue;
            }
            uint32_t d = (uint32_t)(off[cur + 1] - off[cur]);
            int rc = edge_biases(&g, cur, kind, mult, prev, b);
            if (rc != REF_OK) { free(b); free(S); return rc; }
            uint64_t run = 0;
            for (uint32_t j = 0; j < d; ++j) { run += b[j]; S[j] = run; }
            if (d == 0 || run == 0) {              /* dead end */
                if (tele == REF_TELE_NONE) break;
                cur = teleport_target(tele, starts[i], V, seed, cur, s, inst);
                prev = REF_NONE;
                row[s + 1] = cur;
                continue;
            }
            uint64_t x = ref_scale(ref_draw(seed, 0, cur, s, inst), run);
            uint32_t j = upper_bound_u64(S, d, x);
            prev = cur;
            cur = col[off[cur] + j];
            row[s + 1] = cur;
        }
        for (uint32_t t = s; t < L; ++t) row[t + 1] = REF_NONE;
    }
    free(b); free(S);
    return REF_OK;
}

int ref_walk(const uint64_t* off, const uint32_t* col, const uint32_t* w, uint32_t V,
             const uint32_t* starts, const uint64_t* walker_ids, uint64_t n, uint32_t L,
             int kind, const uint32_t mult[3], uint64_t seed, uint32_t* path)
{
    return ref_walk_tele(off, col, w, V, starts, walker_ids, n, L, kind, mult, seed, REF_TELE_NONE, 0,
                         path);
}

/* ------------------------------------------------------------------------ */
/* Layered sampling (Fig. 2(b) loop, Update of Eq. 4 as a visited filter).
 *
 * Instance i owns seeds[inst_off[i] .. inst_off[i+1]).  Its layer-0 frontier
 * is the sorted set of its seeds; visited starts as that set.  At layer l,
 * every frontier vertex v (ascending) selects up to fanout[l] neighbours
 * (attempt keys: vertex v, layer l, instance i) and emits one edge (v, u) per
 * pick, in pick order.  The next frontier is the sorted set of picked
 * vertices minus visited; it is then added to visited.
 *
 * Output: edges grouped by layer, then instance, then source vertex
 * ascending.  edge_off[l * n_inst + i] .. edge_off[l * n_inst + i + 1] is the
 * edge range of (layer l, instance i); edge_off has depth*n_inst+1 entries.
 * frontier sizes per (layer, instance) go to fsize[(depth+1) * n_inst]
 * (layer 0 = deduplicated seeds).  All output arrays are malloc'd here and
 * released with ref_free.                                                    */

static int cmp_u32(const void* a, const void* b)
{
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

static uint32_t sort_unique(uint32_t* a, uint32_t n)
{
    if (n == 0) return 0;
    qsort(a, n, sizeof(uint32_t), cmp_u32);
    uint32_t m = 1;
    for (uint32_t i = 1; i < n; ++i) if (a[i] != a[m - 1]) a[m++] = a[i];
    return m;
}

static int in_sorted(const uint32_t* a, uint32_t n, uint32_t x)
{
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo < n && a[lo] == x;
}

typedef struct { uint32_t* src; uint32_t* dst; uint64_t n, cap; } edge_buf;

static int push_edge(edge_buf* e, uint32_t s, uint32_t d)
{
    if (e->n == e->cap) {
        uint64_t nc = e->cap ? 2 * e->cap : 64;
        uint32_t* ns = (uint32_t*)realloc(e->src, nc * sizeof(uint32_t));
        if (!ns) return REF_ERR_NOMEM;
        e->src = ns;
        uint32_t* nd = (uint32_t*)realloc(e->dst, nc * sizeof(uint32_t));
        if (!nd) return REF_ERR_NOMEM;
        e->dst = nd;
        e->cap = nc;
    }
    e->src[e->n] = s; e->dst[e->n] = d; e->n++;
    return REF_OK;
}

/* Layer sampling (Sec. II-A; Sec. III-B, Fig. 2(b) with the whole frontier as
 * the current frontier): every edge (v, u) of the instance's frontier, in
 * ascending v and then CSR order, is one entry of the NeighborPool; EdgeBias
 * gives each its bias; Select picks k entries without replacement by the
 * same rule as a vertex's neighbours (select_core), with draws keyed
 * {attempt, NONE, layer, instance}.  Picks go to E in pick order. */
static int layer_select(const ref_graph* g, const uint32_t* F, uint32_t nf, uint32_t k, int kind,
                        const uint32_t mult[3], uint64_t seed, uint32_t layer, uint32_t inst,
                        uint32_t attempt_cap, edge_buf* E)
{
    uint64_t D = 0;
    for (uint32_t fi = 0; fi < nf; ++fi) D += g->off[F[fi] + 1] - g->off[F[fi]];
    if (D >= 0xFFFFFFFFull) return REF_ERR_INVALID;
    uint32_t* b = (uint32_t*)malloc(sizeof(uint32_t) * (D ? D : 1));
    uint32_t* idx = (uint32_t*)malloc(sizeof(uint32_t) * (D ? D : 1));
    uint64_t* start = (uint64_t*)malloc(sizeof(uint64_t) * ((uint64_t)nf + 1));
    if (!b || !idx || !start) { free(b); free(idx); free(start); return REF_ERR_NOMEM; }
    uint64_t pos = 0;
    int rc = REF_OK;
    for (uint32_t fi = 0; fi < nf && rc == REF_OK; ++fi) {
        start[fi] = pos;
        rc = edge_biases(g, F[fi], kind, mult, REF_NONE, b + pos);
        pos += g->off[F[fi] + 1] - g->off[F[fi]];
    }
    start[nf] = pos;
    if (rc == REF_OK) {
        key_draws K = { seed, REF_NONE, layer, inst };
        int64_t n = select_core(b, (uint32_t)D, k, attempt_cap, draw_from_key, &K, idx);
        if (n < 0) rc = REF_ERR_NOMEM;
        for (int64_t j = 0; j < n && rc == REF_OK; ++j) {
            uint32_t lo = 0, hi = nf;   /* the pool entry's frontier vertex: last start <= idx */
            while (hi - lo > 1) {
                uint32_t mid = (lo + hi) / 2;
                if (start[mid] <= idx[j]) lo = mid; else hi = mid;
            }
            uint32_t v = F[lo];
            rc = push_edge(E, v, g->col[g->off[v] + (idx[j] - start[lo])]);
        }
    }
    free(b); free(idx); free(start);
    return rc;
}

static int sample_impl(const uint64_t* off, const uint32_t* col, const uint32_t* w, uint32_t V,
                       const uint32_t* seeds, const uint64_t* inst_off, uint32_t n_inst,
                       uint32_t depth, const uint32_t* fanout, int kind, const uint32_t mult[3],
                       uint64_t seed, uint32_t attempt_cap, int layer_mode,
                       uint32_t** out_src, uint32_t** out_dst, uint64_t** out_edge_off,
                       uint64_t** out_fsize)
{
    ref_graph gr = { off, col, w, V };
    if (kind == REF_BIAS_NODE2VEC) return REF_ERR_INVALID;   /* needs a walk's previous vertex */
    uint64_t ngroups = (uint64_t)depth * n_inst;
    edge_buf* per = (edge_buf*)calloc(ngroups ? ngroups : 1, sizeof(edge_buf));
    uint64_t* fsize = (uint64_t*)calloc((uint64_t)(depth + 1) * n_inst + 1, sizeof(uint64_t));
    uint32_t maxd = 0;
    for (uint32_t v = 0; v < V; ++v) {
        uint64_t d = off[v + 1] - off[v];
        if (d > maxd) maxd = (uint32_t)d;
    }
    uint32_t* picks = (uint32_t*)malloc(sizeof(uint32_t) * (maxd ? maxd : 1));
    if (!per || !fsize || !picks) { free(per); free(fsize); free(picks); return REF_ERR_NOMEM; }
    int rc = REF_OK;

    for (uint32_t i = 0; i < n_inst && rc == REF_OK; ++i) {
        uint64_t ns = inst_off[i + 1] - inst_off[i];
        uint32_t* F = (uint32_t*)malloc(sizeof(uint32_t) * (ns ? ns : 1));
        uint32_t* visited = (uint32_t*)malloc(sizeof(uint32_t) * (ns ? ns : 1));
        if (!F || !visited) { free(F); free(visited); rc = REF_ERR_NOMEM; break; }
        for (uint64_t j = 0; j < ns; ++j) {
            F[j] = seeds[inst_off[i] + j];
            if (F[j] >= V) rc = REF_ERR_INVALID;
        }
        if (rc != REF_OK) { free(F); free(visited); break; }
        uint32_t nf = sort_unique(F, (uint32_t)ns);
        memcpy(visited, F, sizeof(uint32_t) * nf);
        uint32_t nvis = nf;
        fsize[i] = nf;

        for (uint32_t l = 0; l < depth && rc == REF_OK; ++l) {
            edge_buf* E = &per[(uint64_t)l * n_inst + i];
            if (layer_mode) {
                rc = layer_select(&gr, F, nf, fanout[l], kind, mult, seed, l, i, attempt_cap, E);
            } else {
                for (uint32_t fi = 0; fi < nf; ++fi) {
                    uint32_t v = F[fi];
                    int64_t n = ref_select(off, col, w, V, v, fanout[l], kind, mult, REF_NONE,
                                           seed, l, i, attempt_cap, picks);
                    if (n < 0) { rc = n == -2 ? REF_ERR_NOMEM : REF_ERR_OVERFLOW; break; }
                    for (int64_t j = 0; j < n && rc == REF_OK; ++j) rc = push_edge(E, v, picks[j]);
                }
            }
            if (rc != REF_OK) break;
            /* Update: next frontier = sorted set of picks minus visited. */
            uint32_t* cand = (uint32_t*)malloc(sizeof(uint32_t) * (E->n ? E->n : 1));
            if (!cand) { rc = REF_ERR_NOMEM; break; }
            memcpy(cand, E->dst, sizeof(uint32_t) * E->n);
            uint32_t nc = sort_unique(cand, (uint32_t)E->n);
            uint32_t nn = 0;
            for (uint32_t j = 0; j < nc; ++j)
                if (!in_sorted(visited, nvis, cand[j])) cand[nn++] = cand[j];
            /* visited := visited U next (both sorted, disjoint): merge. */
            uint32_t* nv = (uint32_t*)malloc(sizeof(uint32_t) * ((uint64_t)nvis + nn + 1));
            if (!nv) { free(cand); rc = REF_ERR_NOMEM; break; }
            uint32_t a = 0, b2 = 0, m = 0;
            while (a < nvis || b2 < nn) {
                if (b2 >= nn || (a < nvis && visited[a] < cand[b2])) nv[m++] = visited[a++];
                else nv[m++] = cand[b2++];
            }
            free(visited); visited = nv; nvis = m;
            free(F); F = cand; nf = nn;
            fsize[(uint64_t)(l + 1) * n_inst + i] = nf;
        }
        free(F); free(visited);
    }

    if (rc == REF_OK) {
        uint64_t total = 0;
        for (uint64_t gix = 0; gix < ngroups; ++gix) total += per[gix].n;
        uint32_t* src = (uint32_t*)malloc(sizeof(uint32_t) * (total ? total : 1));
        uint32_t* dst = (uint32_t*)malloc(sizeof(uint32_t) * (total ? total : 1));
        uint64_t* eo = (uint64_t*)malloc(sizeof(uint64_t) * (ngroups + 1));
        if (!src || !dst || !eo) { free(src); free(dst); free(eo); rc = REF_ERR_NOMEM; }
        else {
            uint64_t p = 0;
            for (uint64_t gix = 0; gix < ngroups; ++gix) {
                eo[gix] = p;
                if (per[gix].n) {
                    memcpy(src + p, per[gix].src, sizeof(uint32_t) * per[gix].n);
                    memcpy(dst + p, per[gix].dst, sizeof(uint32_t) * per[gix].n);
                }
                p += per[gix].n;
            }
            eo[ngroups] = p;
            *out_src = src; *out_dst = dst; *out_edge_off = eo; *out_fsize = fsize;
        }
    }
    for (uint64_t gix = 0; gix < ngroups; ++gix) { free(per[gix].src); free(per[gix].dst); }
    free(per); free(picks);
    if (rc != REF_OK) free(fsize);
    return rc;
}

int ref_sample(const uint64_t* off, const uint32_t* col, const uint32_t* w, uint32_t V,
               const uint32_t* seeds, const uint64_t* inst_off, uint32_t n_inst,
               uint32_t depth, const uint32_t* fanout, int kind, const uint32_t mult[3],
               uint64_t seed, uint32_t attempt_cap,
               uint32_t** out_src, uint32_t** out_dst, uint64_t** out_edge_off,
               uint64_t** out_fsize)
{
    return sample_impl(off, col, w, V, seeds, inst_off, n_inst, depth, fanout, kind, mult, seed,
                       attempt_cap, 0, out_src, out_dst, out_edge_off, out_fsize);
}

/* Layer sampling: ref_sample's loop with layer_select in place of the
 * per-vertex selection; layer_size[l] is the number of pool entries picked
 * per instance at layer l. */
int ref_layer_sample(const uint64_t* off, const uint32_t* col, const uint32_t* w, uint32_t V,
                     const uint32_t* seeds, const uint64_t* inst_off, uint32_t n_inst,
                     uint32_t depth, const uint32_t* layer_size, int kind, uint64_t seed,
                     uint32_t attempt_cap, uint32_t** out_src, uint32_t** out_dst,
                     uint64_t** out_edge_off, uint64_t** out_fsize)
{
    const uint32_t ones[3] = { 1, 1, 1 };
    return sample_impl(off, col, w, V, seeds, inst_off, n_inst, depth, layer_size, kind, ones, seed,
                       attempt_cap, 1, out_src, out_dst, out_edge_off, out_fsize);
}

/* Multi-dimensional random walk (frontier sampling), Sec. II-A, written with
 * the API of Sec. III-C as the case study of Sec. III-D applies it (Figs. 3
 * and 4).  Each instance keeps a pool of pool_size vertices (slot order).
 * At step s:
 *   VertexBias (Eq. 2): the bias of a pool vertex is its degree; a slot whose
 *     entry is not a vertex (>= V, e.g. NONE) has bias 0.
 *   Select: one slot by inverse transform sampling over the pool's prefix sums
 *     in slot order, draw counter {0, NONE, s, instance}.
 *   EdgeBias = 1 (Sec. III-D): one neighbour u of the chosen v, S[t] = t + 1,
 *     draw counter {0, v, s, instance} (the counter of a walk step at v).
 *   Update (Eq. 4): u replaces v in its slot; (v, u) is the step's sampled
 *     edge.
 * A pool whose biases sum to 0 stops the instance; the rest of its rows of
 * src and dst is NONE.  instance_ids (may be NULL) gives each instance's RNG
 * index when only a subset is run. */
int ref_mdrw(const uint64_t* off, const uint32_t* col, uint32_t V, const uint32_t* pools,
             const uint64_t* instance_ids, uint64_t n, uint32_t pool_size, uint32_t steps,
             uint64_t seed, uint32_t* src, uint32_t* dst)
{
    if (pool_size == 0) return REF_ERR_INVALID;
    uint32_t maxd = 0;
    for (uint32_t v = 0; v < V; ++v) {
        uint64_t d = off[v + 1] - off[v];
        if (d > maxd) maxd = (uint32_t)d;
    }
    uint32_t* pool = (uint32_t*)malloc(sizeof(uint32_t) * pool_size);
    uint64_t* S = (uint64_t*)malloc(sizeof(uint64_t) * pool_size);
    uint64_t* Sn = (uint64_t*)malloc(sizeof(uint64_t) * (maxd ? maxd : 1));
    if (!pool || !S || !Sn) { free(pool); free(S); free(Sn); return REF_ERR_NOMEM; }
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t inst = instance_ids ? (uint32_t)instance_ids[i] : (uint32_t)i;
        uint32_t* srow = src + i * (uint64_t)steps;
        uint32_t* drow = dst + i * (uint64_t)steps;
        memcpy(pool, pools + i * (uint64_t)pool_size, sizeof(uint32_t) * pool_size);
        uint32_t s = 0;
        for (; s < steps; ++s) {
            /* VertexBias and the pool's prefix sums */
            uint64_t run = 0;
            for (uint32_t j = 0; j < pool_size; ++j) {
                uint32_t v = pool[j];
                run += v < V ? off[v + 1] - off[v] : 0;
                S[j] = run;
            }
            if (run == 0) break;
            uint64_t x = ref_scale(ref_draw(seed, 0, REF_NONE, s, inst), run);
            uint32_t slot = upper_bound_u64(S, pool_size, x);
            uint32_t v = pool[slot];
            /* EdgeBias = 1 over N(v) */
            uint32_t d = (uint32_t)(off[v + 1] - off[v]);
            for (uint32_t t = 0; t < d; ++t) Sn[t] = (uint64_t)t + 1;
            uint64_t y = ref_scale(ref_draw(seed, 0, v, s, inst), d);
            uint32_t u = col[off[v] + upper_bound_u64(Sn, d, y)];
            /* Update */
            pool[slot] = u;
            srow[s] = v;
            drow[s] = u;
        }
        for (; s < steps; ++s) { srow[s] = REF_NONE; drow[s] = REF_NONE; }
    }
    free(pool); free(S); free(Sn);
    return REF_OK;
}

void ref_free(void* p) { free(p); }
