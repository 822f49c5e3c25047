/*
 * csaw_inputs.c -- seeded synthetic inputs for C-SAW workloads.
 *
 * This module makes graphs and seed sets; it holds none of the selection
 * arithmetic.  Its random numbers come from SplitMix64 (Steele, Lea, Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014), keyed per
 * item so every output is a pure function of (parameters, seed), identical on
 * every machine.  The selection path draws its own numbers with Philox; the
 * two generators are unrelated.
 *
 * Graphs are RMAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): each of the
 * edge_factor * 2^scale edge draws descends `scale` levels, choosing one of the
 * four quadrants with probabilities (a, b, c, 1-a-b-c).  Vertex labels are
 * then permuted by a seeded Feistel network so that hubs are spread over the
 * id space.  Self-loops are dropped, every edge is stored in both directions,
 * rows are sorted ascending and duplicates removed.  The undirected edge
 * {u, v} gets one weight, 1 + (hash(seed, min, max) mod wmax), so both
 * directions carry the same weight.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t sm_next(uint64_t* s)
{
    *s += 0x9E3779B97F4A7C15ull;
    return mix64(*s);
}

/* Stream state of item `idx` in stream `stream` of generator seed `seed`. */
static inline uint64_t stream_state(uint64_t seed, uint64_t stream, uint64_t idx)
{
    return mix64(seed * 0xD1B54A32D192ED03ull + stream) ^ mix64(idx * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull);
}

/* ---- Feistel permutation of [0, 2^scale) ---- */
typedef struct { uint32_t lo_bits, hi_bits; uint64_t key[6]; } feistel;

static void feistel_init(feistel* f, uint32_t scale, uint64_t seed)
{
    f->lo_bits = scale / 2;
    f->hi_bits = scale - f->lo_bits;
    for (int r = 0; r < 6; ++r) f->key[r] = mix64(seed ^ (0xA0761D6478BD642Full * (uint64_t)(r + 1)));
}

static inline uint32_t feistel_apply(const feistel* f, uint32_t x)
{
    if (f->lo_bits == 0) return x;
    uint32_t lm = (1u << f->lo_bits) - 1u;
    uint32_t hm = (f->hi_bits >= 32) ? 0xFFFFFFFFu : ((1u << f->hi_bits) - 1u);
    uint32_t L = x & lm, H = (x >> f->lo_bits) & hm;
    for (int r = 0; r < 6; ++r) {
        if (r & 1) H ^= (uint32_t)mix64(L ^ f->key[r]) & hm;
        else       L ^= (uint32_t)mix64(H ^ f->key[r]) & lm;
    }
    return (H << f->lo_bits) | L;
}

/* ---- RMAT edge draws (multi-threaded; each edge is a pure function of its index) ---- */
typedef struct {
    uint32_t scale; uint64_t seed; uint64_t ta, tb, tc;
    const feistel* perm;
    uint64_t begin, end;
    uint32_t* src; uint32_t* dst;
} draw_job;

static void* draw_worker(void* p)
{
    draw_job* J = (draw_job*)p;
    for (uint64_t e = J->begin; e < J->end; ++e) {
        uint64_t s = stream_state(J->seed, 1, e);
        uint32_t u = 0, v = 0;
        for (uint32_t lvl = 0; lvl < J->scale; ++lvl) {
            uint64_t r = sm_next(&s);
            uint32_t ub, vb;
            if (r < J->ta) { ub = 0; vb = 0; }
            else if (r < J->tb) { ub = 0; vb = 1; }
            else if (r < J->tc) { ub = 1; vb = 0; }
            else { ub = 1; vb = 1; }
            u = (u << 1) | ub;
            v = (v << 1) | vb;
        }
        J->src[e] = feistel_apply(J->perm, u);
        J->dst[e] = feistel_apply(J->perm, v);
    }
    return NULL;
}

static uint64_t prob_threshold(double p)
{
    if (p <= 0.0) return 0;
    if (p >= 1.0) return UINT64_MAX;
    return (uint64_t)(p * 18446744073709551616.0);
}

/* Raw directed RMAT draws (before symmetrisation); src/dst have n_draws entries. */
int csaw_gen_rmat_draws(uint32_t scale, uint64_t n_draws, double a, double b, double c,
                        uint64_t seed, int n_threads, uint32_t* src, uint32_t* dst)
{
    if (scale == 0 || scale > 31) return 1;
    feistel perm;
    feistel_init(&perm, scale, seed ^ 0x5851F42D4C957F2Dull);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    draw_job jobs[256];
    pthread_t th[256];
    uint64_t chunk = (n_draws + (uint64_t)n_threads - 1) / (uint64_t)n_threads;
    for (int t = 0; t < n_threads; ++t) {
        jobs[t].scale = scale; jobs[t].seed = seed;
        jobs[t].ta = prob_threshold(a); jobs[t].tb = prob_threshold(a + b);
        jobs[t].tc = prob_threshold(a + b + c);
        jobs[t].perm = &perm;
        jobs[t].begin = (uint64_t)t * chunk;
        jobs[t].end = jobs[t].begin + chunk > n_draws ? n_draws : jobs[t].begin + chunk;
        if (jobs[t].begin > n_draws) jobs[t].begin = n_draws;
        jobs[t].src = src; jobs[t].dst = dst;
    }
    for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, draw_worker, &jobs[t]);
    draw_worker(&jobs[0]);
    for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
    return 0;
}

/* ---- CSR build: symmetrise, drop self-loops, sort rows, dedup ----
 * Two stable counting sorts (by destination, then by source) give rows sorted
 * ascending.  off has V+1 entries; col must hold 2 * n_draws entries; the
 * number of directed edges kept is returned in *n_edges.                    */
int csaw_gen_build_csr(uint32_t V, uint64_t n_draws, const uint32_t* src, const uint32_t* dst,
                       uint64_t* off, uint32_t* col, uint64_t* n_edges)
{
    uint64_t M = 0;
    uint64_t* cnt = (uint64_t*)calloc((uint64_t)V + 1, sizeof(uint64_t));
    if (!cnt) return 2;
    for (uint64_t e = 0; e < n_draws; ++e) {
        if (src[e] == dst[e]) continue;
        cnt[dst[e]]++; cnt[src[e]]++;
        M += 2;
    }
    uint32_t* ts = (uint32_t*)malloc(sizeof(uint32_t) * (M ? M : 1));   /* sorted by destination */
    uint32_t* td = (uint32_t*)malloc(sizeof(uint32_t) * (M ? M : 1));
    if (!ts || !td) { free(cnt); free(ts); free(td); return 2; }
    /* pass 1: by destination (key = second endpoint of each directed copy) */
    uint64_t run = 0;
    for (uint32_t v = 0; v < V; ++v) { uint64_t c0 = cnt[v]; cnt[v] = run; run += c0; }
    for (uint64_t e = 0; e < n_draws; ++e) {
        uint32_t u = src[e], v = dst[e];
        if (u == v) continue;
        uint64_t p = cnt[v]++; ts[p] = u; td[p] = v;     /* directed u -> v */
        p = cnt[u]++; ts[p] = v; td[p] = u;              /* directed v -> u */
    }
    /* pass 2: stable by source into col, rows then ascending by destination */
    memset(cnt, 0, sizeof(uint64_t) * ((uint64_t)V + 1));
    for (uint64_t p = 0; p < M; ++p) cnt[ts[p]]++;
    run = 0;
    for (uint32_t v = 0; v < V; ++v) { uint64_t c0 = cnt[v]; cnt[v] = run; run += c0; }
    uint64_t* start = (uint64_t*)malloc(sizeof(uint64_t) * ((uint64_t)V + 1));
    if (!start) { free(cnt); free(ts); free(td); return 2; }
    memcpy(start, cnt, sizeof(uint64_t) * V);
    start[V] = M;
    for (uint64_t p = 0; p < M; ++p) col[cnt[ts[p]]++] = td[p];
    free(ts); free(td);
    /* dedup within rows, compacting in place */
    uint64_t w = 0;
    for (uint32_t v = 0; v < V; ++v) {
        off[v] = w;
        uint64_t b0 = start[v], e0 = start[v + 1];
        for (uint64_t p = b0; p < e0; ++p) {
            if (p > b0 && col[p] == col[p - 1]) continue;
            col[w++] = col[p];
        }
    }
    off[V] = w;
    *n_edges = w;
    free(start); free(cnt);
    return 0;
}

/* Weight of every directed edge: 1 + hash(seed, min(u,v), max(u,v)) mod wmax. */
int csaw_gen_weights(uint32_t V, const uint64_t* off, const uint32_t* col, uint32_t wmax,
                     uint64_t seed, uint32_t* w)
{
    if (wmax == 0) return 1;
    for (uint32_t u = 0; u < V; ++u) {
        for (uint64_t p = off[u]; p < off[u + 1]; ++p) {
            uint32_t v = col[p];
            uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
            uint64_t h = mix64(stream_state(seed, 2, (lo << 32) | hi));
            w[p] = 1u + (uint32_t)(h % wmax);
        }
    }
    return 0;
}

/* n vertices drawn uniformly from [0, V) (repeats allowed), stream `stream`. */
int csaw_gen_uniform_vertices(uint64_t n, uint32_t V, uint64_t seed, uint64_t stream, uint32_t* out)
{
    if (V == 0) return 1;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t s = stream_state(seed, 100 + stream, i);
        out[i] = (uint32_t)(sm_next(&s) % V);
    }
    return 0;
}

/* Instance sizes n_i = floor(2^(lo_exp + span * u)), u uniform in [0, 1). */
int csaw_gen_loguniform_sizes(uint32_t n_inst, double lo_exp, double span, uint64_t seed,
                              uint64_t stream, uint64_t* sizes)
{
    for (uint32_t i = 0; i < n_inst; ++i) {
        uint64_t s = stream_state(seed, 200 + stream, i);
        double u = (double)(sm_next(&s) >> 11) * (1.0 / 9007199254740992.0);
        double x = lo_exp + span * u;
        /* 2^x by repeated squaring of the integer part and a series for the fraction */
        uint64_t ip = (uint64_t)x;
        double frac = x - (double)ip;
        double p = 1.0, term = 1.0, ln2f = frac * 0.69314718055994530942;
        for (int k = 1; k < 30; ++k) { term *= ln2f / k; p += term; }
        double v = p * (double)(1ull << ip);
        sizes[i] = (uint64_t)v;
        if (sizes[i] < 1) sizes[i] = 1;
    }
    return 0;
}

/* For each instance i, sizes[i] distinct vertices of [0, V) (Floyd's
 * algorithm with an open-addressing set), written consecutively to out. */
int csaw_gen_distinct_seeds(uint32_t n_inst, const uint64_t* sizes, uint32_t V, uint64_t seed,
                            uint64_t stream, uint32_t* out)
{
    uint64_t maxn = 0;
    for (uint32_t i = 0; i < n_inst; ++i) {
        if (sizes[i] > V) return 1;
        if (sizes[i] > maxn) maxn = sizes[i];
    }
    uint64_t cap = 16;
    while (cap < 2 * maxn + 2) cap <<= 1;
    uint32_t* set = (uint32_t*)malloc(sizeof(uint32_t) * cap);
    if (!set) return 2;
    uint64_t pos = 0;
    for (uint32_t i = 0; i < n_inst; ++i) {
        uint64_t n = sizes[i];
        memset(set, 0xFF, sizeof(uint32_t) * cap);
        uint64_t s = stream_state(seed, 300 + stream, i);
        /* Floyd: for j = V-n .. V-1, pick t in [0, j]; take t unless taken, else j. */
        for (uint64_t j = (uint64_t)V - n; j < V; ++j) {
            uint32_t t = (uint32_t)(sm_next(&s) % (j + 1));
            uint64_t h = mix64(t) & (cap - 1);
            int taken = 0;
            while (set[h] != 0xFFFFFFFFu) { if (set[h] == t) { taken = 1; break; } h = (h + 1) & (cap - 1); }
            uint32_t pick = taken ? (uint32_t)j : t;
            if (taken) {
                h = mix64(pick) & (cap - 1);
                while (set[h] != 0xFFFFFFFFu) h = (h + 1) & (cap - 1);
            }
            set[h] = pick;
            out[pos++] = pick;
        }
    }
    free(set);
    return 0;
}

/* ---- Multi-threaded CSR build (same result as csaw_gen_build_csr) ----
 * Degrees are counted with atomic increments, both directions of every edge
 * are scattered into their rows through atomic cursors (so the order inside a
 * row depends on thread timing), then every row is sorted and deduplicated on
 * its own: the final CSR depends only on the edge multiset.               */
typedef struct {
    int n_threads, t;
    uint64_t n_draws;
    uint32_t V;
    const uint32_t* src; const uint32_t* dst;
    uint64_t* cnt;        /* degree, then cursor */
    uint64_t* start;
    uint32_t* tmp;
    uint64_t* newlen;
    uint64_t* off;
    uint32_t* col;
    uint64_t* next_row;   /* shared dynamic row counter */
    int phase;
} csr_job;

static void sort_u32(uint32_t* a, uint64_t n, uint32_t* scratch)
{
    if (n < 64) {
        for (uint64_t i = 1; i < n; ++i) {
            uint32_t x = a[i];
            uint64_t j = i;
            while (j > 0 && a[j - 1] > x) { a[j] = a[j - 1]; --j; }
            a[j] = x;
        }
        return;
    }
    uint32_t* in = a;
    uint32_t* out = scratch;
    for (int shift = 0; shift < 32; shift += 8) {
        uint64_t c[257];
        memset(c, 0, sizeof(c));
        for (uint64_t i = 0; i < n; ++i) c[((in[i] >> shift) & 255u) + 1]++;
        for (int b = 0; b < 256; ++b) c[b + 1] += c[b];
        for (uint64_t i = 0; i < n; ++i) out[c[(in[i] >> shift) & 255u]++] = in[i];
        uint32_t* t = in; in = out; out = t;
    }
    /* four passes: the sorted data is back in a */
}

static void* csr_worker(void* pv)
{
    csr_job* J = (csr_job*)pv;
    const uint64_t n = J->n_draws;
    const uint64_t lo = n * (uint64_t)J->t / (uint64_t)J->n_threads;
    const uint64_t hi = n * (uint64_t)(J->t + 1) / (uint64_t)J->n_threads;
    if (J->phase == 0) {
        for (uint64_t e = lo; e < hi; ++e) {
            uint32_t u = J->src[e], v = J->dst[e];
            if (u == v) continue;
            __atomic_fetch_add(&J->cnt[u], 1, __ATOMIC_RELAXED);
            __atomic_fetch_add(&J->cnt[v], 1, __ATOMIC_RELAXED);
        }
    } else if (J->phase == 1) {
        for (uint64_t e = lo; e < hi; ++e) {
            uint32_t u = J->src[e], v = J->dst[e];
            if (u == v) continue;
            uint64_t p = __atomic_fetch_add(&J->cnt[u], 1, __ATOMIC_RELAXED);
            J->tmp[p] = v;
            p = __atomic_fetch_add(&J->cnt[v], 1, __ATOMIC_RELAXED);
            J->tmp[p] = u;
        }
    } else {
        uint32_t* scratch = NULL;
        uint64_t scap = 0;
        for (;;) {
            uint64_t r0 = __atomic_fetch_add(J->next_row, 4096, __ATOMIC_RELAXED);
            if (r0 >= J->V) break;
            uint64_t r1 = r0 + 4096 > J->V ? J->V : r0 + 4096;
            for (uint64_t v = r0; v < r1; ++v) {
                uint32_t* row = J->tmp + J->start[v];
                uint64_t d = J->start[v + 1] - J->start[v];
                if (J->phase == 2) {
                    if (d > scap) {
                        free(scratch);
                        scap = d * 2;
                        scratch = (uint32_t*)malloc(sizeof(uint32_t) * scap);
                        if (!scratch) { scap = 0; break; }
                    }
                    sort_u32(row, d, scratch);
                    uint64_t m = 0;
                    for (uint64_t i = 0; i < d; ++i) if (i == 0 || row[i] != row[i - 1]) row[m++] = row[i];
                    J->newlen[v] = m;
                } else {
                    memcpy(J->col + J->off[v], row, sizeof(uint32_t) * J->newlen[v]);
                }
            }
        }
        free(scratch);
    }
    return NULL;
}

static void csr_run(csr_job* jobs, int T, int phase)
{
    pthread_t th[256];
    for (int t = 0; t < T; ++t) jobs[t].phase = phase;
    for (int t = 1; t < T; ++t) pthread_create(&th[t], NULL, csr_worker, &jobs[t]);
    csr_worker(&jobs[0]);
    for (int t = 1; t < T; ++t) pthread_join(th[t], NULL);
}

int csaw_gen_build_csr_mt(uint32_t V, uint64_t n_draws, const uint32_t* src, const uint32_t* dst,
                          int n_threads, uint64_t* off, uint32_t* col, uint64_t* n_edges)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    uint64_t* cnt = (uint64_t*)calloc((uint64_t)V + 1, sizeof(uint64_t));
    uint64_t* start = (uint64_t*)malloc(sizeof(uint64_t) * ((uint64_t)V + 1));
    uint64_t* newlen = (uint64_t*)malloc(sizeof(uint64_t) * ((uint64_t)V + 1));
    if (!cnt || !start || !newlen) { free(cnt); free(start); free(newlen); return 2; }
    csr_job jobs[256];
    uint64_t next_row = 0;
    for (int t = 0; t < n_threads; ++t) {
        csr_job j = { n_threads, t, n_draws, V, src, dst, cnt, start, NULL, newlen, off, col, &next_row, 0 };
        jobs[t] = j;
    }
    csr_run(jobs, n_threads, 0);
    uint64_t run = 0;
    for (uint32_t v = 0; v < V; ++v) { start[v] = run; run += cnt[v]; cnt[v] = start[v]; }
    start[V] = run;
    uint32_t* tmp = (uint32_t*)malloc(sizeof(uint32_t) * (run ? run : 1));
    if (!tmp) { free(cnt); free(start); free(newlen); return 2; }
    for (int t = 0; t < n_threads; ++t) jobs[t].tmp = tmp;
    csr_run(jobs, n_threads, 1);
    next_row = 0;
    csr_run(jobs, n_threads, 2);
    uint64_t w = 0;
    for (uint32_t v = 0; v < V; ++v) { off[v] = w; w += newlen[v]; }
    off[V] = w;
    next_row = 0;
    csr_run(jobs, n_threads, 3);
    *n_edges = w;
    free(tmp); free(cnt); free(start); free(newlen);
    return 0;
}

/* Weights of rows [r0, r1) (thread body of csaw_gen_weights_mt). */
typedef struct { uint32_t r0, r1; const uint64_t* off; const uint32_t* col; uint32_t wmax; uint64_t seed; uint32_t* w; } wjob;

static void* weights_worker(void* pv)
{
    wjob* J = (wjob*)pv;
    for (uint32_t u = J->r0; u < J->r1; ++u) {
        for (uint64_t p = J->off[u]; p < J->off[u + 1]; ++p) {
            uint32_t v = J->col[p];
            uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
            uint64_t h = mix64(stream_state(J->seed, 2, (lo << 32) | hi));
            J->w[p] = 1u + (uint32_t)(h % J->wmax);
        }
    }
    return NULL;
}

int csaw_gen_weights_mt(uint32_t V, const uint64_t* off, const uint32_t* col, uint32_t wmax,
                        uint64_t seed, int n_threads, uint32_t* w)
{
    if (wmax == 0) return 1;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    wjob jobs[256];
    pthread_t th[256];
    /* split by edges so that hub rows do not serialise one thread */
    uint64_t E = off[V];
    uint32_t r = 0;
    for (int t = 0; t < n_threads; ++t) {
        uint64_t target = E * (uint64_t)(t + 1) / (uint64_t)n_threads;
        uint32_t r1 = r;
        while (r1 < V && off[r1] < target) ++r1;
        if (t == n_threads - 1) r1 = V;
        wjob j = { r, r1, off, col, wmax, seed, w };
        jobs[t] = j;
        r = r1;
    }
    for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, weights_worker, &jobs[t]);
    weights_worker(&jobs[0]);
    for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
    return 0;
}
