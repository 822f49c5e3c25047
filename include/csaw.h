/*
 * csaw.h -- C ABI of libcsaw: biased neighbour selection for graph sampling
 * and random walks on one GB300 (sm_103a), after C-SAW (Pandey, Li, Hoisie,
 * Li, Liu, "C-SAW: A Framework for Graph Sampling and Random Walk on GPUs",
 * SC20).
 *
 * What every call computes (the paper's method, in exact integer form):
 *   - EdgeBias (Sec. III-C, Eq. 3): each neighbour u of the vertex v being
 *     expanded gets a uint32 bias b(u): 1 (uniform), the edge weight w(v,u),
 *     the degree of u, or node2vec's second-order bias (Sec. II-A):
 *     w(v,u) * m0 if u is the walk's previous vertex t, w(v,u) * m1 if u is a
 *     neighbour of t, w(v,u) * m2 otherwise; the first step of a walk uses w.
 *   - Inverse transform sampling (Sec. II-B, Theorem 1, Eq. 1): S[i] is the
 *     inclusive uint64 prefix sum of the biases in CSR order, T = S[d-1];
 *     neighbour i owns [S[i-1], S[i]).  Attempt a draws a 64-bit r from
 *     Philox4x32-10 (key = {lo32(seed), hi32(seed)}, counter = {a, vertex,
 *     layer or step, instance}, r = out1 << 32 | out0), maps it to
 *     x = floor(r * T / 2^64) and picks the i whose interval holds x.
 *   - Selection without replacement (Sec. IV-B): the first k distinct picks
 *     in attempt order (repeated sampling).  After CSAW_ATTEMPT_CAP attempts
 *     the remaining picks use updated sampling (the draw is scaled to the
 *     total of the unpicked biases and searched among them), which ends in at
 *     most k more attempts and leaves each pick's conditional law unchanged.
 *     A vertex with at most k neighbours of positive bias takes all of them,
 *     in CSR order, with no draws.
 *   - Layered sampling (Sec. III-B, Fig. 2(b); Update, Eq. 4): each frontier
 *     vertex selects fanout[l] neighbours; every pick is a sampled edge; the
 *     next frontier is the set of picked vertices not yet visited by that
 *     instance (traversal sampling never revisits a vertex, Sec. II-A).
 *   - Random walk (Sec. II-A): one pick per step, with replacement.
 * Results are bit-exact functions of (graph, arguments, rng_seed): they do
 * not depend on batching, launch shape or what else runs on the GPU.
 *
 * Conventions
 *   - All calls return csaw_status; none aborts.  On error,
 *     csaw_last_error() returns a message for the calling thread.
 *   - mem_kind says where the caller's array arguments live:
 *     CSAW_MEM_DEVICE: device pointers; the call is asynchronous on `stream`
 *     (a cudaStream_t, NULL = legacy default stream).
 *     CSAW_MEM_HOST: host pointers; the call copies inputs to the device,
 *     runs, copies outputs back and returns when they are in host memory.
 *   - Invalid vertex / padding value: CSAW_NONE.
 *   - The library owns the objects it returns until the matching destroy or
 *     free call; the caller keeps ownership of every buffer it passes.
 */
#ifndef CSAW_H
#define CSAW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CSAW_OK = 0,
    CSAW_ERR_INVALID = 1,   /* malformed argument or graph */
    CSAW_ERR_NOMEM = 2,     /* device or host allocation failed, or over budget */
    CSAW_ERR_CUDA = 3,      /* a CUDA runtime call failed */
    CSAW_ERR_OVERFLOW = 4,  /* a bias does not fit in 32 bits */
    CSAW_ERR_TIMEOUT = 5,   /* csaw_poll: not finished within the timeout */
    CSAW_ERR_ABORTED = 6,   /* request cancelled or server shut down */
    CSAW_ERR_NOT_FOUND = 7  /* unknown ticket */
} csaw_status;

typedef enum {
    CSAW_BIAS_UNIFORM = 0,
    CSAW_BIAS_EDGE_WEIGHT = 1,
    CSAW_BIAS_NEIGHBOR_DEGREE = 2,
    CSAW_BIAS_NODE2VEC = 3
} csaw_bias_kind;

/* Bias of a call.  n2v_mult = (m0, m1, m2) for CSAW_BIAS_NODE2VEC:
 * multiplier when the neighbour is the previous vertex, when it is adjacent
 * to the previous vertex, otherwise.  node2vec's 1/p, 1, 1/q scaled to
 * integers; p = 2, q = 0.5 gives (1, 2, 4).  Ignored for the other kinds. */
typedef struct {
    int32_t kind;
    uint32_t n2v_mult[3];
} csaw_bias;

enum { CSAW_MEM_HOST = 0, CSAW_MEM_DEVICE = 1 };

#define CSAW_NONE 0xFFFFFFFFu
#define CSAW_FANOUT_ALL 0xFFFFFFFFu
#define CSAW_ATTEMPT_CAP 1024u
#define CSAW_MAX_DEPTH 16u

typedef struct csaw_graph csaw_graph;
typedef struct csaw_sample_result csaw_sample_result;
typedef struct csaw_sample_plan csaw_sample_plan;
typedef struct csaw_server csaw_server;

/* ---------------------------------------------------------------- graph */

/* Build a device-resident graph from CSR.  The graph is the input of every
 * selection (Sec. II-A; all neighbours of a vertex must be present to form
 * its biases, Sec. I and V-A).
 *   row_offsets  uint64[n_vertices + 1], row_offsets[0] = 0,
 *                row_offsets[n_vertices] = n_edges, non-decreasing
 *   cols         uint32[n_edges]: neighbours of v at
 *                cols[row_offsets[v] .. row_offsets[v+1]), strictly ascending
 *                (sorted, no duplicates; node2vec's membership test relies on
 *                it), every entry < n_vertices
 *   weights      uint32[n_edges] edge weights, or NULL for all ones
 *   mem_kind     where the three arrays live (host or device)
 * The arrays are copied; the caller may free them when the call returns (for
 * device inputs, once `stream` has reached this call).  Validation runs on
 * the device and the call waits for it.  Errors: CSAW_ERR_INVALID (any rule
 * above broken, or a row longer than 2^32 - 1), CSAW_ERR_NOMEM, CSAW_ERR_CUDA. */
csaw_status csaw_graph_create(const uint64_t* row_offsets, uint32_t n_vertices,
                              const uint32_t* cols, const uint32_t* weights, uint64_t n_edges,
                              int mem_kind, void* stream, csaw_graph** out);

/* Release the graph's device memory.  Work still queued on it must have
 * finished.  NULL is accepted. */
csaw_status csaw_graph_destroy(csaw_graph* g);

/* Sizes and derived facts of a graph (host values). */
typedef struct {
    uint32_t n_vertices;
    uint64_t n_edges;
    uint32_t max_degree;
    uint32_t max_weight;
    uint64_t device_bytes;   /* device memory the graph holds */
} csaw_graph_info;

csaw_status csaw_graph_get_info(const csaw_graph* g, csaw_graph_info* out);

/* Build the cached cumulative bias array of a static bias kind
 * (CSAW_BIAS_EDGE_WEIGHT or CSAW_BIAS_NEIGHBOR_DEGREE): per edge e of row v,
 * the inclusive uint64 prefix sum of the row's biases up to e -- the CTPS of
 * Sec. II-B computed once instead of at every selection -- and a summary of
 * every 8th sum (9 bytes per edge in all).
 * Afterwards csaw_walk, csaw_sample and plans created later use it for that
 * kind: a walk step or a draw is a binary search (O(log d)) instead of a pass
 * over the row.  Picks are identical (same prefix sums, same draws).  Graphs
 * where some bias of the kind is zero keep the streaming path.  Waits on
 * `stream`.  Errors: CSAW_ERR_INVALID (dynamic or unweighted kind),
 * CSAW_ERR_NOMEM, CSAW_ERR_CUDA. */
csaw_status csaw_graph_build_cdf(csaw_graph* g, int32_t bias_kind, void* stream);

/* Release a cached array.  Plans created while it existed must be destroyed
 * first; no call may be running on the graph. */
csaw_status csaw_graph_drop_cdf(csaw_graph* g, int32_t bias_kind);

/* Device memory through the caller's allocator (e.g. PyTorch's caching
 * allocator, so that a framework's memory accounting covers this library).
 * After this call, every device allocation that later calls on g make goes
 * through alloc: the temporaries of csaw_walk, csaw_walk_ex, csaw_sample,
 * csaw_sample_ex, csaw_layer_sample, csaw_mdrw and csaw_autotune_select, the
 * device arrays of their results, the buffers of plans created afterwards,
 * cached arrays built afterwards and the request buffers of servers on g.
 *   alloc(bytes, stream, ctx)  returns device memory of at least `bytes`
 *               bytes on g's device, 256-byte aligned, first used on
 *               `stream` (a cudaStream_t; NULL = legacy default stream), or
 *               NULL on failure (the call then returns CSAW_ERR_NOMEM)
 *   free(ptr, stream, ctx)     releases ptr; work already queued on `stream`
 *               may still use it (stream-ordered, like cudaFreeAsync)
 * Memory is always released through the pair that allocated it.  NULL
 * alloc and free restore the library's own stream-ordered pool.  The pair may
 * be called from the library's threads (the request server's slots).  The
 * graph's own CSR arrays are not affected.  Not thread-safe against running
 * calls on g.  Errors: CSAW_ERR_INVALID (only one of alloc and free given). */
typedef void* (*csaw_alloc_fn)(uint64_t bytes, void* stream, void* ctx);
typedef void (*csaw_free_fn)(void* ptr, void* stream, void* ctx);
csaw_status csaw_graph_set_allocator(csaw_graph* g, csaw_alloc_fn alloc, csaw_free_fn free, void* ctx);

/* ---------------------------------------------------------------- walks */

/* Biased random walks (Sec. II-A; static bias: edge weight or neighbour
 * degree; dynamic bias: node2vec), one pick per step with replacement.
 *   starts    uint32[n_walkers] start vertices (each < n_vertices)
 *   length    steps per walker
 *   path      uint32[n_walkers][length + 1] row-major output;
 *             path[w][0] = starts[w]; path[w][s+1] is the vertex after step s.
 *             A walker at a vertex whose biases are all zero (or with no
 *             neighbour) stops there; the rest of its row is CSAW_NONE.
 * The draw of walker w at step s uses attempt 0, vertex = its current vertex,
 * layer = s, instance = w.  Errors: CSAW_ERR_INVALID (bad bias kind, a start
 * >= n_vertices for host inputs, n_walkers >= 2^32), CSAW_ERR_OVERFLOW
 * (node2vec: max weight * max multiplier >= 2^32), CSAW_ERR_NOMEM,
 * CSAW_ERR_CUDA.  With device inputs an out-of-range start is caught on the
 * device: its row is filled with CSAW_NONE. */
csaw_status csaw_walk(csaw_graph* g, const uint32_t* starts, uint64_t n_walkers, uint32_t length,
                      const csaw_bias* bias, uint64_t rng_seed, uint32_t* path, int mem_kind,
                      void* stream);

/* Random walk with restart or with jump (Sec. II-A; the Update of Eq. 4
 * returning a vertex other than the sampled neighbour): csaw_walk with
 * options (NULL = plain walk).  With teleport = CSAW_TELEPORT_RESTART or
 * _JUMP, every step of walker w at vertex v first draws attempt 1 (vertex v,
 * layer s, instance w); if the draw's upper 32 bits are below teleport_q32
 * (a per-step probability of teleport_q32 / 2^32) the walker goes to its
 * start vertex (restart) or to vertex floor(r2 * n_vertices / 2^64), r2 the
 * draw of attempt 2 (jump), instead of to a neighbour.  A walker at a vertex
 * with no neighbour of positive bias teleports the same way instead of
 * stopping.  After a teleport a node2vec walk has no previous vertex (its
 * next step uses the weights alone).  Teleporting walks always stream the
 * biases (a cached cumulative array is not used).
 * build_cdf = 1 (no teleport, static bias whose biases are all positive, no
 * cached array of the kind on g): the call first builds the cumulative array
 * of the kind over the whole graph, as csaw_graph_build_cdf does, into a
 * temporary of 9 bytes per edge (stream-ordered, freed by the call), and
 * every step is then a search of it instead of a pass over the row: the
 * same paths, with the array's construction inside the call.  Ignored
 * otherwise.  For edge weights the temporary holds only the summaries of the
 * prefix sums (every 8th and 64th) and per-vertex records {start, end,
 * total}, about 1.14 bytes per edge + 32 per vertex, and a step forms its
 * 8-edge group's sums from the weights; for neighbour degree it holds the
 * whole array (9 bytes per edge + 32 per vertex).
 * phase_ms (not NULL): the call records CUDA events on `stream` around its
 * phases, waits for the stream, and stores the device time of the array's
 * construction in phase_ms[0] (0 when nothing is built) and of the walk
 * kernels in phase_ms[1].  Errors: those of csaw_walk, and CSAW_ERR_INVALID
 * for an unknown teleport mode. */
#define CSAW_TELEPORT_NONE 0
#define CSAW_TELEPORT_RESTART 1
#define CSAW_TELEPORT_JUMP 2

typedef struct {
    int32_t teleport;        /* CSAW_TELEPORT_* */
    uint32_t teleport_q32;   /* teleport probability per step, in units of 2^-32 */
    uint32_t build_cdf;      /* 1: see below */
    float* phase_ms;         /* NULL, or float[2]: see below */
} csaw_walk_opts;

csaw_status csaw_walk_ex(csaw_graph* g, const uint32_t* starts, uint64_t n_walkers, uint32_t length,
                         const csaw_bias* bias, uint64_t rng_seed, uint32_t* path, int mem_kind,
                         void* stream, const csaw_walk_opts* opts);

/* Random walks over a graph kept in host memory (out-of-memory sampling,
 * Sec. V-A: graph partitions and workload-aware partition scheduling).
 *   row_offsets, cols, weights  a host CSR as for csaw_graph_create (weights
 *                 NULL = all ones); only read, never copied whole
 *   device_budget_bytes  the device memory for one partition slot: vertex
 *                 ranges are cut so that a range's offsets and columns (and for
 *                 edge weight its weights and 8-byte prefix sums) fit it
 *   starts, path  host arrays as for csaw_walk with host memory
 *   stats         if not NULL: partitions, partition loads, bytes loaded
 * Each round loads the partition that holds the most active walkers and
 * advances every walker in it until it leaves the partition, finishes or
 * meets a dead end.  Draws and prefix sums are those of csaw_walk, so the
 * paths equal csaw_walk's for the same graph, starts and seed.  Bias: uniform
 * or edge weight.  Walker state and the path use device memory beyond the
 * budget.  Synchronous on `stream`.  Errors: CSAW_ERR_INVALID (bad CSR
 * offsets or columns, bias kind or start), CSAW_ERR_NOMEM (a row larger than the budget,
 * or device allocation), CSAW_ERR_CUDA. */
typedef struct {
    uint32_t partitions;     /* vertex ranges the graph was cut into */
    uint64_t loads;          /* partition uploads (scheduling rounds) */
    uint64_t bytes_loaded;   /* host-to-device bytes of those uploads */
    uint64_t reuses;         /* rounds whose partition was still in a slot (no upload) */
    uint64_t pinned_bytes;   /* host bytes page-locked for the call (opts->pin_host) */
    uint32_t direct;         /* 1: the walk read the host arrays in place (opts->direct) */
} csaw_oom_stats;

/* Options of the out-of-memory calls (NULL = defaults). */
typedef struct {
    uint32_t slots;          /* device partition slots, each of device_budget_bytes
                                (0 = the call's default; at most 8) */
    uint32_t pin_host;       /* 1: page-lock the host columns and weights for the
                                duration of the call (cudaHostRegister), so that
                                partition copies run behind the selection; a
                                refused registration falls back to pageable copies */
    uint32_t direct;         /* walks, 1: read the host CSR in place instead of
                                copying partitions (see csaw_walk_oom_ex) */
} csaw_oom_opts;

/* The partitions csaw_walk_oom cuts a host CSR into for a device budget
 * (host only; no device work).  Vertex ranges [bounds[q], bounds[q+1]) are
 * taken greedily in vertex order, each as long as its offsets (8 bytes per
 * row + 8) and, per edge, its column (4) and, when weighted, its weight (4)
 * and prefix sum (8) fit device_budget_bytes.
 *   bounds      NULL to ask for the count only, else bounds_cap entries
 *               receiving the n_partitions + 1 range starts (the last is
 *               n_vertices)
 * Errors: CSAW_ERR_INVALID (NULL pointers, no vertices, decreasing offsets,
 * bounds too short), CSAW_ERR_NOMEM (a row larger than the budget). */
csaw_status csaw_oom_plan(const uint64_t* row_offsets, uint32_t n_vertices, int weighted,
                          uint64_t device_budget_bytes, uint32_t* bounds, uint32_t bounds_cap,
                          uint32_t* n_partitions);

csaw_status csaw_walk_oom(const uint64_t* row_offsets, const uint32_t* cols, const uint32_t* weights,
                          uint32_t n_vertices, uint64_t n_edges, uint64_t device_budget_bytes,
                          const uint32_t* starts, uint64_t n_walkers, uint32_t length,
                          const csaw_bias* bias, uint64_t rng_seed, uint32_t* path,
                          csaw_oom_stats* stats, void* stream);

/* csaw_walk_oom with options (NULL: 2 slots, no pinning).  With two or more
 * slots, each round also loads the partition with the second most active
 * walkers into another slot, on a stream of its own, while the round runs
 * (Sec. V-B); a round whose partition is still in a slot loads nothing
 * (stats->reuses).  Paths are those of csaw_walk_oom and csaw_walk.
 * opts->direct = 1, on a device that reads pageable host memory coherently
 * (cudaDevAttrPageableMemoryAccess, e.g. a Grace-attached GPU), with cols
 * and weights 16-byte aligned: no partition is copied.  The device builds,
 * from the host weights read in place, the summaries of their row prefix
 * sums (every 8th and 64th) and per-vertex records {start, end, total}
 * (about 1.14 bytes per edge + 32 per vertex, which must fit
 * slots x device_budget_bytes), and each step reads one record, bisects the
 * summaries and reads one 32-byte group of weights and the picked column
 * from host memory.  Columns are checked on the device before the walk.
 * stats->direct reports the mode; otherwise the call partitions as above. */
csaw_status csaw_walk_oom_ex(const uint64_t* row_offsets, const uint32_t* cols, const uint32_t* weights,
                             uint32_t n_vertices, uint64_t n_edges, uint64_t device_budget_bytes,
                             const uint32_t* starts, uint64_t n_walkers, uint32_t length,
                             const csaw_bias* bias, uint64_t rng_seed, uint32_t* path,
                             csaw_oom_stats* stats, void* stream, const csaw_oom_opts* opts);

/* Layered sampling (as csaw_sample) over a graph kept in host memory
 * (out-of-memory sampling, Sec. V-A; partition transfers overlapped with
 * sampling, Sec. V-B).
 *   row_offsets, cols, weights  a host CSR as for csaw_graph_create (weights
 *                 NULL = all ones); read, never copied whole
 *   device_budget_bytes  the device memory of one partition slot: vertex
 *                 ranges are cut so that a range's columns, weights and the
 *                 prefix sums of its hub rows fit it (16 bytes per edge; see
 *                 csaw_oom_plan with weighted = 1)
 *   seeds, inst_offsets, n_instances, depth, fanout, bias, rng_seed
 *                 host arrays and arguments as for csaw_sample (bias: uniform,
 *                 edge weight or neighbour degree)
 *   opts          slots (default 2) and host pinning; stats as csaw_walk_oom
 * The row offsets and the degrees stay on the device (16 bytes per vertex
 * beyond the budget), as do the frontiers and the sampled edges.  Per layer,
 * the partitions that hold frontier vertices are taken in the order of how
 * many frontier entries they hold (workload-aware scheduling, Sec. V-A); the
 * next partition is copied into another slot while the current one is
 * sampled.  Draws, prefix sums and the result's layout are those of
 * csaw_sample, so the result is identical to csaw_sample's on the same graph
 * and arguments.  Every bias must be positive (weights >= 1; for neighbour
 * degree, no edge into a vertex without neighbours).  Returns when the result
 * is complete; read it with csaw_sample_get_view / csaw_sample_copy_edges and
 * release it with csaw_result_free.  Errors: CSAW_ERR_INVALID (bad CSR, bias,
 * seeds or offsets, a zero bias), CSAW_ERR_NOMEM (a row larger than the
 * budget, or device allocation), CSAW_ERR_CUDA. */
csaw_status csaw_sample_oom(const uint64_t* row_offsets, const uint32_t* cols, const uint32_t* weights,
                            uint32_t n_vertices, uint64_t n_edges, uint64_t device_budget_bytes,
                            const uint32_t* seeds, const uint64_t* inst_offsets, uint32_t n_instances,
                            uint32_t depth, const uint32_t* fanout, const csaw_bias* bias,
                            uint64_t rng_seed, const csaw_oom_opts* opts, csaw_oom_stats* stats,
                            void* stream, csaw_sample_result** out);

/* Multi-dimensional random walk, or frontier sampling (Sec. II-A), as the
 * API of Sec. III-C expresses it in the case study of Sec. III-D (Figs. 3-4):
 * each instance keeps a pool of pool_size vertices, and every step
 *   1. selects one pool slot with probability proportional to its vertex's
 *      degree (VertexBias, Eq. 2), by inverse transform sampling over the
 *      pool's prefix sums in slot order;
 *   2. selects one neighbour u of that vertex v uniformly (EdgeBias = 1);
 *   3. puts u in v's slot (Update, Eq. 4) and emits the sampled edge (v, u).
 *   pools      uint32[n_instances][pool_size] initial pools, row-major; an
 *              entry >= n_vertices (e.g. CSAW_NONE) is an empty slot (bias 0)
 *   pool_size  1 .. CSAW_MDRW_MAX_POOL
 *   steps      steps per instance
 *   src, dst   uint32[n_instances][steps] row-major outputs: the edge of step s
 *              of instance i is (src[i][s], dst[i][s]).  An instance whose
 *              pool degrees sum to zero stops; the rest of its rows are
 *              CSAW_NONE.
 * The pool draw of instance i at step s uses attempt 0, vertex = CSAW_NONE,
 * layer = s, instance = i; the neighbour draw uses vertex = v (the counter of
 * a walk step at v), so a one-slot pool walks exactly like csaw_walk with
 * uniform bias.  Edge weights are not used.  With host memory the call
 * copies in, runs and copies out before it returns; with device memory it is
 * queued on `stream`.  The pools buffer is only read.  Errors:
 * CSAW_ERR_INVALID (NULL graph or buffers, pool_size out of range,
 * n_instances >= 2^32), CSAW_ERR_NOMEM, CSAW_ERR_CUDA. */
#define CSAW_MDRW_MAX_POOL 65536u

csaw_status csaw_mdrw(csaw_graph* g, const uint32_t* pools, uint64_t n_instances, uint32_t pool_size,
                      uint32_t steps, uint64_t rng_seed, uint32_t* src, uint32_t* dst, int mem_kind,
                      void* stream);

/* ---------------------------------------------------------------- sampling */

/* Layered biased neighbour sampling over many independent instances
 * (Sec. III-B, Fig. 2(b); instances, Sec. IV-A; batched multi-instance
 * sampling, Sec. V-B).
 *   seeds         uint32[inst_offsets[n_instances]]: instance i's seeds are
 *                 seeds[inst_offsets[i] .. inst_offsets[i+1]); duplicates are
 *                 merged
 *   inst_offsets  uint64[n_instances + 1], non-decreasing, starting at 0
 *   depth         number of layers (1 .. CSAW_MAX_DEPTH)
 *   fanout        uint32[depth] HOST array: picks per frontier vertex at each
 *                 layer, or CSAW_FANOUT_ALL
 *   bias          UNIFORM, EDGE_WEIGHT or NEIGHBOR_DEGREE (NODE2VEC needs a
 *                 walk's previous vertex and is rejected)
 * The draws of frontier vertex v of instance i at layer l use vertex = v,
 * layer = l, instance = i.  Output edges are grouped by layer, then instance,
 * then source vertex ascending; each vertex's picks are in pick order.
 * seeds/inst_offsets live in mem_kind memory.  The call runs the layers on
 * `stream` and waits on it once per layer (to size the next layer's buffers),
 * so it returns with the result complete.  The result lives on the device;
 * read it with csaw_sample_get_view or copy it with csaw_sample_copy_edges,
 * release it with csaw_result_free.
 * Errors: CSAW_ERR_INVALID, CSAW_ERR_NOMEM, CSAW_ERR_CUDA. */
csaw_status csaw_sample(csaw_graph* g, const uint32_t* seeds, const uint64_t* inst_offsets,
                        uint32_t n_instances, uint32_t depth, const uint32_t* fanout,
                        const csaw_bias* bias, uint64_t rng_seed, int mem_kind, void* stream,
                        csaw_sample_result** out);

/* Selection options.  attempt_cap: repeated-sampling attempts before the
 * remaining picks switch to updated sampling (Sec. IV-B, Fig. 5(b)).  The
 * default CSAW_ATTEMPT_CAP keeps the first k distinct hits of the draw
 * sequence; 0 takes every pick by updated sampling -- one draw per pick, no
 * rejection loop, the exact form of the paper's bipartite region search
 * (Sec. IV-B, Theorem 2) generalised to any number of earlier picks.  Both
 * give every pick the law b_j / (total of the unpicked biases); they use the
 * draws differently, so their outputs differ. */
typedef struct {
    uint32_t attempt_cap;
} csaw_sample_opts;

/* csaw_sample with options (NULL = defaults). */
csaw_status csaw_sample_ex(csaw_graph* g, const uint32_t* seeds, const uint64_t* inst_offsets,
                           uint32_t n_instances, uint32_t depth, const uint32_t* fanout,
                           const csaw_bias* bias, uint64_t rng_seed, int mem_kind, void* stream,
                           const csaw_sample_opts* opts, csaw_sample_result** out);

/* Layer sampling (Sec. II-A: a constant number of neighbours for all the
 * vertices of the frontier together), written as Fig. 2(b) with the whole
 * frontier as the current frontier: per instance and layer l, the
 * NeighborPool is every edge (v, u) of the instance's frontier, ascending v
 * and then CSR order, with its EdgeBias (uniform, edge weight or neighbour
 * degree); Select picks layer_size[l] entries without replacement by the rule
 * of csaw_sample (first distinct hits of repeated sampling, updated sampling
 * after opts->attempt_cap attempts, all positive entries when there are at
 * most layer_size[l]), with the draw of attempt a keyed {a, CSAW_NONE, l,
 * instance}; Update is that of csaw_sample.  Arguments, result layout
 * (edges grouped by layer, then instance, in pick order), ownership and
 * errors are those of csaw_sample_ex, with layer_size in place of fanout
 * (CSAW_FANOUT_ALL takes the whole pool).  The pool of one instance must
 * hold fewer than 2^32 edges. */
csaw_status csaw_layer_sample(csaw_graph* g, const uint32_t* seeds, const uint64_t* inst_offsets,
                              uint32_t n_instances, uint32_t depth, const uint32_t* layer_size,
                              const csaw_bias* bias, uint64_t rng_seed, int mem_kind, void* stream,
                              const csaw_sample_opts* opts, csaw_sample_result** out);

typedef struct {
    uint32_t depth;
    uint32_t n_instances;
    uint64_t n_edges;
    /* host, depth*n_instances + 1 entries: edges of (layer l, instance i) are
     * [edge_offsets[l*n_instances + i], edge_offsets[l*n_instances + i + 1])
     * in one numbering that runs over all layers */
    const uint64_t* edge_offsets;
    /* host, depth*n_instances entries: frontier size of (layer l, instance i)
     * (layer 0 = the instance's distinct seeds) */
    const uint64_t* frontier_sizes;
    /* host arrays of `depth` device pointers.  Layer l's edges are
     * src[l][j], dst[l][j] for j < edge_offsets[(l+1)*n_instances] -
     * edge_offsets[l*n_instances], in the order described above. */
    const uint32_t* const* src;
    const uint32_t* const* dst;
} csaw_sample_view;

/* Fill *view.  csaw_sample returns once its result is complete, so this does
 * not wait.  The pointers stay valid until csaw_result_free. */
csaw_status csaw_sample_get_view(csaw_sample_result* r, csaw_sample_view* view);

/* Copy the sampled edges of all layers, concatenated in layer order, to host
 * arrays of n_edges entries each.  Synchronous. */
csaw_status csaw_sample_copy_edges(csaw_sample_result* r, uint32_t* src, uint32_t* dst);

/* Release a result returned by this library (a csaw_sample_result or a
 * csaw_result).  NULL is accepted. */
void csaw_result_free(void* result);

/* ---------------------------------------------------------------- batched plans */

/* A sample plan: csaw_sample's whole multi-instance, multi-layer pipeline
 * (the batched multi-instance sampling of Sec. V-B, one frontier queue of
 * (vertex, instance) entries across all instances) for a fixed instance count,
 * seed budget, depth, fanout and bias, with every device buffer allocated
 * once at its upper bound and the pipeline captured into one CUDA graph.
 * Each run copies a new batch of seeds in and launches the graph: no host
 * waits, no allocation.  Results are identical to csaw_sample on the same
 * arguments.
 * Upper bounds: layer l emits at most |F_l| * min(fanout[l], max degree)
 * edges; |F_0| <= max_seeds and |F_{l+1}| <= min(edges of layer l,
 * n_instances * n_vertices).  A plan whose non-last layer may produce 2^32 or
 * more edges is rejected (CSAW_ERR_INVALID).
 * Errors: CSAW_ERR_INVALID, CSAW_ERR_NOMEM, CSAW_ERR_CUDA. */
csaw_status csaw_sample_plan_create(csaw_graph* g, uint32_t n_instances, uint64_t max_seeds,
                                    uint32_t depth, const uint32_t* fanout, const csaw_bias* bias,
                                    csaw_sample_plan** out);

/* csaw_sample_plan_create with selection options (NULL = defaults). */
csaw_status csaw_sample_plan_create_ex(csaw_graph* g, uint32_t n_instances, uint64_t max_seeds,
                                       uint32_t depth, const uint32_t* fanout, const csaw_bias* bias,
                                       const csaw_sample_opts* opts, csaw_sample_plan** out);

/* Run the plan on n_seeds seeds (<= max_seeds) split by inst_offsets
 * (n_instances + 1 entries, inst_offsets[n_instances] = n_seeds), in host or
 * device memory per mem_kind; asynchronous on `stream`.  Host inputs are
 * validated on the host; device inputs are checked on the device and a bad
 * seed or offset is reported by the next csaw_sample_plan_get_view. */
csaw_status csaw_sample_plan_run(csaw_sample_plan* p, const uint32_t* seeds, uint64_t n_seeds,
                                 const uint64_t* inst_offsets, uint64_t rng_seed, int mem_kind,
                                 void* stream);

/* Wait for the last run and describe its result (same layout as
 * csaw_sample_view; the device arrays belong to the plan and are overwritten
 * by its next run). */
csaw_status csaw_sample_plan_get_view(csaw_sample_plan* p, csaw_sample_view* view);

/* Wait for the last run and copy its edges (all layers, concatenated) to
 * host arrays of n_edges entries. */
csaw_status csaw_sample_plan_copy_edges(csaw_sample_plan* p, uint32_t* src, uint32_t* dst);

/* Capacity-based device bytes of the plan's buffers and its selection launch
 * shape (any pointer may be NULL). */
csaw_status csaw_sample_plan_get_info(const csaw_sample_plan* p, uint64_t* device_bytes,
                                      uint32_t* theta_warp, uint32_t* select_blocks);

csaw_status csaw_sample_plan_destroy(csaw_sample_plan* p);

/* ---------------------------------------------------------------- tuning */

/* Launch shape of the selection kernel for one bias kind on one graph.
 * theta_warp: frontier vertices of degree <= theta_warp (at most 256) are
 * handled by one warp, larger ones by a CTA (the paper's warp-centric
 * selection, Sec. IV-A, with a CTA path added for long neighbour lists);
 * blocks_per_sm: resident CTAs per SM of the persistent grid (0 = as many as
 * fit).  The shape changes speed only, never results. */
typedef struct {
    uint32_t theta_warp;
    uint32_t blocks_per_sm;
} csaw_select_tuning;

csaw_status csaw_set_select_tuning(csaw_graph* g, int32_t bias_kind, const csaw_select_tuning* t);
csaw_status csaw_get_select_tuning(const csaw_graph* g, int32_t bias_kind, csaw_select_tuning* t);

/* Autotuner: times csaw_sample on the given (host) workload for every
 * theta_warp in {32, 64, 128, 256} and every blocks_per_sm up to the
 * occupancy limit, keeps the fastest on the graph and returns it in *best. */
csaw_status csaw_autotune_select(csaw_graph* g, const uint32_t* seeds, const uint64_t* inst_offsets,
                                 uint32_t n_instances, uint32_t depth, const uint32_t* fanout,
                                 const csaw_bias* bias, uint64_t rng_seed, void* stream,
                                 csaw_select_tuning* best);

/* ---------------------------------------------------------------- serving */

/* A request server over one resident graph.  Requests (sampling or walks, in
 * any mix of sizes) are admitted in arrival order while their device-memory
 * estimate fits budget_bytes and one of `slots` slots is free; every slot has
 * its own CUDA stream, so admitted requests run concurrently and their work
 * overlaps on the GPU.  A request that arrives while others run is admitted as
 * soon as a slot and enough budget are free.  Continuous batching: a slot that
 * frees up takes the oldest waiting request and, with it, up to max_batch - 1
 * other waiting requests of the same kind and bias that fit the budget; their
 * instances (sampling) or walkers (walks) run as one multi-instance launch
 * (the batched multi-instance sampling of Sec. V-B) and finish together.
 * Batches that can produce more than 2^18 sampled edges run on low-priority
 * streams and smaller ones on high-priority streams, so that a small batch's
 * blocks are scheduled ahead of the waiting blocks of large ones; a batch
 * holds only its own stream while it runs (its device memory is freed
 * stream-ordered, without waiting for other slots' kernels).
 * Each request's draws depend only on its own arguments and seed, so its
 * result is bit-for-bit the one that csaw_sample / csaw_walk return for it
 * alone.  The paper has no serving layer: this runs its selection (Sec.
 * III-IV) for a stream of independent instances (Sec. IV-A). */
typedef struct {
    uint64_t budget_bytes;   /* device bytes that admitted requests may hold at once */
    uint32_t slots;          /* concurrent batches (1 .. 256) */
    uint32_t max_batch;      /* requests per batch (0 = 32; 1 = no batching) */
} csaw_server_opts;

enum { CSAW_REQ_SAMPLE = 0, CSAW_REQ_WALK = 1 };

/* A request; all arrays are host memory and are copied by csaw_submit. */
typedef struct {
    int32_t kind;                  /* CSAW_REQ_SAMPLE or CSAW_REQ_WALK */
    csaw_bias bias;
    uint64_t rng_seed;
    /* sampling (as csaw_sample) */
    const uint32_t* seeds;
    const uint64_t* inst_offsets;
    uint32_t n_instances;
    uint32_t depth;
    const uint32_t* fanout;
    /* walks (as csaw_walk) */
    const uint32_t* starts;
    uint64_t n_walkers;
    uint32_t length;
} csaw_request;

/* A finished request: host arrays owned by the result (csaw_result_free). */
typedef struct {
    uint32_t tag;                  /* set by the library */
    int32_t kind;
    csaw_status status;            /* outcome of the request */
    /* sampling: layout of csaw_sample_view, edges of all layers concatenated */
    uint32_t depth;
    uint32_t n_instances;
    uint64_t n_edges;
    uint64_t* edge_offsets;
    uint64_t* frontier_sizes;
    uint32_t* src;
    uint32_t* dst;
    /* walks: path [n_walkers][length + 1] as csaw_walk */
    uint64_t n_walkers;
    uint32_t length;
    uint32_t* path;
    /* admission estimate and steady-clock times (ns) */
    uint64_t device_bytes_estimate;
    int64_t t_submit_ns, t_admit_ns, t_start_ns, t_finish_ns;
} csaw_result;

typedef struct {
    uint32_t pending;
    uint32_t running;
    uint64_t bytes_in_use;
    uint64_t budget_bytes;
} csaw_server_stats_t;

/* Errors: CSAW_ERR_INVALID, CSAW_ERR_NOMEM, CSAW_ERR_CUDA. */
csaw_status csaw_server_create(csaw_graph* g, const csaw_server_opts* opts, csaw_server** out);

/* Stops the server: requests not yet admitted finish with CSAW_ERR_ABORTED,
 * running ones complete; results not yet polled are released.  The graph
 * must outlive the server. */
csaw_status csaw_server_destroy(csaw_server* s);

/* Queue a request; *ticket identifies it.  Its arguments are checked here
 * (offsets, seeds and starts in range, fanouts positive), so a batch never
 * fails for one request's input.  Errors: CSAW_ERR_INVALID (bad arguments),
 * CSAW_ERR_NOMEM (its estimate exceeds the whole budget), CSAW_ERR_ABORTED
 * (server shutting down). */
csaw_status csaw_submit(csaw_server* s, const csaw_request* r, uint64_t* ticket);

/* Wait up to timeout_us (< 0: forever, 0: no wait) for a request.  When it
 * has finished, *out receives its result (the caller then owns it and the
 * ticket is retired) and the return value is the request's own status.
 * Errors: CSAW_ERR_TIMEOUT (not finished; poll again), CSAW_ERR_NOT_FOUND
 * (unknown or retired ticket), CSAW_ERR_ABORTED (cancelled or shut down). */
csaw_status csaw_poll(csaw_server* s, uint64_t ticket, int64_t timeout_us, csaw_result** out);

/* Cancel a request that has not been admitted yet; it finishes with
 * CSAW_ERR_ABORTED.  CSAW_ERR_INVALID if it already started. */
csaw_status csaw_cancel(csaw_server* s, uint64_t ticket);

csaw_status csaw_server_stats(csaw_server* s, csaw_server_stats_t* out);

/* ---------------------------------------------------------------- no allocation */

/* One selection layer that allocates no device memory.
 *
 * The paper has no counterpart to this call.  It exists for callers that
 * cannot allocate device memory while they run: code living inside another
 * framework's fixed memory budget, runtimes without a device allocator, or a
 * host thread that must not touch the allocator.  It runs the selection of
 * one sampling layer -- the same kernels and draws as csaw_sample's layer
 * `layer` -- for n given (vertex, instance) pairs, with every temporary in a
 * fixed device array of CSAW_NOALLOC_SCRATCH_BYTES that the library holds on
 * every GPU that loads it, until the process exits.
 *   vertices, instances  device uint32[n]: entry e selects from the
 *                neighbours of vertices[e] with the draws of instance
 *                instances[e] (attempt keys (a, vertex, layer, instance))
 *   k            picks per vertex (CSAW_FANOUT_ALL for all)
 *   out_src, out_dst  device uint32[capacity]: entry e's picks are at
 *                [out_offsets[e], out_offsets[e+1]), in pick order
 *   capacity     must be at least n * min(k, max degree)
 *   out_offsets  device uint64[n + 1] (exclusive scan of the pick counts)
 * Limits: n <= CSAW_NOALLOC_MAX_ITEMS; a graph whose maximum degree needs more
 * than the scratch left for one CTA's cumulative array (about 5.5 million
 * neighbours) is rejected.  Errors: CSAW_ERR_INVALID (limits, NULL arrays,
 * a vertex outside the graph, node2vec bias, a current device other than the
 * graph's), CSAW_ERR_CUDA.  n = 0 is valid: out_offsets[0] is set to 0.
 * The call issues work on `stream` and waits once, after checking the
 * vertices, before it launches the selection.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.  The first call made on a device
 * looks up the array's device address there; make that first call before
 * any stream capture.  Every call shares the one array and clears the parts
 * that must start at zero: calls that overlap on the GPU race on it, so
 * serialise them (one stream, one host thread at a time). */
#define CSAW_NOALLOC_MAX_ITEMS (1u << 20)
#define CSAW_NOALLOC_SCRATCH_BYTES (64ull << 20)
csaw_status csaw_select_noalloc(csaw_graph* g, const uint32_t* vertices, const uint32_t* instances,
                                uint32_t n, uint32_t k, uint32_t layer, const csaw_bias* bias,
                                uint64_t rng_seed, uint32_t* out_src, uint32_t* out_dst,
                                uint64_t capacity, uint64_t* out_offsets, void* stream);

/* ---------------------------------------------------------------- counters */

/* Selection counters of the attempts-per-pick measurement (the iterations
 * per pick of Sec. VI / Fig. 10), kept by a library built with -DCSAW_STATS
 * (libcsaw_stats.so; the default build keeps none and returns
 * CSAW_ERR_INVALID).  Counted over every csaw_sample-family selection since
 * the last reset, on all devices' streams after a device synchronisation:
 *   [0] draws consumed: a selection consumes its attempts up to the one that
 *       gave its last pick (repeated sampling), or all CSAW_ATTEMPT_CAP of
 *       them and one per updated-sampling pick
 *   [1] picks of the selections that drew (take-all selections draw nothing)
 *   [2] draws evaluated (whole warp rounds of 32, plus updated-sampling draws)
 *   [3] picks by updated sampling
 *   [4] warp items, [5] CTA items, [6] shared-hub items, [7] unused
 * reset: zero them after reading. */
csaw_status csaw_selection_stats(uint64_t counters[8], int reset);

/* ---------------------------------------------------------------- misc */

/* Message of the last failed call on this thread ("" if none). */
const char* csaw_last_error(void);

/* ABI version: major * 10000 + minor * 100 + patch. */
uint32_t csaw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CSAW_H */
