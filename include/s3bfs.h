/*
 * s3bfs.h -- C ABI of the GB300 (sm_103a) S3BFS level-step library.
 *
 * The library computes breadth-first-search levels with the S3BFS method of
 * Tithi, Fogel and Chowdhury, "An Optimal Level-synchronous Shared-memory
 * Parallel BFS Algorithm with Optimal parallel Prefix-sum Algorithm and its
 * Implications for Energy Consumption" (arXiv 2209.08764): every level
 * gathers the frontier's degrees, prefix-sums them, splits the level's edges
 * into near-equal chunks, scans neighbours writing level and parent
 * without locks or atomic read-modify-writes, keeps each newly reached vertex
 * once (its final owner keeps it) and compacts the next frontier with a
 * second prefix sum (Fig. 1; Algorithm paragraph).
 *
 * All entry points are plain C: pointers and sizes only.  Every integer on the
 * path is int32 (vertex ids, CSR offsets, levels).  Functions return BFS_OK
 * (0) or a negative BFS_E_* code; bfs_strerror() turns a code into text and
 * bfs_last_error() gives the detail of the last failure on this host thread.
 */
#ifndef S3BFS_H
#define S3BFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define BFS_OK 0
#define BFS_E_INVAL (-1)      /* bad argument: n, nnz, CSR contents, src, k, NULL pointer */
#define BFS_E_MULTIGRAPH (-2) /* a row repeats a neighbour (the owner-as-parent dedup needs a simple graph) */
#define BFS_E_NOMEM (-3)      /* device or pinned-host allocation failed, or bfs_opts.max_device_bytes reached */
#define BFS_E_CUDA (-4)       /* a CUDA runtime call or kernel launch failed; see bfs_last_error() */
#define BFS_E_TIMEOUT (-5)    /* a device-side wait (grid barrier or scan look-back) hit its limit */
#define BFS_E_CHECK (-6)      /* checked build only: an index outside its array (the access was skipped) */

/* ---- bfs_create_csr flags ---------------------------------------------- */
#define BFS_DEVICE_PTRS 1 /* row_ptr / col_idx are device pointers (else host pointers) */
#define BFS_VALIDATE 2    /* check the CSR on the host before use (see bfs_create_csr) */
#define BFS_DEDUP 4       /* sort every row and drop duplicate neighbours and self-loops */
#define BFS_SYMMETRIC 8   /* every edge has its reverse (an undirected graph); checked with
                             BFS_VALIDATE.  Enables the bitmask path of bfs_run_batch */

/* ---- bfs_opts.debug_flags (tests only) --------------------------------- */
#define BFS_DEBUG_STALL_BARRIER 1 /* the last CTA never arrives at the first grid barrier,
                                     so the wait runs out and bfs_run returns BFS_E_TIMEOUT */
#define BFS_DEBUG_CHECK_INJECT 2  /* checked build only: the source's row start is set past
                                     col_idx, so the range check stops the traversal with
                                     BFS_E_CHECK before any such access */

/* Tuning knobs; a zero field takes the default.  NULL = all defaults. */
typedef struct bfs_opts {
  int32_t chunk_edges;      /* grain: minimum edges per warp chunk.  Level l runs
                               P_l = min(P, ceil(e_l / chunk_edges)) warps, the
                               work-sensitive thread count of Fig. 1 (the
                               paper's own formula is chunk_edges = 1).  Default 64 */
  int32_t ctas;             /* persistent grid size G in CTAs; 0 = every CTA that can be
                               co-resident on the device */
  int32_t persistent;       /* 1 (default): one cooperative launch runs all levels,
                               separated by device grid barriers; -1: one launch per
                               phase with a host read of the level sizes in between */
  int32_t work_insensitive; /* 1: every warp of the grid is active at every level
                               (chunks of ceil(e_l / P) edges; no small-level mode),
                               the comparison arm of the Experimental Results */
  int32_t spin_limit_ms;    /* limit of every device-side wait; default 1000 ms */
  int32_t debug_flags;      /* BFS_DEBUG_* (tests only); default 0 */
  int32_t relabel;          /* visited bits in shared memory: 0 (default) = for every
                               vertex when n <= 2^18, else for the 2^18 highest-degree
                               vertices after a degree-descending renumbering, when
                               they hold >= half of the edge endpoints, else (graph
                               not skewed, direction = 0) for every vertex when
                               n <= 2^20; 1 = always renumber; -1 = neither.
                               Renumbering is internal: inputs and outputs keep the
                               caller's vertex ids */
  int32_t batch_bitmask;    /* bfs_run_batch on a BFS_SYMMETRIC graph: 0 (default) =
                               groups of up to 64 sources share one traversal with a
                               64-bit mask per vertex; -1 = one traversal per source */
  int32_t small_level_edges;/* a level with at most this many edges (and the small
                               levels that follow it) runs on one CTA with CTA
                               barriers while the rest of the grid waits at one grid
                               barrier: high-diameter graphs have thousands of tiny
                               levels.  0 = default (256 per warp of one CTA: 8192 with
                               32-warp CTAs, 2048 with 8-warp CTAs), -1 = never */
  int32_t cta_warps;        /* warps per CTA of the level loop: 8 (four CTAs per SM),
                               or 16, 24, 32 (one CTA per SM, one copy of the
                               shared-memory visited bits; 128, 80 or 64 registers a
                               thread); 0 = 32 when visited bits are kept, else 16 */
  int32_t direction;        /* 0 (default): every level top-down, the S3BFS level step.
                               1: direction-optimising (needs BFS_SYMMETRIC, else
                               bfs_create_csr fails with BFS_E_INVAL): a level whose
                               frontier edges exceed m_u / do_alpha (m_u = degree sum
                               of the unvisited vertices) runs bottom-up -- every
                               unvisited vertex looks for a parent in the frontier --
                               and the traversal turns top-down again once the
                               frontier shrinks below n / do_beta (Beamer et al.,
                               SC 2012; the paper names bottom-up steps as compatible
                               with S3BFS in its conclusion).  Levels are the same;
                               parents are another valid BFS tree.  Persistent loop
                               only: with persistent = -1 every level is top-down */
  int32_t do_alpha;         /* 0 = 15 */
  int32_t do_beta;          /* 0 = 18 */
  int32_t do_gamma;         /* a top-down level turns bottom-up only if, besides the
                               alpha test, its frontier's edges exceed do_gamma times
                               the unvisited vertices of degree > 0 (on a GPU a
                               bottom-up test costs about what a top-down one does);
                               0 = 2, -1 = no such test (Beamer's rule alone) */
  int32_t reserved;         /* must be 0 */
  int64_t max_device_bytes; /* cap on the device memory this handle allocates, at create
                               time and later (the bitmask-batch and queued-batch buffers
                               are allocated at their first use); an allocation that
                               would pass it fails with BFS_E_NOMEM and the call
                               allocates nothing more.  0 = no cap */
} bfs_opts;

/* Per-level record written to bfs_stats.per_level, BFS_LEVEL_FIELDS int32 each. */
#define BFS_LEVEL_FIELDS 9
/* [0] n_l          frontier size (vertices at distance l)
 * [1] e_l          edges the level scans (sum of frontier out-degrees)
 * [2] c_l          candidates emitted by the explore step (n_{l+1} <= c_l <= e_l)
 * [3] active_warps P_l, warps that explored this level
 * [4] active_sms   distinct SMs hosting those warps (-1 with one launch per phase)
 * [5] ns           device time of the level, explore to the end of the compact
 *                  barrier, from the global timer (-1 with one launch per phase)
 * [6] ns_explore   the part of [5] up to the end of the explore barrier
 *                  (bottom-up: of the neighbour scan)
 * [7] direction    0 top-down, 1 bottom-up
 * [8] work         neighbour entries examined (top-down: e_l) */

/* Statistics of one traversal (all optional). */
typedef struct bfs_stats {
  int32_t num_levels;     /* non-empty levels, = 1 + the largest distance reached */
  int32_t active_ctas;    /* G, CTAs of the persistent grid */
  int64_t reached;        /* vertices with level >= 0 */
  int64_t edges_scanned;  /* sum of e_l = out-degree sum of reached vertices */
  int64_t candidates;     /* sum of c_l */
  float ms_level_step;    /* device time of the level loop (all levels), CUDA events */
  float ms_total;         /* device time including initialisation */
  int32_t *per_level;     /* in: optional host buffer of per_level_cap * BFS_LEVEL_FIELDS int32 */
  int32_t per_level_cap;  /* in: capacity in levels; levels beyond it are counted, not recorded */
  int32_t launches;       /* kernels the call launched (for a bitmask batch group: the group's) */
  int64_t work_edges;     /* neighbour entries the kernels examined: edges_scanned for a
                             top-down traversal, fewer with bottom-up levels; for a bitmask
                             batch group, the pulled entries of all its levels */
} bfs_stats;

typedef struct bfs_graph bfs_graph; /* opaque; owned by the library */

/*
 * bfs_create_csr -- take a graph and allocate everything a traversal needs.
 *
 * Graph: n vertices, nnz directed edges in CSR form: row_ptr[n+1] int32 with
 * row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz; col_idx[nnz] int32 with
 * 0 <= col_idx[e] < n.  Out-edges are explored, so a directed CSR is allowed;
 * an undirected graph is given with both directions.  The graph must be
 * simple within each row (no repeated neighbour): the dedup step keeps a
 * candidate (v, u) when parent[v] still equals u after the level, which is
 * unique per v only if u reaches v by one edge (Fig. 1's owner check, with the
 * owner id taken to be the parent vertex).  Self-loops are harmless.
 *
 * Ownership: the CSR is COPIED into library-owned device memory; the caller
 * may free its arrays when this returns.  With BFS_DEVICE_PTRS the arrays are
 * read as device pointers, otherwise as host pointers.  BFS_VALIDATE checks
 * all the conditions above on the host (BFS_E_INVAL / BFS_E_MULTIGRAPH);
 * BFS_DEDUP instead rewrites every row sorted, without duplicates or
 * self-loops.  Without either flag the CSR is trusted; a repeated neighbour
 * may then make bfs_run fail with BFS_E_MULTIGRAPH.
 *
 * Work memory (all device, allocated here once): level and parent arrays
 * (n each), two frontier records of n+1 entries x 3 int32, candidate pairs
 * for up to nnz edges, per-warp scan state and the per-level statistics.
 * Limits: 1 <= n < 2^31 - 8, 0 <= nnz < 2^31 - 64.
 *
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream).  All work of
 * this graph is ordered on it.  The current CUDA device at this call is the
 * graph's device.  Returns BFS_OK and *out, or an error code and *out = NULL.
 */
int bfs_create_csr(int32_t n, int32_t nnz, const int32_t *row_ptr, const int32_t *col_idx, int flags,
                   const bfs_opts *opts, void *cuda_stream, bfs_graph **out);

/*
 * bfs_run -- one traversal from src (Parallel-BFS(s, P), Fig. 1).
 *
 * level_out[n] receives hop distances (level[src] = 0, -1 = unreachable, the
 * paper's infinity).  parent_out[n] (nullable) receives a BFS tree:
 * parent[src] = src, -1 where unreachable, otherwise a vertex one level up
 * with an edge to v.  The tree is not unique; which writer wins the benign
 * race decides it (Algorithm paragraph).  Each output may be a device pointer
 * (written in place by the kernels) or a host pointer (copied back at the
 * end); the kind is detected per pointer.  Blocks until the traversal is
 * complete.  stats (nullable) receives the statistics.  Errors: BFS_E_INVAL
 * (src out of range, NULL level_out), BFS_E_TIMEOUT, BFS_E_MULTIGRAPH,
 * BFS_E_CUDA.  Outputs are undefined on error; the graph stays usable after
 * BFS_E_INVAL, BFS_E_TIMEOUT and BFS_E_MULTIGRAPH.
 */
int bfs_run(bfs_graph *g, int32_t src, int32_t *level_out, int32_t *parent_out, bfs_stats *stats);

/*
 * bfs_run_batch -- k traversals on the same graph, one per source.
 *
 * levels_out[k*n] (source-major: traversal i at levels_out + i*n), and
 * parents_out[k*n] (nullable), device or host pointers as for bfs_run.  stats
 * (nullable) points to k records.  Results are those of k calls of bfs_run
 * (levels identical; parents a valid BFS tree, not necessarily the same one).
 *
 * On a graph created with BFS_SYMMETRIC (and opts.batch_bitmask = 0) the
 * sources are taken 64 at a time in one launch: every vertex keeps a 64-bit
 * mask of the sources that reached it and pulls its neighbours' frontier
 * masks each level (multi-source BFS; not in the paper, whose distance
 * definition it keeps).  Its working memory (3 x 8 bytes per vertex, plus
 * 2 x 64 x n int32 for host output buffers) is allocated at the first such
 * call.  In each stats record of such a group, ms_level_step and ms_total are
 * those of the whole group and candidates = reached - 1.  Otherwise the
 * sources run one after another.  With the persistent loop, no per-level
 * records requested and both outputs on the same side (device or host), the
 * traversals are queued back to back, up to 8 ahead of the host, which
 * checks each one as it finishes.  Host outputs then go through eight device
 * staging slots (2 x n int32 each, allocated at the first such call) and a
 * second stream copies traversal i's outputs while the next traversals run,
 * so pinned host buffers cost little beyond the traversals themselves.
 *
 * Errors as for bfs_run; on error the index of the failing source (or group)
 * is in bfs_last_error().
 */
int bfs_run_batch(bfs_graph *g, const int32_t *srcs, int32_t k, int32_t *levels_out, int32_t *parents_out,
                  bfs_stats *stats);

/* bfs_destroy -- free everything the graph owns.  NULL is a no-op. */
void bfs_destroy(bfs_graph *g);

/* bfs_strerror -- static text for a status code. */
const char *bfs_strerror(int code);

/* bfs_last_error -- detail of the last failing call on this host thread
 * (thread-local, valid until the next call into the library). */
const char *bfs_last_error(void);

/* bfs_graph_info -- n, nnz and the persistent grid (CTAs, warps) of a graph;
 * any output pointer may be NULL. */
int bfs_graph_info(const bfs_graph *g, int32_t *n, int32_t *nnz, int32_t *ctas, int32_t *warps);

/* bfs_run_frontiers -- debug form of bfs_run that also returns every level's
 * frontier (Fig. 1: CurLevelVertices after the owner check and linearisation).
 *
 * Only the checked build (libs3bfs_checked.so, compiled with S3BFS_CHECKED=1:
 * every global index range-checked, BFS_E_CHECK instead of an out-of-range
 * access) implements it; the production library returns BFS_E_INVAL.
 * frontiers_out: HOST array of n int32 receiving F_0, F_1, ... back to back
 * in caller ids (F_0 = [src]); bfs_stats.per_level gives each n_l, and their
 * sum is stats->reached.  Order within a level is arbitrary; as sets the
 * levels are exact.  Other arguments as for bfs_run. */
int bfs_run_frontiers(bfs_graph *g, int32_t src, int32_t *level_out, int32_t *parent_out, bfs_stats *stats,
                      int32_t *frontiers_out);

/* bfs_graph_device_bytes -- device memory the graph currently holds (what
 * bfs_opts.max_device_bytes caps), in bytes; -1 if g is NULL.  Buffers that
 * bitmask batches and queued batches allocate at their first use count from
 * then on. */
int64_t bfs_graph_device_bytes(const bfs_graph *g);

/*
 * bfs_run_csr_noalloc -- one traversal that allocates no memory at all.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they traverse, e.g. code running inside a
 * host framework whose caching allocator owns the GPU's memory (a second
 * allocator would fragment its pool or exceed its budget), or latency-critical
 * loops where cudaMalloc / cudaFree would synchronise the device and stall
 * other streams.  It never calls cudaMalloc, cudaFree or any allocating
 * library routine.
 *
 * Arguments: a CSR as for bfs_create_csr, but as DEVICE pointers owned by the
 * caller (row_ptr[n+1], col_idx[nnz]; read only, no alignment needed); the
 * source; and DEVICE outputs level_out[n] and parent_out[n] (both required),
 * with the meaning of bfs_run.  cuda_stream as for bfs_create_csr.  Blocks until
 * the traversal is complete.
 *
 * Working memory: one static device array of about 40 MB that every GPU
 * loading this library's device code reserves until the process exits.  It
 * bounds the sizes: 1 <= n <= 262,144 and 0 <= nnz <= 2,097,152; larger graphs
 * are rejected with BFS_E_INVAL and a message in bfs_last_error().  The CSR is
 * range-checked on every call (BFS_E_INVAL); it must be simple within rows, as
 * for bfs_create_csr without BFS_VALIDATE.
 *
 * Every call, from any thread or stream, shares that one array, which keeps
 * the last call's contents; each call clears the state that must start at
 * zero.  Calls that overlapped on the GPU would race on the array and give
 * wrong results, so the library holds a per-device lock for the whole of
 * each call (which returns only once its traversal is done): calls from
 * different host threads on one device run one after another.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and the grid size; make that first call before any
 * stream capture.
 */
int bfs_run_csr_noalloc(int32_t n, int32_t nnz, const int32_t *row_ptr, const int32_t *col_idx, int32_t src,
                        int32_t *level_out, int32_t *parent_out, void *cuda_stream);

/* ---- query server: continuous batching over a pool of graphs ------------ */

typedef struct bfs_server bfs_server; /* opaque; owned by the library */

typedef struct bfs_server_opts {
  int32_t slots;             /* queries running at once (<= 128 and <= the grid's CTAs);
                                0 = 64 */
  int32_t levels_per_launch; /* level steps a launch may run before the scheduler
                                retires and admits; 0 = 64 (a launch also ends when a
                                query finishes, and after the current step when a
                                submission arrives) */
  int32_t chunk_edges;       /* grain, as bfs_opts.chunk_edges; 0 = 64 */
  int32_t cta_warps;         /* 8, 16 or 32 warps per CTA; 0 = 16 */
  int32_t spin_limit_ms;     /* device wait limit; 0 = 1000 */
  int32_t local_levels;      /* > 0: a query that gets one CTA and whose level has at most
                                256 edges per warp runs up to this many levels per step on
                                that CTA alone, with CTA barriers; 0 = off (the default:
                                on the serving pool it did not lower p99 and it cut the
                                saturated throughput) */
  int64_t arena_bytes;       /* device memory for the working buffers of running
                                queries (admission waits while it is full);
                                0 = half of the free memory, at most 32 GiB */
} bfs_server_opts;

typedef struct bfs_completion {
  int64_t tag;           /* the caller's tag from bfs_server_submit */
  int32_t graph, src;
  int32_t status;        /* BFS_OK or an error code (outputs undefined then) */
  int32_t num_levels;
  int64_t reached, edges_scanned;
  double t_submit_us;    /* host steady clock, microseconds: submitted, */
  double t_admit_us;     /* admitted (its memory taken, level 0 set), */
  double t_done_us;      /* and seen finished, with its outputs written */
} bfs_completion;

/*
 * bfs_server_create -- a server over ngraphs graphs made by bfs_create_csr on
 * the current device (the graphs stay owned by the caller and must outlive
 * the server).  Queries on any of them are admitted into free slots while
 * their working memory (about 24 bytes per vertex and 12 per edge of their
 * graph) fits in the server's arena, and run together: every level of every
 * running query is the S3BFS level step of bfs_run (Fig. 1) on its share of
 * the grid (at least one CTA, the rest in proportion to the level's edge
 * count).  Batching queries is not in the paper.  cuda_stream as for
 * bfs_create_csr.
 */
int bfs_server_create(bfs_graph *const *graphs, int32_t ngraphs, const bfs_server_opts *opts, void *cuda_stream,
                      bfs_server **out);

/*
 * bfs_server_submit -- queue one traversal of graph `graph` (index into the
 * create-time array) from src.  level_out / parent_out (nullable; both may be
 * NULL to discard the result) receive the result as in bfs_run, device or
 * host pointers; they must stay valid until the query's completion is
 * returned by bfs_server_poll.  Host-side only: nothing runs until the next
 * poll.  May be called from any thread, also while another thread is inside
 * bfs_server_poll: a launch then running returns after its current level
 * step (a host-mapped wake flag), so that the next poll admits the query.
 * Errors: BFS_E_INVAL.
 */
int bfs_server_submit(bfs_server *s, int32_t graph, int32_t src, int32_t *level_out, int32_t *parent_out,
                      int64_t tag);

/*
 * bfs_server_poll -- one scheduling round: admit queued queries, run one
 * launch over every running query (it returns when a query finishes or after
 * levels_per_launch levels), retire the finished ones.  Up to cap completion
 * records are written to out (the rest are kept for later polls); *ndone is
 * their number.  Blocks for the launch, without holding the server's lock
 * (submissions from other threads proceed meanwhile).  Call it in a loop
 * while queries are queued or running (bfs_server_pending), from one thread
 * at a time (a second concurrent call fails with BFS_E_INVAL).
 */
int bfs_server_poll(bfs_server *s, bfs_completion *out, int32_t cap, int32_t *ndone);

/* bfs_server_pending -- queries queued (not admitted) and running. */
int bfs_server_pending(bfs_server *s, int32_t *queued, int32_t *running);

/* bfs_server_destroy -- free the server (not the graphs).  NULL is a no-op. */
void bfs_server_destroy(bfs_server *s);

#ifdef __cplusplus
}
#endif

#endif /* S3BFS_H */
