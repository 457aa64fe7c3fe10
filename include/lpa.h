/*
 * lpa.h -- C ABI of liblpa: GPU label propagation (GVE-LPA, Sahu, arXiv
 * 2312.08140) for NVIDIA GB300 (sm_103a).
 *
 * Terms follow the paper (Section 3): an undirected graph G(V, E, w) with
 * w_ij = w_ji is given as CSR holding both directions of every edge;
 * N = |V|; C_i is the label (community id) of vertex i; one "sweep" is one
 * call of lpaMove in Algorithm 1.
 *
 * Conventions for every entry point:
 *   - The return value is an lpa_status; no call aborts the process.  On
 *     error, output arguments are left untouched and lpa_last_error() gives a
 *     one-line reason (thread-local).
 *   - "device" pointers are CUDA device (or managed) pointers of the current
 *     device; "host" pointers are ordinary or pinned host memory.
 *   - The library owns what it allocates and frees it in the matching
 *     *_destroy call.  The caller owns every buffer it passes in and every
 *     stream.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls documented as asynchronous only enqueue work on it.
 *   - A handle may be used by one host thread at a time, and its runs must be
 *     ordered (one stream, or explicit synchronisation between streams).
 *   - Vertex ids and labels are int32 (N <= 2^31 - 1); entry counts are int64.
 */
#ifndef LPA_H_
#define LPA_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LPA_OK = 0,
    LPA_ERR_INVALID_ARG = 1,    /* a scalar argument or pointer is out of its documented range */
    LPA_ERR_INVALID_GRAPH = 2,  /* CSR failed validation (offsets, index range, weights) */
    LPA_ERR_OUT_OF_MEMORY = 3,  /* a device or pinned allocation failed */
    LPA_ERR_CUDA = 4,           /* a CUDA runtime call failed; see lpa_last_error() */
    LPA_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
    LPA_ERR_BUSY = 6,           /* serving: the request does not fit the HBM budget right now */
    LPA_ERR_NOT_FOUND = 7,      /* serving: unknown ticket */
    LPA_ERR_NOT_READY = 8       /* serving: ticket not finished yet */
} lpa_status;

/* Sweep semantics.
 * LPA_MODE_SYNC       Jacobi reading of Algorithm 1: every vertex of sweep t
 *                     reads the labels left by sweep t-1; ties go to the
 *                     smallest label id (Section 4.1.5).  Only vertices with a
 *                     neighbour that changed in sweep t-1 are scanned (vertex
 *                     pruning, Section 4.1.4); this never changes the result
 *                     because a vertex's pick depends on its neighbours'
 *                     labels only.  Deterministic.
 * LPA_MODE_ASYNC      Algorithm 1 as the paper runs it (Section 4.1): labels
 *                     are updated in place while other vertices read them,
 *                     with vertex pruning.  Each sweep scans the unprocessed
 *                     vertices, then the vertices marked during that scan
 *                     that were not in it (the serial loop reaches those later
 *                     in the same sweep); a vertex is scanned at most once per
 *                     sweep, and one already scanned keeps a new mark for the
 *                     next sweep.  dN counts both passes.  Results depend on
 *                     timing.
 * LPA_MODE_SYNC_FULL  LPA_MODE_SYNC without pruning: every vertex is scanned
 *                     in every sweep.  Same labels as LPA_MODE_SYNC. */
typedef enum {
    LPA_MODE_SYNC = 0,
    LPA_MODE_ASYNC = 1,
    LPA_MODE_SYNC_FULL = 2
} lpa_mode;

/* OR into the mode of lpa_run / lpa_run_profiled / lpa_batch_run / lpa_autotune
 * for the non-strict tie-break of Section 4.1.5 (one of the most weighted
 * labels chosen pseudo-randomly through a modulo of the label id), read
 * as: vertex i (id within its graph) in its graph's sweep t draws
 * r = SplitMix64((t << 32) | i) mod n and takes, among the most weighted
 * labels, the first one at or after r in cyclic label order (the label c
 * minimising (c - r) mod n, c within the graph).  Deterministic, so the
 * synchronous modes stay exact; since a non-strict pick depends on the sweep,
 * pruning no longer leaves the result unchanged, and LPA_MODE_SYNC |
 * LPA_NONSTRICT runs as LPA_MODE_SYNC_FULL (every vertex every sweep).
 * Not accepted by lpa_serve_*. */
#define LPA_NONSTRICT 0x100

/* Mode flag, LPA_MODE_ASYNC only (LPA_ERR_INVALID_ARG with the synchronous
 * modes): the pruning rule of FLPA (Section 2), under which a vertex whose
 * label changes to c marks unprocessed only the neighbours whose label is not
 * c, instead of every neighbour (Section 4.1.4).  A neighbour already in c
 * gains weight for c and keeps it in the usual case, so the frontiers shrink;
 * the results are those of a different (still asynchronous) algorithm.
 * Not accepted by lpa_serve_*. */
#define LPA_PRUNE_OTHER 0x200

/* lpa_graph_create / lpa_batch_create flags */
#define LPA_HOST_PTRS   0u  /* offsets/indices/weights are host memory; the library copies them */
#define LPA_DEVICE_PTRS 1u  /* they are device memory; the library copies them (unless LPA_BORROW) */
#define LPA_BORROW      2u  /* with LPA_DEVICE_PTRS: use the caller's device arrays in place; they
                               must stay alive and unchanged until *_destroy.  Indices that are not
                               16-byte aligned are copied all the same (the sweeps move index rows
                               with 16-byte bulk copies) */

/* Storage order of the vertices (lpa_graph_create / lpa_batch_create flags,
 * at most one).  The library may store a graph's vertices in an order of its
 * own; labels in and out are always the caller's vertex ids, initial labels
 * are the ids (Algorithm 1) and ties go by id, so results are those of the
 * caller's graph: LPA_MODE_SYNC gives the same labels in every order, and
 * the asynchronous modes differ only in the order the parallel sweep meets
 * the vertices (Algorithm 1 leaves that order open).  A reordered graph is a
 * library copy even when LPA_BORROW is given.
 *   LPA_REORDER_DEGREE   single graphs: vertices by decreasing degree bucket
 *                        ceil(log2 d), then by id -- the labels that most
 *                        gathers read sit together in memory and in L2
 *   LPA_REORDER_SHUFFLE  each graph's vertices in a pseudo-random order of
 *                        their own (a Feistel permutation of its id range):
 *                        the asynchronous sweep, which walks stored vertices
 *                        in order, then meets a graph's vertices in a random
 *                        order even when the graph spans many waves of warps.
 *                        The default of lpa_batch_create.
 *   LPA_KEEP_ORDER       lpa_batch_create: keep the caller's order. */
#define LPA_REORDER_DEGREE  4u
#define LPA_REORDER_SHUFFLE 8u
#define LPA_KEEP_ORDER      16u

/* Per-sweep history kept in lpa_run_info (sweeps beyond this are still run). */
#define LPA_MAX_RECORDED_ITERS 64
/* Degree bins of lpa_config (thread, warp, three block sizes). */
#define LPA_BINS 5

typedef struct {
    int32_t iterations;    /* sweeps performed, including the one that met the tolerance */
    int32_t exit_reason;   /* 0: dN/N <= tolerance; 1: max_iters reached; 2: nothing to run
                              (N == 0 or max_iters == 0) */
    int64_t changed[LPA_MAX_RECORDED_ITERS];  /* dN of each sweep (Algorithm 1) */
    int64_t active[LPA_MAX_RECORDED_ITERS];   /* vertices scanned in each sweep */
    int64_t scanned[LPA_MAX_RECORDED_ITERS];  /* CSR entries of the scanned vertices */
    int64_t edges_touched;                    /* sum of scanned[] over all sweeps */
} lpa_run_info;

typedef struct {
    int64_t n;             /* vertices (sum over graphs for a batch) */
    int64_t nnz;           /* stored CSR entries */
    int32_t num_graphs;    /* 1 for lpa_graph_t */
    int32_t weighted;      /* 0: unit weights (weights == NULL at create) */
    int32_t exact;         /* 1: every per-label sum is computed exactly, so LPA_MODE_SYNC is
                              bit-exact against an exact-arithmetic reference: all weights are
                              integers (or unit) and every weighted degree is < 2^31 (the
                              library's own copy, summed in 32-bit integers) or < 2^24
                              (borrowed weights, summed in fp32) */
    int32_t weight_bytes;  /* bytes per entry of the weights the sweeps read: 0 (unit), 1 (integer
                              weights <= 255 in the library's copy), 4 (other) */
    int64_t max_degree;
    int64_t device_bytes;  /* device memory the handle holds */
    int64_t sweeps_total;  /* sweeps run on this handle since creation (all runs) */
    int64_t scanned_total; /* CSR entries scanned by those sweeps */
    int64_t launches_total;/* kernel launches of the lpa_run calls on this handle */
    int32_t rows_distinct; /* 1: a single graph whose every row lists its neighbours in strictly
                              increasing order as given (so none twice); the first LPA_MODE_SYNC
                              sweep then reads no labels (each is still its vertex's id) and takes
                              the heaviest entry of each row.  0 for batches and other graphs. */
    int32_t storage_order; /* 0: the caller's order, 1: LPA_REORDER_DEGREE, 2: LPA_REORDER_SHUFFLE */
} lpa_graph_props;

/* Launch parameters of the sweep.  Vertices are binned by degree d:
 *   d <= small_max                  one thread per vertex, row held in registers
 *   small_max < d <= warp_max       one warp per vertex, per-warp shared-memory table
 *   warp_max  < d <= mid_max        one 128-thread block per vertex, shared table
 *   mid_max   < d <= large_max      one 256-thread block per vertex, shared table
 *   d > large_max                   one 512-thread block per vertex, 8192-slot shared
 *                                   table; a row whose distinct labels overflow it is
 *                                   split over hash partitions of its labels: it is
 *                                   read once in slices grouped by partition, then
 *                                   aggregated by one block per partition (rows
 *                                   beyond that path's limits are rescanned by one
 *                                   block per partition)
 * A sweep is "dense" (every vertex with an entry is scanned, no frontier
 * compaction) when the vertices changed since the previous compaction hold
 * at least dense_permille / 1000 of all entries; the first sweep is always
 * dense (Algorithm 1 starts with every vertex unprocessed); 1001 = never
 * otherwise.  Scanning a vertex whose neighbours did not change never
 * changes its label in LPA_MODE_SYNC, so this choice affects speed only.
 * lpa_graph_set_config validates: 1 <= small_max <= 8, small_max < warp_max
 * <= 256, warp_max < mid_max <= 2048, mid_max < large_max <= 4096,
 * 0 <= dense_permille <= 1001. */
typedef struct {
    int32_t small_max;
    int32_t warp_max;
    int32_t mid_max;
    int32_t large_max;
    int32_t dense_permille;
} lpa_config;

/* Time per phase of one run, from CUDA events recorded around every launch
 * (lpa_run_profiled).  Times in milliseconds. */
typedef struct {
    int32_t iterations;
    int32_t reserved;
    float   init_ms;
    float   finish_ms[LPA_MAX_RECORDED_ITERS];          /* apply + frontier compaction + control */
    float   sweep_ms[LPA_MAX_RECORDED_ITERS][LPA_BINS]; /* per degree bin of lpa_config */
    int64_t bin_vertices[LPA_MAX_RECORDED_ITERS][LPA_BINS];
    int64_t bin_entries[LPA_MAX_RECORDED_ITERS][LPA_BINS];
    int64_t bin_changed[LPA_MAX_RECORDED_ITERS][LPA_BINS];
    int64_t bin_changed_entries[LPA_MAX_RECORDED_ITERS][LPA_BINS];  /* entries of changed vertices */
} lpa_profile;

typedef struct lpa_graph  *lpa_graph_t;
typedef struct lpa_batch  *lpa_batch_t;
typedef struct lpa_server *lpa_server_t;

/* Library version string, e.g. "lpa-gb300 0.1". */
const char *lpa_version(void);

/* Static text for a status code. */
const char *lpa_status_string(lpa_status st);

/* Reason for the last non-OK status returned on this thread ("" if none). */
const char *lpa_last_error(void);

/* The tolerance test of Algorithm 1 (Section 4.1.3), dN / N <= tolerance,
 * as the integer every run compares dN against: a sweep of a graph with n
 * vertices meets the tolerance when dN <= *out = floor(tolerance * n), the
 * product rounded once to fp64 (for decimal tolerances such as 0.05 and
 * n < 2^31 this equals the exact floor of the decimal times n).  Host only:
 * needs no GPU.  LPA_ERR_INVALID_ARG unless 0 <= tolerance <= 1,
 * 0 <= n <= 2^31 - 1 and out != NULL. */
lpa_status lpa_tolerance_threshold(double tolerance, int64_t n, int64_t *out);

/* ---------------------------------------------------------------- graphs */

/* Build a graph handle from CSR (Section 3: undirected, w_ij = w_ji).
 *   n         vertices, 0 <= n <= 2^31 - 1
 *   nnz       stored entries, >= 0; offsets[n] must equal nnz
 *   offsets   int64[n+1], offsets[0] == 0, non-decreasing
 *   indices   int32[nnz], each in [0, n); rows need not be sorted; an entry
 *             (i, i) is a self-loop, skipped by the sweep (Algorithm 1,
 *             scanCommunities) and counted by lpa_modularity
 *   weights   float32[nnz] finite and >= 0, or NULL for unit weights (the
 *             paper's setting, Table 1).  Symmetry is the caller's contract
 *             and is not checked.
 *   flags     LPA_HOST_PTRS | LPA_DEVICE_PTRS, optionally | LPA_BORROW, optionally one storage
 *             order (LPA_REORDER_DEGREE, LPA_REORDER_SHUFFLE)
 * Validates the CSR on the device (returns LPA_ERR_INVALID_GRAPH on failure)
 * and synchronises `stream` before returning.  Device memory: the CSR copy
 * (unless borrowed) plus about 21 bytes per vertex of working state (two
 * label buffers, flags, the frontier bitmap, bin lists and change marks) and
 * 8 more per vertex once lpa_modularity has been called, taken from the
 * library's per-device memory pool; lpa_graph_props reports the total. */
lpa_status lpa_graph_create(int64_t n, int64_t nnz, const int64_t *offsets, const int32_t *indices,
                            const float *weights, uint32_t flags, void *stream, lpa_graph_t *out);

/* Waits for all work on the graph's device (as cudaFree does), then returns
 * the graph's memory to the library's pool, which keeps it for the next
 * graph or batch created on that device. */
lpa_status lpa_graph_destroy(lpa_graph_t g);

/* Gives the pool's cached (freed, not in use) device memory back to the
 * driver on every device; memory of live graphs and batches is unaffected.
 * No counterpart in the paper: a memory-management call of this library. */
lpa_status lpa_release_cached_memory(void);

/* Properties of a handle (host struct).  Waits for all work on the device
 * (cudaDeviceSynchronize) so that the cumulative counters are current. */
lpa_status lpa_graph_props_get(lpa_graph_t g, lpa_graph_props *out);

/* Read or replace the degree-bin launch parameters (see lpa_config). */
lpa_status lpa_graph_get_config(lpa_graph_t g, lpa_config *out);
lpa_status lpa_graph_set_config(lpa_graph_t g, const lpa_config *cfg);

/* Test hook for the bounded device-side waits (no counterpart in the paper).
 * block_threads 128, 256 or 512: in the next run that launches the row
 * kernel of that block size past its first-sweep shortcut, the first block to
 * produce a tile leaves that tile's index copy unissued, once; the warps
 * waiting on it give up after 2 s and the run returns LPA_ERR_TIMEOUT,
 * leaving the context usable (the next run starts clean).  0 cancels a
 * pending request.  Other values: LPA_ERR_INVALID_ARG. */
lpa_status lpa_graph_debug_stall(lpa_graph_t g, int32_t block_threads);

/* Run label propagation (Algorithm 1, lpa()): C <- [0..N), then sweeps until
 * dN/N <= tolerance (Section 4.1.3; the paper uses 0.05) or max_iters sweeps
 * (Section 4.1.2; the paper uses 20).
 *   mode        lpa_mode
 *   tolerance   in [0, 1]; a sweep meets it when dN <= floor(tolerance * N)
 *               (lpa_tolerance_threshold)
 *   max_iters   in [0, 1 << 20]
 *   labels_out  device int32[n], caller-owned; receives C
 *   info        host pointer or NULL.  When non-NULL the call waits for the
 *               run to finish and fills it; when NULL the call only enqueues
 *               work on `stream` and returns.
 * The whole loop runs on the device (a CUDA graph with a device-side loop
 * condition): no host round trip per sweep. */
lpa_status lpa_run(lpa_graph_t g, lpa_mode mode, double tolerance, int32_t max_iters,
                   int32_t *labels_out, void *stream, lpa_run_info *info);

/* Same result as lpa_run, but every launch is issued from the host and timed
 * with CUDA events; per-phase times and per-bin counts go to *prof (host).
 * Blocks until done.  For profiling only: slower than lpa_run. */
lpa_status lpa_run_profiled(lpa_graph_t g, lpa_mode mode, double tolerance, int32_t max_iters,
                            int32_t *labels_out, void *stream, lpa_run_info *info, lpa_profile *prof);

/* Modularity Q of a labelling (Eq. 1, Section 3.2, community form):
 *   Q = sum_c [ sigma_c / 2m - (Sigma_c / 2m)^2 ]
 * with 2m the sum of all stored entries' weights, sigma_c the weight of
 * entries (i, j) with C_i = C_j = c and Sigma_c the sum of weighted degrees
 * K_i over i in c.  Sums in fp64.  Q = 0 when 2m = 0.
 *   labels  device int32[n], each in [0, n) (else LPA_ERR_INVALID_ARG)
 *   q_out   host double; the call synchronises `stream` before returning. */
lpa_status lpa_modularity(lpa_graph_t g, const int32_t *labels, double *q_out, void *stream);

/* What an autotuner call did (host struct). */
typedef struct {
    int32_t cached;         /* 1: the configuration came from the process-wide cache; nothing was timed */
    int32_t candidates;     /* configurations timed, the one in force before the call included */
    float   search_ms;      /* wall time of the call */
    float   default_ms;     /* best timed run of the configuration in force before the call (on the sample) */
    float   chosen_ms;      /* best timed run of the chosen configuration (on the sample) */
    int32_t sample_graphs;  /* graphs in the timed sample */
    int32_t reserved;
} lpa_autotune_info;

/* Pick the degree-bin launch parameters (lpa_config) for this graph and run
 * mode -- the GPU counterpart of the paper's scheduling choice (Section
 * 4.1.1: OpenMP dynamic scheduling in chunks of 2048 vertices).  A log2
 * degree histogram of the graph, taken on the device, bins the vertices under
 * every candidate (limits are powers of two); candidates that bin them as an
 * earlier one does are skipped.  One pass of coordinate descent over
 * warp_max, mid_max, small_max, large_max and dense_permille, starting from
 * the configuration in force (itself a candidate), times each candidate with
 * `trials` runs of lpa_run (best kept, after one untimed run).  The winner is
 * applied to the handle and copied to *chosen (host, nullable); *info (host,
 * nullable) receives what the call did.  Choices are cached for the life of
 * the process, keyed by mode, weight storage and the histogram rounded to
 * 1/64 of the vertices and of the entries per bucket: a later call on a
 * workload of the same shape applies the cached choice without timing.
 * Results do not depend on the configuration (it moves work between
 * kernels, not the arithmetic), so LPA_MODE_SYNC labels stay the same.
 * Synchronous; uses a label buffer of its own, no caller buffer is touched. */
lpa_status lpa_autotune(lpa_graph_t g, lpa_mode mode, double tolerance, int32_t max_iters,
                        int32_t trials, void *stream, lpa_config *chosen, lpa_autotune_info *info);

/* Forgets every cached autotuner choice. */
lpa_status lpa_autotune_cache_clear(void);

/* Modularity of a labelling, as lpa_modularity, for callers that cannot let
 * the library allocate device memory: the CSR stays in the caller's device
 * arrays (same rules as lpa_graph_create; not validated here) and the working
 * memory is a fixed array inside the library, sized for at most 1,048,576
 * vertices (larger n returns LPA_ERR_INVALID_ARG).  The paper has no
 * counterpart to this entry point; it exists for code that may not call
 * cudaMalloc: a plugin whose host framework owns all device memory through
 * its own pool, or a latency-critical loop that cannot afford an allocation.
 *   n, nnz, offsets, indices, weights   device CSR (weights NULL = unit)
 *   labels   device int32[n], each in [0, n)
 *   q_out    host double; the call synchronises `stream` before returning.
 * Allocates nothing.  The first call on each device (and again after that
 * device's context is recreated) looks up the array's device address; make
 * it before any stream capture.  Every call uses the same array and clears
 * what must start at zero: calls that run concurrently on the GPU race. */
lpa_status lpa_modularity_noalloc(int64_t n, int64_t nnz, const int64_t *offsets, const int32_t *indices,
                                  const float *weights, const int32_t *labels, double *q_out, void *stream);

/* ---------------------------------------------------------------- batches */

/* G independent graphs packed back to back into one handle, solved together
 * by one device-side loop (each graph keeps its own dN, tolerance test and
 * sweep count, Algorithm 1 per graph).
 *   graph_vtx_off   host int64[G+1]: graph g owns vertices [vo[g], vo[g+1])
 *   graph_edge_off  host int64[G+1]: and entries [eo[g], eo[g+1])
 *   offsets         int64[N+1] positions into the packed indices (global),
 *                   offsets[vo[g]] == eo[g]
 *   indices         int32[E], LOCAL vertex ids of the entry's own graph
 *   weights         float32[E] or NULL
 *   flags           as lpa_graph_create (LPA_BORROW is not accepted: indices
 *                   are rewritten to global ids in the library's copy); each
 *                   graph's vertices are stored shuffled (LPA_REORDER_SHUFFLE)
 *                   unless LPA_KEEP_ORDER is given
 * Synchronises `stream`. */
lpa_status lpa_batch_create(int32_t G, const int64_t *graph_vtx_off, const int64_t *graph_edge_off,
                            const int64_t *offsets, const int32_t *indices, const float *weights,
                            uint32_t flags, void *stream, lpa_batch_t *out);

lpa_status lpa_batch_destroy(lpa_batch_t b);

lpa_status lpa_batch_props_get(lpa_batch_t b, lpa_graph_props *out);

/* Run every graph of the batch: labels_out is device int32[N] with LOCAL ids
 * (graph g's labels lie in [0, n_g)); infos is host lpa_run_info[G] or NULL
 * (non-NULL makes the call wait, as in lpa_run).  Each graph's info holds its
 * own iterations, exit_reason and changed[]; the scan counts (active[],
 * scanned[], edges_touched) are kept for the whole batch only and stay 0 in
 * the per-graph infos when G > 1 (lpa_batch_props_get reports the batch's
 * scanned_total). */
lpa_status lpa_batch_run(lpa_batch_t b, lpa_mode mode, double tolerance, int32_t max_iters,
                         int32_t *labels_out, void *stream, lpa_run_info *infos);

/* Degree-bin launch parameters of a batch (as lpa_graph_get_config /
 * lpa_graph_set_config). */
lpa_status lpa_batch_get_config(lpa_batch_t b, lpa_config *out);
lpa_status lpa_batch_set_config(lpa_batch_t b, const lpa_config *cfg);

/* lpa_autotune for a batch: the same search, each candidate timed on a
 * sample of the batch -- the shortest prefix of its graphs holding at least
 * sample_permille / 1000 of its entries (1..1000; 1000 = the whole batch),
 * run as a batch of its own that reads the parent's CSR in place (the graphs
 * of a batch are independent draws, so a prefix is a sample of them).  The
 * histogram and the cache key are the whole batch's. */
lpa_status lpa_batch_autotune(lpa_batch_t b, lpa_mode mode, double tolerance, int32_t max_iters, int32_t trials,
                              int32_t sample_permille, void *stream, lpa_config *chosen, lpa_autotune_info *info);

/* Modularity of graph g of the batch for LOCAL labels (device int32[n_g]). */
lpa_status lpa_batch_modularity(lpa_batch_t b, int32_t g, const int32_t *labels, double *q_out,
                                void *stream);

/* ---------------------------------------------------------------- serving */

/* Continuous batching of independent label propagation requests.  Small
 * requests share a device-resident arena that a worker thread advances one
 * sweep per cycle; a request joins at the next cycle after its copy to the
 * device and leaves when its own test (dN/N <= tolerance or max_iters sweeps,
 * Algorithm 1) is met.  Each request keeps its own counters, so in the
 * synchronous mode its labels are the same as a run on its own.  Requests
 * with at least solo_min_entries entries run on a separate lane (their own
 * graph and stream, one at a time).  Labels come back as host int32[n] in the
 * request's own vertex ids. */
typedef struct {
    int64_t hbm_budget_bytes;   /* device memory the server may hold: arena + solo-lane graphs */
    int64_t arena_vertices;     /* vertex capacity of the shared arena (>= 1) */
    int64_t arena_entries;      /* CSR entry capacity of the shared arena (>= 1) */
    int32_t max_slots;          /* requests in the arena at once (>= 2) */
    int32_t mode;               /* lpa_mode; LPA_MODE_SYNC_FULL is run as LPA_MODE_SYNC */
    double  tolerance;          /* in [0, 1] */
    int32_t max_iters;          /* in [0, 1 << 20] */
    int64_t solo_min_entries;   /* requests with at least this many entries use the solo lane; 0 = never */
} lpa_serve_config;

typedef struct {
    int64_t cycles;             /* arena cycles run so far */
    int32_t active;             /* requests in the arena now */
    int32_t pending;            /* requests copied or queued but not yet running */
    int64_t arena_bytes;        /* device memory held by the arena */
    int64_t solo_bytes;         /* device memory reserved by queued or running solo requests */
} lpa_serve_stats_t;

/* Allocates the arena on the current device and starts the worker threads. */
lpa_status lpa_serve_create(const lpa_serve_config *cfg, lpa_server_t *out);

/* Queues a request given as host CSR (same rules as lpa_graph_create).  Here
 * the host checks only offsets[0] == 0 and offsets[n] == nnz; an arena
 * request's rows, indices and weights are checked on the device while it is
 * admitted, and a request that fails is never run: its ticket is reported
 * by lpa_serve_poll like any other and lpa_serve_fetch returns
 * LPA_ERR_INVALID_GRAPH for it.  A solo-lane request is uploaded to device
 * memory here and validated by lpa_graph_create on the solo lane, a failure
 * likewise reported at fetch; the solo lane's streams have the lowest
 * priority, so the arena's cycles run first.  The data is copied (pageable
 * buffers) or read by DMA and waited for (page-locked buffers) before
 * returning, so the caller may reuse its buffers at once.  Returns
 * LPA_ERR_BUSY when it does not fit now (no free slot, vertex or entry range,
 * or device-memory budget); the caller may retry after results are released.
 * *ticket identifies the request. */
lpa_status lpa_serve_submit(lpa_server_t s, int64_t n, int64_t nnz, const int64_t *offsets,
                            const int32_t *indices, const float *weights, uint64_t *ticket);

/* Non-blocking: writes up to cap finished tickets (each reported once). */
lpa_status lpa_serve_poll(lpa_server_t s, uint64_t *done, int32_t cap, int32_t *n_done);

/* Copies a finished request's labels (host int32[n], nullable) and run info
 * (nullable).  An arena request's info holds iterations, exit_reason and
 * changed[]; its active[], scanned[] and edges_touched stay 0 (the arena
 * keeps no per-request scan counts).  A solo-lane request's
 * info is that of its lpa_run.  LPA_ERR_NOT_READY while it runs,
 * LPA_ERR_NOT_FOUND if unknown, the request's own error (e.g.
 * LPA_ERR_INVALID_GRAPH) if it failed. */
lpa_status lpa_serve_fetch(lpa_server_t s, uint64_t ticket, int32_t *labels_host, lpa_run_info *info);

/* Forgets a finished request's result. */
lpa_status lpa_serve_release(lpa_server_t s, uint64_t ticket);

/* Snapshot of the server's counters into a host struct; takes the server's
 * lock but never waits on the device.  LPA_ERR_INVALID_ARG if s or out is NULL. */
lpa_status lpa_serve_stats(lpa_server_t s, lpa_serve_stats_t *out);

/* Stops the workers (requests not finished are dropped) and frees the arena. */
lpa_status lpa_serve_destroy(lpa_server_t s);

#ifdef __cplusplus
}
#endif

#endif /* LPA_H_ */
