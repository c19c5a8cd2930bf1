/*
 * bbtc.h -- C ABI of the block-based triangle counting library (sm_103a).
 *
 * Method: Yasar, Rajamanickam, Berry & Catalyurek, "A Block-Based Triangle
 * Counting Algorithm on Heterogeneous Environments" (arXiv 2009.12457).
 *
 * The library counts the 3-cliques of a simple undirected graph (Sec. 2,
 * "Triangle Counting Problem") with the paper's pipeline, every step of which
 * runs in this library's own CUDA kernels on one GPU:
 *
 *   bbtc_graph_create : canonical simple edge set, degree, non-decreasing
 *                       degree order, orientation u < v (Sec. 2, Sec. 4.1)
 *   bbtc_count        : p x p symmetric partition and blocks G_ij (Sec. 2,
 *                       Sec. 4.1), task composition (Sec. 4.2, Alg. 4), task
 *                       estimate and order (Sec. 5), per-task counting by
 *                       bbTC-Intersect (Alg. 5) or bbTC-HMap (Alg. 6), and the
 *                       sum of the per-task counts (Alg. 9).
 *
 * Conventions for every entry point:
 *  - Every call returns a bbtc_status; no call aborts or traps. On an error,
 *    outputs are left untouched and bbtc_last_error() describes the cause.
 *  - Ids are int32 (n <= 2^31 - 1), edge offsets int64, counts uint64.
 *  - Pointers are HOST pointers unless a flag or field says otherwise.
 *  - A handle is not thread-safe; distinct handles may be used from distinct
 *    host threads.
 *  - Calls are synchronous with respect to the host: when a call returns, its
 *    outputs are written and the caller's input buffers are no longer read.
 */
#ifndef BBTC_H
#define BBTC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bbtc_graph *bbtc_graph_t; /* opaque; owns the device-resident oriented CSR */

typedef enum {
  BBTC_OK = 0,
  BBTC_EINVAL = 1,     /* invalid argument or malformed CSR */
  BBTC_ENOMEM = 2,     /* device or host allocation failed, or the budget is too small */
  BBTC_ECUDA = 3,      /* a CUDA runtime call failed */
  BBTC_ETIMEOUT = 4,   /* a bounded device wait ran out (opts.timeout_ms) */
  BBTC_ECANCELLED = 5, /* the request was cancelled before it ran */
  BBTC_EINTERNAL = 6   /* an internal consistency check failed */
} bbtc_status;

/* Per-task counting kernel (Sec. 4.3; the paper's isDense choice, Alg. 7). */
typedef enum {
  BBTC_KERNEL_AUTO = 0,      /* choose per staged list N(G_jk, v): bitmap when its value
                                range fits on chip, else hash table or sorted search by
                                its length (hash_threshold) */
  BBTC_KERNEL_INTERSECT = 1, /* bbTC-Intersect (Alg. 5): sorted-list search */
  BBTC_KERNEL_HASHMAP = 2    /* bbTC-HMap (Alg. 6): direct-address bitmap over the list's
                                value range when it fits on chip, else hash table */
} bbtc_kernel;

/* Symmetric partition of the degree order into p parts (Sec. 2 V^p, Sec. 4.1). */
typedef enum {
  BBTC_PARTITION_EDGES = 0, /* contiguous parts balanced on oriented edges:
                               c_i = min{ r : rowptr[r] >= ceil(i*m/p) } */
  BBTC_PARTITION_PROBE = 1  /* probe-based: bounds the largest block |G_ij| (Sec. 4.4's
                               m_max, hence lambda) by bisection on a bound B, each
                               probe closing part after part as late as its column's
                               blocks stay within B; parts end on one of
                               min(2048, 64p) grains balanced on undirected degree */
} bbtc_partition;

/* bbtc_graph_create flags */
#define BBTC_INPUT_DEVICE 0x1u    /* rowptr/colidx are DEVICE pointers on the current device */
#define BBTC_INPUT_SYMMETRIC 0x2u /* caller guarantees every edge is listed under both
                                     endpoints; only entries u < v are then read as edges */

typedef struct {
  uint32_t struct_size;         /* sizeof(bbtc_opts); set by bbtc_opts_init */
  int32_t p;                    /* blocks per side, 1 <= p <= 64; 0 = choose from the graph
                                   (resident: 1 below 65,536 edges, else 2; under a device
                                   budget: 2, 4 or 8 as m grows) */
  int32_t kernel;               /* bbtc_kernel */
  uint32_t timeout_ms;          /* 0 = no limit on the counting kernel's bounded waits */
  uint64_t device_budget_bytes; /* 0 = blocks resident; else the counting step keeps at most
                                   this many bytes of blocks on the device, streaming them
                                   from pinned host memory (the plan's block arrays move
                                   there; their pinned buffers are kept for reuse by later
                                   streamed plans, up to 64 GiB, until the process exits);
                                   preparation itself still uses device memory */
  uint64_t *per_vertex_out;     /* NULL, or n uint64 (ORIGINAL ids): triangles at each vertex */
  uint64_t *per_task_out;       /* NULL, or bbtc_num_tasks(p) uint64 in Alg. 4 order */
  void *stream;                 /* cudaStream_t to run on; NULL = the handle's own stream */
  uint32_t flags;               /* BBTC_OUT_DEVICE: the two output arrays are device pointers */
  int32_t hash_threshold;       /* AUTO: a staged list N(G_jk, v) whose value range is too
                                   wide for a bitmap is hashed when it is longer than this,
                                   else searched sorted; 0 = built-in default (16);
                                   at most 2^28 */
  uint64_t *per_graph_out;      /* NULL, or one uint64 per graph of a batch handle
                                   (bbtc_graph_create_batch / bbtc_count_batch) */
  int32_t chunk;                /* in-edges per work item of the counting kernel; 0 = auto */
  int32_t partition;            /* bbtc_partition; part of the plan's identity like p */
  uint64_t *per_task_cycles_out; /* NULL, or bbtc_num_tasks(p) uint64 in Alg. 4 order: SM
                                    clock cycles the counting kernel's warps spent on each
                                    task's work items (the measured side of the Sec. 5
                                    workload estimate) */
  uint32_t *per_edge_out;       /* NULL, or m uint32: the support of each oriented edge (the
                                   triangles that contain it; the input of k-truss, Sec. 1),
                                   in the order of bbtc_graph_get_oriented's colidx. Resident
                                   counts only (device_budget_bytes = 0) */
  const uint8_t *task_mask;     /* NULL, or bbtc_num_tasks(p) bytes (host), one per task in
                                   Alg. 4 order: only the tasks with a nonzero byte are
                                   counted, and the total (and the optional outputs) cover
                                   those tasks alone. The tasks are independent (Sec. 4.2),
                                   so ranks that count disjoint shares of them sum to the
                                   whole count (the multi-GPU form of Alg. 7 / Alg. 9).
                                   Read (copied to the device) during the call; the caller
                                   keeps it. bbtc_count, resident or budgeted, only:
                                   bbtc_count_batch ignores it, bbtc_count_async refuses it */
} bbtc_opts;

#define BBTC_OUT_DEVICE 0x1u

/* Fill *opts with defaults (p = 0, AUTO kernel, resident, no optional outputs). */
void bbtc_opts_init(bbtc_opts *opts);

/*
 * Copy an undirected graph into a new handle and run the graph-only steps of
 * the method: drop self-loops and duplicate entries (Sec. 2 assumes a simple
 * graph), compute degrees, order vertices by (degree, id) ascending (Sec. 4.1;
 * ties by original id), and orient every edge from the lower to the higher
 * position (Sec. 2: N(G,u) = {v : (u,v) in E, u < v}).
 *
 *   n       number of vertices, 0 <= n <= 2^31 - 1
 *   rowptr  n+1 int64 offsets, rowptr[0] = 0, non-decreasing
 *   colidx  rowptr[n] int32 neighbour ids in [0, n); an edge may be listed
 *           under one or both endpoints, in any order, repeated, and
 *           self-loops are allowed (all are ignored beyond the simple graph)
 *   flags   BBTC_INPUT_DEVICE and/or BBTC_INPUT_SYMMETRIC
 *   out     receives the handle
 *
 * Ownership: the caller keeps rowptr/colidx (they are only read during the
 * call). The handle owns its device memory until bbtc_graph_destroy.
 * Errors: EINVAL for n out of range, NULL pointers with edges present,
 * rowptr[0] != 0, a decreasing rowptr, or any colidx outside [0, n), or more
 * than 2^32 - 1 simple edges; ENOMEM; ECUDA.
 */
bbtc_status bbtc_graph_create(int64_t n, const int64_t *rowptr, const int32_t *colidx,
                              uint32_t flags, bbtc_graph_t *out);

/* As bbtc_graph_create, but run on `stream` (a cudaStream_t; NULL = a new
 * stream owned by the handle). The handle keeps using `stream` by default. */
bbtc_status bbtc_graph_create_async(int64_t n, const int64_t *rowptr, const int32_t *colidx,
                                    uint32_t flags, void *stream, bbtc_graph_t *out);

/*
 * One handle for a batch of ng independent graphs, prepared together as their
 * disjoint union (one canonicalisation, order and orientation pass). Graph g
 * owns the union's vertices [vertex_offsets[g], vertex_offsets[g+1]). Within
 * a graph the degree order and the orientation are the same as for the graph
 * alone (ties by id keep each graph's own order), no triangle spans two
 * graphs, and bbtc_count with opts.per_graph_out returns every graph's exact
 * count from one counting launch over the union.
 *
 *   ng              number of graphs, >= 1
 *   vertex_offsets  ng+1 HOST int64: 0 = offsets[0] <= ... <= offsets[ng] = N
 *   rowptr          N+1 int64 offsets of the union's rows (host, or device
 *                   with BBTC_INPUT_DEVICE)
 *   colidx          rowptr[N] int32 neighbour ids LOCAL to the row's graph:
 *                   an entry of a row of graph g lies in [0, n_g)
 *
 * Errors: as bbtc_graph_create, plus EINVAL for decreasing offsets or an
 * entry outside its graph.
 */
bbtc_status bbtc_graph_create_batch(int32_t ng, const int64_t *vertex_offsets,
                                    const int64_t *rowptr, const int32_t *colidx, uint32_t flags,
                                    void *stream, bbtc_graph_t *out);

/*
 * Count the triangles of the handle's graph with bbTC at p x p blocks:
 * contiguous symmetric partition of the degree order (opts->partition:
 * balanced on oriented edges, or probe-based to bound the largest block),
 * tasks (i,j,k), i <= j <= k (Alg. 4), ordered by the Sec. 5 estimate
 * and drained by a persistent work-stealing kernel, each task counted as
 * sum over (u,v) in G_ij of |N(G_ik,u) ∩ N(G_jk,v)| (Alg. 5 / Alg. 6).
 *
 *   count  receives the exact total (host uint64)
 *   opts   NULL = defaults; see bbtc_opts for the optional outputs
 *
 * Errors: EINVAL (p outside 0..64, an unknown kernel or partition,
 * opts->struct_size too small), ENOMEM
 * (also when device_budget_bytes cannot hold one task's blocks), ETIMEOUT,
 * ECUDA.
 */
bbtc_status bbtc_count(bbtc_graph_t g, const bbtc_opts *opts, uint64_t *count);

/*
 * Build the resident plan of the handle for opts' p (0 = automatic), kernel,
 * hash_threshold, chunk and partition -- partition, blocks, tasks, estimates and work
 * items (Sec. 2, Sec. 4.1-4.2, Sec. 5) -- without counting; keep it when it
 * already matches. Later counts with the same options only read the plan.
 * Other options are ignored. Synchronous.
 * Errors: EINVAL (NULL handle, bad options); ENOMEM; ECUDA.
 */
bbtc_status bbtc_graph_plan(bbtc_graph_t g, const bbtc_opts *opts);

/*
 * Count ng independent handles in one persistent launch (Sec. 4.2 tasks of
 * all of them drained together).
 *
 * Resident (device_budget_bytes = 0): each handle keeps its own plan for
 * (p, kernel, hash_threshold, chunk, partition) -- built first, on the handle, when it
 * does not match -- and one counting launch takes the work items of all the
 * handles, largest handles first. p = 0 picks p per handle from its size.
 * Handles that already hold a matching resident plan are only read, so
 * concurrent calls on other streams may share them.
 * Under a device budget: the handles' oriented CSRs are gathered into one
 * union (positions offset per handle), planned once and counted with its
 * blocks streamed; p = 0 picks p from the union's size.
 *
 *   gs         ng handles (NULL entries are reported, the rest still counted)
 *   counts     receives ng uint64 totals (host)
 *   per_graph  NULL, or receives each handle's status
 *
 * Options other than p, kernel, hash_threshold, chunk, partition, timeout_ms,
 * stream and device_budget_bytes are ignored (no per-task, per-vertex or per-graph
 * outputs).
 * Errors: EINVAL for ng < 0, a NULL handle (its status is EINVAL and the
 * others are still counted) or handles on different devices; ENOMEM;
 * ETIMEOUT; ECUDA.
 */
bbtc_status bbtc_count_batch(const bbtc_graph_t *gs, int32_t ng, const bbtc_opts *opts,
                             uint64_t *counts, bbtc_status *per_graph);

/*
 * Allocation-free count. The paper has no counterpart to this entry point: it
 * exists for callers that cannot allocate device memory at the moment they
 * count. Examples are a serving loop that reserves all of its GPU memory at
 * start-up and forbids later allocations, code running while another memory
 * manager (a framework's caching allocator) owns the free device memory, and
 * hooks invoked from inside an allocator, where cudaMalloc would re-enter it.
 *
 * It runs the same counting kernel as bbtc_count on the plan that an earlier
 * bbtc_count or bbtc_graph_get_plan call built for the same p on this handle.
 * Its scratch (work-stealing counter, status, per-task accumulators) is a
 * fixed 8 KiB device array inside the library, which every GPU that loads the
 * library holds until the process exits. The call makes no cudaMalloc,
 * cudaMallocAsync, cudaFree or other allocating call.
 *
 *   p             1..16: the fixed array holds at most 816 task counters
 *   count_dev     DEVICE pointer to one uint64: the total
 *   per_task_dev  NULL, or DEVICE pointer to bbtc_num_tasks(p) uint64, in the same task
 *                 order as bbtc_count's per_task_out
 *   stream        cudaStream_t (NULL = the handle's stream); the call is
 *                 asynchronous: outputs are ready when the stream reaches them
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current, guarded so that concurrent first calls
 * from several host threads are safe); make that first call before any stream
 * capture. A failed look-up is remembered and every later call on that device
 * returns ECUDA. Every call shares the one array and it keeps the last call's
 * contents: each call clears what it needs, but calls whose work overlaps on
 * the GPU (other streams, other host threads) race on it and must be ordered
 * by the caller.
 * Errors: EINVAL for a NULL handle or count_dev, p outside 1..16, or no plan
 * for p on the handle; ECUDA.
 */
bbtc_status bbtc_count_noalloc(bbtc_graph_t g, int32_t p, uint64_t *count_dev,
                               uint64_t *per_task_dev, void *stream);

/*
 * Enqueue a count on opts->stream (NULL = the handle's stream) without
 * allocating and without waiting: the plan for (p, kernel, hash_threshold,
 * chunk, partition) must already exist on the handle (built by bbtc_count or
 * bbtc_graph_get_plan), and every output is a DEVICE pointer: total_dev (one
 * uint64), opts->per_task_out and opts->per_graph_out (nullable;
 * opts->flags must include BBTC_OUT_DEVICE when they are set);
 * opts->per_vertex_out and opts->task_mask must be NULL. Because it only enqueues kernels and
 * copies on one stream, the call can be captured into a CUDA graph and
 * replayed. The handle's plan scratch is shared by its calls: calls on one
 * handle must not overlap on the GPU. opts->timeout_ms is ignored.
 * Errors: EINVAL when no plan matches or an output is not allowed; ECUDA.
 */
bbtc_status bbtc_count_async(bbtc_graph_t g, const bbtc_opts *opts, uint64_t *total_dev);

/* Free the handle and its device memory. Accepts NULL. */
void bbtc_graph_destroy(bbtc_graph_t g);

/* Message of the calling thread's most recent error ("" if none). */
const char *bbtc_last_error(void);

/* Number of tasks for p parts: p(p+1)(p+2)/6 (Sec. 4.2). 0 for p < 1. */
uint64_t bbtc_num_tasks(int32_t p);

/* ------------------------------------------------------------ inspection */

typedef struct {
  int64_t n;             /* vertices */
  int64_t m;             /* simple undirected edges (= oriented edges) */
  int64_t dplus_max;     /* largest out-degree after orientation */
  int64_t deg_max;       /* largest undirected degree */
  uint64_t device_bytes; /* device memory held by the handle */
  uint64_t wedges_in;    /* sum over oriented edges (u,v) of d+(v) */
  uint64_t wedges_out;   /* sum over vertices u of d+(u)(d+(u)-1)/2 */
  int64_t num_graphs;    /* graphs in the handle (1 unless built as a batch) */
} bbtc_graph_info;

/* Sizes and work figures of the handle's graph (the two wedge sums are
 * computed on the device at the first call). */
bbtc_status bbtc_graph_get_info(bbtc_graph_t g, bbtc_graph_info *info);

/* Device time of the handle's most recent steps, measured with CUDA events
 * on the stream each step ran on. */
typedef struct {
  double prep_ms;      /* bbtc_graph_create: a1-a4 (after any host-to-device copy) */
  double plan_ms;      /* last bbtc_count: a5-a8 (0 when the plan was reused) */
  double count_ms;     /* last bbtc_count: the counting kernel (a9); with a device
                          budget, the whole streamed count (copies included) */
  int64_t work_items;  /* work items drained by that kernel */
  int64_t stream_rounds;      /* last budgeted count: rounds of block copies */
  uint64_t stream_h2d_bytes;  /* last budgeted count: block bytes copied to the device */
  double stream_copy_ms;      /* last budgeted count: device time of those copies */
  uint64_t stream_block_bytes;  /* last budgeted count: bytes of all the plan's streamed
                                   blocks (each block once) */
  uint64_t stream_device_peak_bytes; /* last budgeted count: high-water mark of the library's
                                        device memory during the count (the handle's
                                        oriented CSR and plan tables, which stay resident,
                                        plus the block pool of at most the budget); the
                                        library's idle cached blocks are released before
                                        a budgeted count */
  int32_t stream_mode;        /* last budgeted count: 1 = every block CSR kept on the device
                                 and each in-edge block copied once; 2 = blocks placed round
                                 by round in the pool and re-copied when evicted */
} bbtc_timings;

bbtc_status bbtc_graph_get_timings(bbtc_graph_t g, bbtc_timings *t);

/*
 * Device memory the library can still use on `device` (an ordinal): the free
 * bytes the driver reports, plus the bytes that the device's stream-ordered
 * pool holds without using them, plus the library's idle cached blocks (the
 * library allocates from that pool, keeps freed blocks of 64 MB and more for
 * later calls of a similar size, and releases them when an allocation fails,
 * so the driver's figure alone undercounts). pool_used excludes the idle
 * cached blocks. Any output may be NULL. Used by callers that admit work by
 * free device memory, such as the serving loop; the paper has no counterpart.
 * Errors: EINVAL for an unknown device; ECUDA.
 */
bbtc_status bbtc_device_memory(int32_t device, uint64_t *available, uint64_t *total,
                               uint64_t *pool_reserved, uint64_t *pool_used);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t bbtc_kernel_launches(void);

/*
 * Copy the oriented CSR to host arrays (any may be NULL to skip it):
 * rowptr n+1 int64 and colidx m int32 in degree-order positions (rows sorted
 * ascending), perm n int32 (perm[r] = original id at position r), degree n
 * int64 (undirected simple degree by ORIGINAL id).
 */
bbtc_status bbtc_graph_get_oriented(bbtc_graph_t g, int64_t *rowptr, int32_t *colidx,
                                    int32_t *perm, int64_t *degree);

/*
 * The plan bbtc_count builds for p (Sec. 2, Sec. 4.2, Sec. 5), as host copies
 * (any output may be NULL); the handle's current plan when it has this p
 * (whatever its partition), else a new one with the edge-balanced partition: cuts p+1 int32 (c_0 = 0, c_p = n), block_nnz p*p
 * int64 (|G_ij|, row-major), tasks 3*|T| int32 ((i,j,k) in Alg. 4 order),
 * estimate |T| double (ExecTime in Alg. 4 order), order |T| int32 (task
 * indices, non-increasing estimate, ties in Alg. 4 order).
 */
bbtc_status bbtc_graph_get_plan(bbtc_graph_t g, int32_t p, int32_t *cuts, int64_t *block_nnz,
                                int32_t *tasks, double *estimate, int32_t *order);

#ifdef __cplusplus
}
#endif

#endif /* BBTC_H */
