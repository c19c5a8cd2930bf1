// graph.cuh -- the graph handle and the per-p plan it caches.
#pragma once

#include "common.cuh"

namespace bbtc {

// Entries allocated for a column array of m entries: the counting kernel reads
// columns as aligned groups of four, up to three entries past a list's end, so
// every column array is padded to a multiple of four entries and one group
// more (the extra entries are never counted).
inline int64_t padded_columns(int64_t m) { return ((m + 3) & ~int64_t(3)) + 4; }

// One in-edge of block G_ab (a = part(u), b = part(v)), 16 bytes: source u,
// destination v, the position e of (u, v) among the columns, and the end f of
// u's run in block G_ab (one past its last column), so that for the diagonal
// tasks (i, j, j) the probe run of (u, v) is [e + 1, f) with no lookup.
// Positions are uint32 stored in int32 fields.
using InEdge = int4;

// Where the counting kernel finds the three blocks of task t = (i, j, k):
//  - the in-edges of G_ij, grouped by v: element x of the task's range lives
//    at ie[x - ie_off];
//  - N(G_ik, u) for u in V_i: columns [rp_ik[r * rs_ik], rp_ik[r * rs_ik + 1])
//    with r = u - c_i, of ci_ik, where column position q lives at
//    ci_ik[q - ci_ik_off];
//  - N(G_jk, v) for v in V_j: likewise through rp_jk / rs_jk / ci_jk.
// Resident plans point into the oriented CSR itself: rp is the split table
// (row r of part a holds the CSR positions where its runs in blocks a..p-1
// start, then its end; rs = p - a + 1). Streamed plans point at physical
// per-block copies (rs = 1). For k == j, G_ik is G_ij and the in-edge
// position indexes it directly.
struct TaskDesc {
  const InEdge *ie;
  int64_t ie_off;
  const uint32_t *rp_ik;
  const int32_t *ci_ik;
  int64_t ci_ik_off;
  const uint32_t *rp_jk;
  const int32_t *ci_jk;
  int64_t ci_jk_off;
  int32_t rs_ik, rs_jk;
  int32_t c_i, c_j;
  int32_t diag;  // k == j
  int32_t task;  // index in Alg. 4 order
};

// One unit of counting work: the in-edges [x0, x1) of block G_ij (grouped by
// destination v) for task t = (i, j, k).
struct WorkItem {
  int32_t task;
  int32_t flags;  // bits 0-1: 0 INTERSECT, 1 HASHMAP, 2 AUTO; bits 2..: AUTO hash threshold
  int64_t x0, x1;
};

// Everything bbtc_count builds for one p (Sec. 2 partition, Sec. 4.2 tasks,
// Sec. 5 estimate and order), cached on the handle until p changes.
struct Plan {
  int p = 0;
  int64_t ntasks = 0;
  int32_t *cuts = nullptr;      // p+1
  int32_t h_cuts[65] = {0};     // host copy of the cuts
  // blocks G_ab of the resident plan, read in place from the oriented CSR
  // (Sec. 4.1, the blocks of a row are consecutive runs of its sorted list):
  // spl[h_spl_off[a] + r * (p - a + 1) + (b - a)] = CSR position where row
  // c_a + r enters block b (b = p: the row's end)
  uint32_t *spl = nullptr;
  int64_t h_spl_off[65] = {0};
  // physical block CSR (streamed plans only): blocks (a, b), a <= b, in
  // row-major order; block (a, b)'s row pointers are rp[rpb[a*p+b] .. + |V_a|]
  // and hold positions in ci, the block-major concatenation of all blocks'
  // columns; in-edge positions then index ci
  uint32_t *rp = nullptr;
  int32_t *ci = nullptr;
  int64_t h_rpb[64 * 64] = {0};
  int64_t total_rp = 0;
  TaskDesc *desc = nullptr;     // T, in Alg. 4 order
  InEdge *ie = nullptr;         // m: in-edges grouped by (part(u), v)
  int64_t *boff = nullptr;      // p*(p+1): block (i,j) in-edges = [boff[i*(p+1)+j], +1)
  int32_t *tasks = nullptr;     // 3*T: (i,j,k) in Alg. 4 order
  double *est = nullptr;        // T: ExecTime in Alg. 4 order
  int32_t *order = nullptr;     // T: task indices by non-increasing estimate
  int64_t nitems = 0;
  WorkItem *items = nullptr;    // work items, heaviest task first
  int32_t kernel_mode = -1;     // bbtc_kernel the items were built for
  int32_t hash_threshold = 0;
  int32_t chunk_req = 0;        // requested in-edges per item (0 = automatic)
  int32_t partition = 0;        // bbtc_partition the cuts were built with
  int64_t bstar = -1;           // probe-based partition: the bound B* on every block
  int64_t chunk = 0;            // in-edges per item used
  // counting scratch owned by the plan: [0] work-stealing head, [1] status,
  // [2] total, [3, 3+T) per-task counts, [3+T, 3+T+ng) per-graph counts
  unsigned long long *scratch = nullptr;
  int blocks_per_sm[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // occupancy of each counting-kernel mode
  // streamed mode: the block arrays live in pinned host memory instead
  bool streamed = false;
  uint32_t *h_rp = nullptr;
  int32_t *h_ci = nullptr;
  InEdge *h_ie = nullptr;
  uint64_t bytes = 0;
};

constexpr int SCR_HEAD = 0, SCR_STATUS = 1, SCR_TOTAL = 2, SCR_TASKS = 3;

}  // namespace bbtc

struct StreamStatsLite {
  int64_t rounds = 0;
  uint64_t h2d_bytes = 0;
  double copy_ms = 0;
  uint64_t block_bytes = 0;
  uint64_t device_peak = 0;
  int32_t mode = 0;
};

struct bbtc_graph {
  int64_t n = 0;
  int64_t m = 0;
  int nb = 1;                  // bits per vertex id: 2^nb >= n
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t *rowptr = nullptr;   // oriented CSR (degree-order positions), n+1
  int32_t *colidx = nullptr;   // m, rows sorted ascending
  int32_t *esrc = nullptr;     // m, source position of each oriented edge
  int32_t *perm = nullptr;     // n, perm[r] = original id at position r
  int32_t *deg = nullptr;      // n, undirected simple degree by original id
  int64_t dplus_max = 0;
  int64_t deg_max = 0;
  int32_t ng = 1;              // graphs in the handle (a batch is their disjoint union)
  int64_t *voff = nullptr;     // device, ng+1 vertex offsets (batch handles only)
  int32_t *gid = nullptr;      // device, n: graph of each position (batch handles only)
  uint64_t bytes = 0;
  bbtc::Plan plan;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  bool plan_timed = false;
  StreamStatsLite stream_stats;
  double stream_stats_total_ms = -1.0;  // >= 0 when the last count was streamed
  bool wedges_known = false;
  uint64_t wedges_in = 0, wedges_out = 0;
};

namespace bbtc {

// a1-a4: build g's oriented CSR from an input CSR already on the device.
// For a batch handle (g->ng > 1, g->voff set), colidx holds ids local to each
// row's graph; they are offset into the union and g->gid is filled.
bbtc_status prepare_graph(bbtc_graph *g, const int64_t *d_rowptr, const int32_t *d_colidx,
                          int64_t nnz, bool symmetric);

// a5-a8: partition, blocks, tasks, estimate, order and work items for p.
// partition: 0 = contiguous parts balanced on oriented edges, 1 = probe-based
// (bounds the largest block).
bbtc_status build_plan(bbtc_graph *g, int p, int kernel_mode, int hash_threshold, int chunk,
                       cudaStream_t s, int partition = 0);
inline bool plan_matches(const Plan &pl, int p, int kernel_mode, int hash_threshold, int chunk,
                         int partition = 0) {
  return pl.p == p && pl.kernel_mode == kernel_mode && pl.hash_threshold == hash_threshold &&
         pl.chunk_req == chunk && pl.partition == partition;
}

// a5, probe-based: cuts (device, p+1) of the partition that bounds the largest
// block load by B* (returned on the host). Synchronises s.
bbtc_status pbd_partition(const bbtc_graph *g, int p, int32_t *d_cuts, int64_t *h_bstar,
                          cudaStream_t s);
void free_plan(Plan *pl, cudaStream_t s);
void free_plan_host(Plan *pl);  // pinned host copies of a streamed plan

// Occupancy of the counting kernel (set at plan time so that a count only
// enqueues work).
bbtc_status configure_count_kernels(Plan *pl);

// a9-a10: per-task counts (plan scratch, Alg. 4 order), optional per-vertex
// counts by position (vertex_count, device, n), per-graph counts (plan
// scratch) and per-edge support by column position (edge_sup, device, m,
// zeroed by the caller; resident plans index the oriented CSR, so this is the
// order of g->colidx); the total goes to the plan scratch. Enqueues only.
bbtc_status run_count(bbtc_graph *g, const Plan &pl, unsigned long long *vertex_count,
                      bool per_graph, uint32_t timeout_ms, cudaStream_t s,
                      cudaEvent_t ev_begin, cudaEvent_t ev_end,
                      unsigned long long *task_cycles = nullptr, unsigned *edge_sup = nullptr,
                      const uint8_t *task_mask = nullptr);
// The three parts of run_count: zero the outputs, drain items [item0,
// item0 + nitems) in one persistent launch (accumulating), sum the tasks.
bbtc_status count_reset(bbtc_graph *g, const Plan &pl, unsigned long long *vertex_count,
                        bool per_graph, cudaStream_t s);
// task_mask (device, nullable): one byte per task; items of tasks whose byte is
// zero are skipped.
bbtc_status count_launch(bbtc_graph *g, const Plan &pl, int64_t item0, int64_t nitems,
                         unsigned long long *vertex_count, bool per_graph, uint32_t timeout_ms,
                         cudaStream_t s, unsigned long long *task_cycles = nullptr,
                         unsigned *edge_sup = nullptr, const uint8_t *task_mask = nullptr);
bbtc_status count_finish(const Plan &pl, cudaStream_t s);
// The error of a nonzero status word left by the counting kernel: 1 = it
// passed opts.timeout_ms (ETIMEOUT), 2 = a bulk copy wait ran out (EINTERNAL).
bbtc_status count_status_error(const char *where, int32_t status, uint32_t timeout_ms);

// Counts the handles gs[0, ng) (each holding a resident plan) in one
// persistent launch over all their work items; counts[i] is gs[i]'s total.
// Reads the plans only. Synchronises s.
bbtc_status count_plans(bbtc_graph *const *gs, int32_t ng, uint32_t timeout_ms, cudaStream_t s,
                        uint64_t *counts);

// Physical per-block copies of a resident plan's blocks (pl.rp, pl.ci,
// pl.h_rpb), with the in-edge positions re-pointed at them; the step before a
// plan streams. Frees the split table.
bbtc_status plan_physical_blocks(const bbtc_graph *g, Plan &pl, cudaStream_t s);

// a11: count with the blocks streamed from pinned host memory through a
// device pool of `budget` bytes (two halves, double-buffered).
struct StreamStats {
  int64_t rounds = 0;
  uint64_t h2d_bytes = 0;
  double copy_ms = 0, count_ms = 0, total_ms = 0;
  uint64_t block_bytes = 0;  // every streamed block once
  uint64_t device_peak = 0;  // pool high-water mark during the count
  int32_t mode = 0;          // 1: block CSRs resident, in-edge blocks once; 2: general
};
bbtc_status run_count_streamed(bbtc_graph *g, Plan &pl, uint64_t budget,
                               unsigned long long *vertex_count, bool per_graph,
                               uint32_t timeout_ms, cudaStream_t s, StreamStats *stats,
                               unsigned long long *task_cycles = nullptr,
                               const uint8_t *task_mask = nullptr);

// Work figures of the oriented graph (device): sum_{(u,v)} d+(v) and
// sum_u d+(u)(d+(u)-1)/2.
bbtc_status wedge_sums(const bbtc_graph *g, uint64_t *in_sum, uint64_t *out_sum,
                       cudaStream_t s);

// Gathers handles into one union handle (positions of handle h offset by the
// vertices of the handles before it, graph-of-position filled); used by
// bbtc_count_batch. The caller destroys the union.
bbtc_status union_of(const bbtc_graph_t *gs, int32_t ng, cudaStream_t s, bbtc_graph **out);

// Default p when the caller passes 0: small for resident counts, growing with
// m when blocks stream under a device budget.
int default_p(const bbtc_graph *g, bool budgeted = false);

}  // namespace bbtc
