/*
 * bbtc_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of block-based triangle
 * counting (bbTC, Yasar, Rajamanickam, Berry & Catalyurek, arXiv 2009.12457).
 * Only the test suite, the package smoke check and the benchmark's CPU
 * baseline leg may call this file; the CUDA library shares no code with it.
 *
 * Every quantity is an integer except the task-order estimate (Sec. 5), which
 * is only used to order work. Steps follow the paper's order:
 *
 *   canonical simple edge set  (Sec. 2: simple undirected G=(V,E), (u,v) with u<v)
 *   degree                     (Sec. 2, Sec. 4.1)
 *   order by degree            (Sec. 4.1: non-decreasing degree order)
 *   orientation                (Sec. 2: N(G,u) = {v : (u,v) in E, u < v})
 *   partition / cuts           (Sec. 2 vertex partition V^p; Sec. 4.1)
 *   probe-based partition      (Sec. 4.1 symmetric rectilinear partition, Sec. 4.4 lambda)
 *   block sizes |G_ij|         (Sec. 2 G_ij; Sec. 4.4 lambda)
 *   task composition           (Sec. 4.2, Alg. 4)
 *   task estimate + order      (Sec. 5, ExecTime)
 *   per-task count             (Sec. 4.3, Alg. 5 bbTC-Intersect, Alg. 6 bbTC-HMap)
 *   whole-graph count          (Sec. 3, Alg. 2 TC-Intersect with Alg. 1, Alg. 3 TC-HMap)
 *   per-vertex and per-edge    (Alg. 9's per-vertex counts; edge support for k-truss, Sec. 1)
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *  - Alg. 1 compares A[b] = B[b] in its first branch; the intended test is
 *    A[a] = B[b] (the algorithm counts common elements of two sorted lists).
 *  - The degree used for ordering is the undirected simple-graph degree.
 *  - Ties in degree are broken by the original vertex id, ascending.
 *  - Edges point from the lower to the higher position in the degree order.
 *  - The partition is contiguous in that order: c_0 = 0, c_p = n and, for
 *    0 < i < p, c_i = min{ r : rowptr[r] >= ceil(i*m/p) } on the oriented CSR.
 *  - Alg. 3 / Alg. 6 leave H's initial value unstated; here it is -1.
 *  - ExecTime(t) = |G_ij| * max(delta(G_ik), delta(G_jk)), delta(G_ab) =
 *    |G_ab| / |V_a| (0 when V_a is empty); ties keep Alg. 4's order.
 *
 * Parity pins (tests, not this file): brute force over all vertex triples,
 * trace(A^3)/6, closed forms (K_n, wheels, friendship, complete tripartite,
 * bipartite/grid/tree = 0), sum of per-vertex counts = 3T, the task count
 * p(p+1)(p+2)/6 against the paper's tiles/tasks table, and agreement of the
 * two whole-graph and the two per-task algorithms.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- helpers */

static int cmp_u64(const void *x, const void *y) {
  uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
  return (a > b) - (a < b);
}

/* first index in [lo, hi) of sorted list L whose value is >= x */
static int64_t lower_bound_i32(const int32_t *L, int64_t lo, int64_t hi, int64_t x) {
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if ((int64_t)L[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

/* ------------------------------------------------ canonical simple edges */

/*
 * Sec. 2 treats G as a simple undirected graph and writes each edge (u,v) with
 * u < v. Input: any CSR listing an edge in one or both directions, possibly
 * with duplicates and self-loops. Output: the sorted set of keys
 * (min << 32) | max over entries with endpoints that differ. keys_out must hold
 * rowptr[n] entries. Returns m, the number of simple undirected edges.
 */
int64_t orc_canonical_edges(int64_t n, const int64_t *rowptr, const int32_t *colidx,
                            uint64_t *keys_out) {
  int64_t cnt = 0;
  for (int64_t u = 0; u < n; ++u) {
    for (int64_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
      int64_t v = colidx[e];
      if (v == u) continue;
      uint64_t a = (uint64_t)(u < v ? u : v), b = (uint64_t)(u < v ? v : u);
      keys_out[cnt++] = (a << 32) | b;
    }
  }
  qsort(keys_out, (size_t)cnt, sizeof(uint64_t), cmp_u64);
  int64_t m = 0;
  for (int64_t i = 0; i < cnt; ++i)
    if (i == 0 || keys_out[i] != keys_out[i - 1]) keys_out[m++] = keys_out[i];
  return m;
}

/* Undirected simple degree of every vertex (reading of the ordering degree). */
void orc_degree(int64_t n, int64_t m, const uint64_t *keys, int64_t *deg) {
  memset(deg, 0, sizeof(int64_t) * (size_t)n);
  for (int64_t e = 0; e < m; ++e) {
    deg[keys[e] >> 32] += 1;
    deg[keys[e] & 0xFFFFFFFFULL] += 1;
  }
}

/* ------------------------------------------------------- order by degree */

static const int64_t *g_sort_deg; /* comparator context (single-threaded) */

static int cmp_by_degree(const void *x, const void *y) {
  int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
  if (g_sort_deg[a] != g_sort_deg[b]) return g_sort_deg[a] < g_sort_deg[b] ? -1 : 1;
  return (a > b) - (a < b);
}

/*
 * Sec. 4.1: vertices re-ordered in non-decreasing degree order. perm[r] is the
 * original id at position r; rank[v] is the position of original vertex v.
 */
void orc_order_by_degree(int64_t n, const int64_t *deg, int32_t *rank, int32_t *perm) {
  for (int64_t v = 0; v < n; ++v) perm[v] = (int32_t)v;
  g_sort_deg = deg;
  qsort(perm, (size_t)n, sizeof(int32_t), cmp_by_degree);
  g_sort_deg = NULL;
  for (int64_t r = 0; r < n; ++r) rank[perm[r]] = (int32_t)r;
}

/* ------------------------------------------------------------ orientation */

/*
 * Sec. 2: with vertices named by their position in the order, each edge is
 * stored once as (u,v) with u < v and N(G,u) = {v : (u,v) in E, u < v}.
 * Output: oriented CSR in position space, each row sorted ascending.
 * rowptr_out has n+1 entries, colidx_out m.
 */
void orc_orient(int64_t n, int64_t m, const uint64_t *keys, const int32_t *rank,
                int64_t *rowptr_out, int32_t *colidx_out) {
  uint64_t *ok = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
  for (int64_t e = 0; e < m; ++e) {
    uint64_t ra = (uint64_t)rank[keys[e] >> 32];
    uint64_t rb = (uint64_t)rank[keys[e] & 0xFFFFFFFFULL];
    ok[e] = ra < rb ? (ra << 32) | rb : (rb << 32) | ra;
  }
  qsort(ok, (size_t)m, sizeof(uint64_t), cmp_u64);
  memset(rowptr_out, 0, sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t e = 0; e < m; ++e) rowptr_out[(ok[e] >> 32) + 1] += 1;
  for (int64_t u = 0; u < n; ++u) rowptr_out[u + 1] += rowptr_out[u];
  for (int64_t e = 0; e < m; ++e) colidx_out[e] = (int32_t)(ok[e] & 0xFFFFFFFFULL);
  free(ok);
}

/* --------------------------------------------- whole-graph counts (Sec. 3) */

/* Alg. 1 (nIntersect), with the first comparison read as A[a] = B[b]. */
uint64_t orc_n_intersect(const int32_t *A, int64_t na, const int32_t *B, int64_t nb) {
  int64_t a = 0, b = 0;
  uint64_t c = 0;
  while (a < na && b < nb) {
    if (A[a] == B[b]) { ++c; ++a; ++b; }
    else if (A[a] < B[b]) ++a;
    else ++b;
  }
  return c;
}

/* Alg. 2 (TC-Intersect) over the oriented CSR. */
uint64_t orc_tc_intersect(int64_t n, const int64_t *rp, const int32_t *ci) {
  uint64_t tau = 0;
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
      int64_t v = ci[e];
      tau += orc_n_intersect(ci + rp[u], rp[u + 1] - rp[u], ci + rp[v], rp[v + 1] - rp[v]);
    }
  return tau;
}

/* Alg. 3 (TC-HMap) over the oriented CSR; H starts at -1 for every vertex. */
uint64_t orc_tc_hmap(int64_t n, const int64_t *rp, const int32_t *ci) {
  int64_t *H = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t v = 0; v < n; ++v) H[v] = -1;
  uint64_t tau = 0;
  for (int64_t u = 0; u < n; ++u) {
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) H[ci[e]] = u;
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
      int64_t v = ci[e];
      for (int64_t f = rp[v]; f < rp[v + 1]; ++f)
        if (H[ci[f]] == u) ++tau;
    }
  }
  free(H);
  return tau;
}

/*
 * Per-vertex triangle counts in ORIGINAL ids: every triangle found by Alg. 2's
 * loops adds one to each of its three corners. perm maps positions to ids.
 */
void orc_per_vertex(int64_t n, const int64_t *rp, const int32_t *ci, const int32_t *perm,
                    uint64_t *cnt_out) {
  memset(cnt_out, 0, sizeof(uint64_t) * (size_t)n);
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
      int64_t v = ci[e];
      int64_t a = rp[u], b = rp[v];
      while (a < rp[u + 1] && b < rp[v + 1]) {
        if (ci[a] == ci[b]) {
          cnt_out[perm[u]] += 1; cnt_out[perm[v]] += 1; cnt_out[perm[ci[a]]] += 1;
          ++a; ++b;
        } else if (ci[a] < ci[b]) ++a;
        else ++b;
      }
    }
}

/*
 * Edge support: for every oriented edge (u,v) at position e of the oriented
 * CSR, the number of triangles that contain it. The paper names k-truss
 * decomposition among the consumers of triangle counts (Sec. 1); an edge's
 * support is its input. Each triangle u < v < w found by merging N(u) and
 * N(v) adds one to (u,v), to (u,w) and to (v,w); the merge visits w at its
 * position in both rows, so all three positions are known.
 */
void orc_edge_support(int64_t n, const int64_t *rp, const int32_t *ci, uint32_t *sup_out) {
  memset(sup_out, 0, sizeof(uint32_t) * (size_t)(rp[n] > 0 ? rp[n] : 1));
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
      int64_t v = ci[e];
      int64_t a = rp[u], b = rp[v];
      while (a < rp[u + 1] && b < rp[v + 1]) {
        if (ci[a] == ci[b]) {
          sup_out[e] += 1; sup_out[a] += 1; sup_out[b] += 1;
          ++a; ++b;
        } else if (ci[a] < ci[b]) ++a;
        else ++b;
      }
    }
}

/* ------------------------------------------------------------- partition */

/*
 * Contiguous partition of the ordered vertices into p parts balanced on
 * oriented edges: c_0 = 0, c_p = n, c_i = min{ r : rowptr[r] >= ceil(i*m/p) }.
 */
void orc_cuts(int64_t n, const int64_t *rp, int32_t p, int32_t *cuts) {
  int64_t m = rp[n];
  cuts[0] = 0;
  cuts[p] = (int32_t)n;
  for (int32_t i = 1; i < p; ++i) {
    int64_t target = (i * m + p - 1) / p;
    int64_t r = 0;
    while (r < n && rp[r] < target) ++r;
    cuts[i] = (int32_t)r;
  }
}

/* Part index of position r: the i with c_i <= r < c_{i+1}. */
static int32_t part_of(int64_t r, int32_t p, const int32_t *cuts) {
  int32_t i = 0;
  /* empty parts (c_i = c_{i+1}) own nothing: stop at the first c_{i+1} > r */
  while (i + 1 < p && cuts[i + 1] <= r) ++i;
  return i;
}

/* |G_ij| for all (i,j) in row-major p*p order (Sec. 2 definition of G_ij). */
void orc_block_nnz(int64_t n, const int64_t *rp, const int32_t *ci, int32_t p,
                   const int32_t *cuts, int64_t *nnz) {
  memset(nnz, 0, sizeof(int64_t) * (size_t)p * (size_t)p);
  for (int64_t u = 0; u < n; ++u) {
    int32_t i = part_of(u, p, cuts);
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) nnz[(int64_t)i * p + part_of(ci[e], p, cuts)] += 1;
  }
}

/* ------------------------------------ probe-based symmetric partition (PBD) */

/*
 * Sec. 4.1 asks for a symmetric rectilinear partition that keeps every block
 * small, and Sec. 4.4 measures a partition by its load imbalance
 * lambda = m_max / m_avg over the p(p+1)/2 blocks G_ij, i <= j. The paper
 * uses PBD from a cited report without restating it. The reading taken
 * here is a probe-and-bisect heuristic on the largest block load m_max:
 *
 *  1. Grains. The degree order is cut into G = min(2048, 64p) contiguous
 *     grains balanced on undirected degree (each vertex weighs d(v) = its
 *     out-degree plus its in-degree, so a grain carries about 2m/G of row
 *     and column load): b_0 = 0, b_G = n and, for 0 < t < G,
 *     b_t = min{ r : D(r) >= ceil(t*2m/G) } with D(r) = sum_{r'<r} d(r').
 *     Part boundaries are chosen among the grain boundaries.
 *  2. Loads. L[g][h] = edges (u,v) with u in grain g and v in grain h, and
 *     load(r0,r1,c0,c1) = edges with u in grains [r0,r1) and v in [c0,c1).
 *  3. Probe(B). Part 0 starts at grain x_0 = 0. Given x_0 .. x_i, part i
 *     ends at the largest x_{i+1} in (x_i, G] such that its diagonal block
 *     load(x_i,x_{i+1},x_i,x_{i+1}) and every block above it,
 *     load(x_k,x_{k+1},x_i,x_{i+1}) for k < i, are at most B. Once x_i = G
 *     the remaining parts are empty. The probe fails when no x_{i+1}
 *     exists or when x_p < G. Every block G_ki with k <= i is fixed when
 *     part i closes, so a successful probe bounds every block by B.
 *  4. Bisection. lo = ceil(m / (p(p+1)/2)) - 1 (no partition has all blocks
 *     below the average), hi = m (a single part passes). While hi - lo > 1:
 *     mid = lo + (hi - lo) / 2; hi = mid if Probe(mid) passes, else lo = mid.
 *     B* = hi and the cuts are c_i = b_{x_i} of Probe(B*).
 */

int32_t orc_pbd_grains(int32_t p) {
  int32_t G = 64 * p;
  return G < 2048 ? G : 2048;
}

/* Grain boundaries b[0..G] of step 1. */
void orc_pbd_grain_bounds(int64_t n, const int64_t *rp, const int32_t *ci, int32_t G,
                          int32_t *b) {
  int64_t m = rp[n];
  int64_t *w = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  for (int64_t u = 0; u < n; ++u) {
    w[u] += rp[u + 1] - rp[u];
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) w[ci[e]] += 1;
  }
  b[0] = 0;
  b[G] = (int32_t)n;
  for (int32_t t = 1; t < G; ++t) {
    int64_t target = ((int64_t)t * 2 * m + G - 1) / G;
    int64_t r = 0, D = 0; /* D = D(r) */
    while (r < n && D < target) D += w[r++];
    b[t] = (int32_t)r;
  }
  free(w);
}

/* Prefix table S[(G+1) x (G+1)] of step 2: S[r][c] = edges with u in grains
 * [0, r) and v in grains [0, c). */
void orc_pbd_prefix(int64_t n, const int64_t *rp, const int32_t *ci, int32_t G, const int32_t *b,
                    int64_t *S) {
  int64_t W = (int64_t)G + 1;
  /* grain of each position: the g with b_g <= r < b_{g+1} */
  int32_t *gr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t g = 0; g < G; ++g)
    for (int64_t r = b[g]; r < b[g + 1]; ++r) gr[r] = g;
  memset(S, 0, sizeof(int64_t) * (size_t)(W * W));
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) S[(gr[u] + 1) * W + gr[ci[e]] + 1] += 1;
  free(gr);
  for (int64_t r = 1; r < W; ++r)
    for (int64_t c = 1; c < W; ++c)
      S[r * W + c] += S[(r - 1) * W + c] + S[r * W + c - 1] - S[(r - 1) * W + c - 1];
}

int64_t orc_pbd_load(int32_t G, const int64_t *S, int32_t r0, int32_t r1, int32_t c0,
                     int32_t c1) {
  int64_t W = (int64_t)G + 1;
  return S[r1 * W + c1] - S[r0 * W + c1] - S[r1 * W + c0] + S[r0 * W + c0];
}

/* Step 3: returns 1 and the grain cuts x[0..p] when Probe(B) passes, else 0. */
int32_t orc_pbd_probe(int32_t G, const int64_t *S, int32_t p, int64_t B, int32_t *x) {
  x[0] = 0;
  for (int32_t i = 0; i < p; ++i) {
    if (x[i] == G) {
      x[i + 1] = G;
      continue;
    }
    int32_t best = -1;
    for (int32_t t = x[i] + 1; t <= G; ++t) {
      int ok = orc_pbd_load(G, S, x[i], t, x[i], t) <= B;
      for (int32_t k = 0; ok && k < i; ++k) ok = orc_pbd_load(G, S, x[k], x[k + 1], x[i], t) <= B;
      if (!ok) break; /* every load only grows with t */
      best = t;
    }
    if (best < 0) return 0;
    x[i + 1] = best;
  }
  return x[p] == G;
}

/* Steps 1-4: the cuts c[0..p] of the partition; returns B*. */
int64_t orc_pbd_cuts(int64_t n, const int64_t *rp, const int32_t *ci, int32_t p, int32_t *cuts) {
  int32_t G = orc_pbd_grains(p);
  int64_t m = rp[n];
  int32_t *b = (int32_t *)malloc(sizeof(int32_t) * (size_t)(G + 1));
  int64_t *S = (int64_t *)malloc(sizeof(int64_t) * (size_t)(G + 1) * (size_t)(G + 1));
  int32_t *x = (int32_t *)malloc(sizeof(int32_t) * (size_t)(p + 1));
  orc_pbd_grain_bounds(n, rp, ci, G, b);
  orc_pbd_prefix(n, rp, ci, G, b, S);
  int64_t nblocks = (int64_t)p * (p + 1) / 2;
  int64_t lo = (m + nblocks - 1) / nblocks - 1, hi = m;
  while (hi - lo > 1) {
    int64_t mid = lo + (hi - lo) / 2;
    if (orc_pbd_probe(G, S, p, mid, x)) hi = mid; else lo = mid;
  }
  orc_pbd_probe(G, S, p, hi, x);
  for (int32_t i = 0; i <= p; ++i) cuts[i] = b[x[i]];
  free(b);
  free(S);
  free(x);
  return hi;
}

/* ------------------------------------------------------- task composition */

/* Sec. 4.2: |T| = p(p+1)(p+2)/6. */
int64_t orc_num_tasks(int32_t p) {
  return (int64_t)p * (p + 1) * (p + 2) / 6;
}

/* Alg. 4: every (i,j,k) with i <= j <= k, in the order of its three loops. */
int64_t orc_task_list(int32_t p, int32_t *ti, int32_t *tj, int32_t *tk) {
  int64_t t = 0;
  for (int32_t i = 0; i < p; ++i)
    for (int32_t j = i; j < p; ++j)
      for (int32_t k = j; k < p; ++k) { ti[t] = i; tj[t] = j; tk[t] = k; ++t; }
  return t;
}

/* Sec. 5 task estimate: ExecTime(t) = |G_ij| * max(delta(G_ik), delta(G_jk)). */
void orc_exec_time(int32_t p, const int32_t *cuts, const int64_t *nnz, double *est) {
  int64_t t = 0;
  for (int32_t i = 0; i < p; ++i)
    for (int32_t j = i; j < p; ++j)
      for (int32_t k = j; k < p; ++k) {
        int64_t vi = cuts[i + 1] - cuts[i], vj = cuts[j + 1] - cuts[j];
        double dik = vi > 0 ? (double)nnz[(int64_t)i * p + k] / (double)vi : 0.0;
        double djk = vj > 0 ? (double)nnz[(int64_t)j * p + k] / (double)vj : 0.0;
        est[t++] = (double)nnz[(int64_t)i * p + j] * (dik > djk ? dik : djk);
      }
}

static const double *g_sort_est;

static int cmp_by_estimate(const void *x, const void *y) {
  int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
  if (g_sort_est[a] != g_sort_est[b]) return g_sort_est[a] > g_sort_est[b] ? -1 : 1;
  return (a > b) - (a < b);
}

/* Tasks in non-increasing estimate; equal estimates keep Alg. 4's order. */
void orc_order_tasks(int64_t nt, const double *est, int32_t *order) {
  for (int64_t t = 0; t < nt; ++t) order[t] = (int32_t)t;
  g_sort_est = est;
  qsort(order, (size_t)nt, sizeof(int32_t), cmp_by_estimate);
  g_sort_est = NULL;
}

/* ------------------------------------------------- per-task counts (Sec. 4.3) */

/* N(G_ab, u): the part of u's sorted row whose columns lie in V_b. */
static void partial_list(const int64_t *rp, const int32_t *ci, int64_t u, int32_t b,
                         const int32_t *cuts, int64_t *lo, int64_t *hi) {
  *lo = lower_bound_i32(ci, rp[u], rp[u + 1], cuts[b]);
  *hi = lower_bound_i32(ci, *lo, rp[u + 1], cuts[b + 1]);
}

/* Alg. 5 (bbTC-Intersect) for task (i,j,k). */
uint64_t orc_bbtc_intersect_task(int64_t n, const int64_t *rp, const int32_t *ci,
                                 const int32_t *cuts, int32_t i, int32_t j, int32_t k) {
  (void)n;
  uint64_t tau = 0;
  for (int64_t u = cuts[i]; u < cuts[i + 1]; ++u) {
    int64_t ij_lo, ij_hi, ik_lo, ik_hi;
    partial_list(rp, ci, u, j, cuts, &ij_lo, &ij_hi);
    partial_list(rp, ci, u, k, cuts, &ik_lo, &ik_hi);
    for (int64_t e = ij_lo; e < ij_hi; ++e) {
      int64_t v = ci[e], jk_lo, jk_hi;
      partial_list(rp, ci, v, k, cuts, &jk_lo, &jk_hi);
      tau += orc_n_intersect(ci + ik_lo, ik_hi - ik_lo, ci + jk_lo, jk_hi - jk_lo);
    }
  }
  return tau;
}

/* Alg. 6 (bbTC-HMap) for task (i,j,k); H spans V_k and starts at -1. */
uint64_t orc_bbtc_hmap_task(int64_t n, const int64_t *rp, const int32_t *ci,
                            const int32_t *cuts, int32_t i, int32_t j, int32_t k) {
  (void)n;
  int64_t vk = cuts[k + 1] - cuts[k];
  int64_t *H = (int64_t *)malloc(sizeof(int64_t) * (size_t)(vk > 0 ? vk : 1));
  for (int64_t x = 0; x < vk; ++x) H[x] = -1;
  uint64_t tau = 0;
  for (int64_t u = cuts[i]; u < cuts[i + 1]; ++u) {
    int64_t ik_lo, ik_hi, ij_lo, ij_hi;
    partial_list(rp, ci, u, k, cuts, &ik_lo, &ik_hi);
    for (int64_t e = ik_lo; e < ik_hi; ++e) H[ci[e] - cuts[k]] = u;
    partial_list(rp, ci, u, j, cuts, &ij_lo, &ij_hi);
    for (int64_t e = ij_lo; e < ij_hi; ++e) {
      int64_t v = ci[e], jk_lo, jk_hi;
      partial_list(rp, ci, v, k, cuts, &jk_lo, &jk_hi);
      for (int64_t f = jk_lo; f < jk_hi; ++f)
        if (H[ci[f] - cuts[k]] == u) ++tau;
    }
  }
  free(H);
  return tau;
}

/*
 * Every triangle u < v < w (positions) lies in exactly one task:
 * (part(u), part(v), part(w)), i <= j <= k because parts are contiguous
 * (Sec. 4.2). This classifies the triangles found by a whole-graph merge and
 * accumulates one count per task, indexed in Alg. 4 order.
 */
void orc_classify_triangles(int64_t n, const int64_t *rp, const int32_t *ci, int32_t p,
                            const int32_t *cuts, uint64_t *per_task) {
  int64_t nt = orc_num_tasks(p);
  memset(per_task, 0, sizeof(uint64_t) * (size_t)nt);
  /* index of (i,j,k) in Alg. 4 order, tabulated by enumeration */
  int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)p * p * p);
  int64_t t = 0;
  for (int32_t i = 0; i < p; ++i)
    for (int32_t j = i; j < p; ++j)
      for (int32_t k = j; k < p; ++k) idx[((int64_t)i * p + j) * p + k] = t++;
  for (int64_t u = 0; u < n; ++u) {
    int32_t bu = part_of(u, p, cuts);
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
      int64_t v = ci[e];
      int32_t bv = part_of(v, p, cuts);
      int64_t a = rp[u], b = rp[v];
      while (a < rp[u + 1] && b < rp[v + 1]) {
        if (ci[a] == ci[b]) {
          per_task[idx[((int64_t)bu * p + bv) * p + part_of(ci[a], p, cuts)]] += 1;
          ++a; ++b;
        } else if (ci[a] < ci[b]) ++a;
        else ++b;
      }
    }
  }
  free(idx);
}

/* ------------------------------------------------------- workload figures */

/*
 * Algorithmic bytes of the counting step on the oriented CSR, with 4-byte ids:
 *   wmin   = 4 * (m + sum over oriented edges (u,v) of d+(v))
 *            (each edge read once, and the out-list of v read once per edge
 *             that enters v -- the candidates that may close a wedge)
 *   wmerge = 4 * sum over oriented edges (u,v) of (d+(u) + d+(v))
 *   wedges = sum over oriented edges (u,v) of d+(v)
 */
void orc_work_figures(int64_t n, const int64_t *rp, const int32_t *ci, uint64_t *wmin,
                      uint64_t *wmerge, uint64_t *wedges) {
  uint64_t m = (uint64_t)rp[n], w = 0, mg = 0;
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
      int64_t v = ci[e];
      uint64_t dv = (uint64_t)(rp[v + 1] - rp[v]), du = (uint64_t)(rp[u + 1] - rp[u]);
      w += dv;
      mg += du + dv;
    }
  *wmin = 4 * (m + w);
  *wmerge = 4 * mg;
  *wedges = w;
}

/* ------------------------------------------- single-vertex count (sampling) */

static int cmp_i32(const void *x, const void *y) {
  int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
  return (a > b) - (a < b);
}

/* sorted distinct neighbours of x other than x itself; returns their number */
static int64_t simple_neighbours(const int64_t *rowptr, const int32_t *colidx, int64_t x,
                                 int32_t *buf) {
  int64_t len = 0;
  for (int64_t e = rowptr[x]; e < rowptr[x + 1]; ++e)
    if (colidx[e] != x) buf[len++] = colidx[e];
  qsort(buf, (size_t)len, sizeof(int32_t), cmp_i32);
  int64_t u = 0;
  for (int64_t i = 0; i < len; ++i)
    if (i == 0 || buf[i] != buf[i - 1]) buf[u++] = buf[i];
  return u;
}

/*
 * Triangles containing vertex x, by the definition (Sec. 2): the number of
 * edges {y, z} between two distinct neighbours y < z of x. Reads the input
 * CSR directly, which must list every edge under both endpoints. Used to
 * check sampled per-vertex counts on graphs too large for the full oracle.
 */
uint64_t orc_vertex_triangles(int64_t n, const int64_t *rowptr, const int32_t *colidx,
                              int64_t x) {
  (void)n;
  int64_t dx = rowptr[x + 1] - rowptr[x];
  int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)(dx > 0 ? dx : 1));
  int64_t ns = simple_neighbours(rowptr, colidx, x, S);
  uint64_t t = 0;
  for (int64_t a = 0; a < ns; ++a) {
    int64_t y = S[a];
    int64_t dy = rowptr[y + 1] - rowptr[y];
    int32_t *Ny = (int32_t *)malloc(sizeof(int32_t) * (size_t)(dy > 0 ? dy : 1));
    int64_t ny = simple_neighbours(rowptr, colidx, y, Ny);
    /* common elements of S and Ny that are greater than y */
    t += orc_n_intersect(S + a + 1, ns - a - 1, Ny, ny);
    free(Ny);
  }
  free(S);
  return t;
}
