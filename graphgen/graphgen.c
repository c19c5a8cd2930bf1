/*
 * graphgen.c -- seeded synthetic graph generators (R-MAT, G(n,m), Chung-Lu).
 *
 * These produce the INPUTS that both the CUDA library and the CPU oracle
 * consume. Nothing here performs any step of triangle counting: no
 * de-duplication, no ordering, no orientation, no counting. The output is a
 * symmetrised CSR in which every drawn pair (a,b) is listed as b in row a and
 * as a in row b, duplicates and self-loops included exactly as drawn; removing
 * them is the counting method's own first step.
 *
 * Randomness: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014) used as a counter-based generator. Draw i
 * of stream s under seed S is the (i+1)-th output of the SplitMix64 sequence
 * whose initial state is mix(S + gamma*(s+1)), i.e. mix(state0 + gamma*(i+1)).
 * Every draw is addressable by (seed, stream, index), so generation is
 * parallel and independent of the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t gg_draw(uint64_t seed, uint64_t stream, uint64_t index) {
  uint64_t state0 = gg_mix(seed + GG_GAMMA * (stream + 1));
  return gg_mix(state0 + GG_GAMMA * (index + 1));
}

/* Uniform integer in [0, n) from 32 random bits (multiply-shift). */
static inline uint32_t gg_below(uint32_t bits, uint32_t n) {
  return (uint32_t)(((uint64_t)bits * (uint64_t)n) >> 32);
}

/*
 * R-MAT (Chakrabarti, Zhan & Faloutsos 2004): each of the M = edge_factor * 2^scale
 * pairs descends `scale` levels of the adjacency matrix, choosing quadrant
 * (row bit, col bit) = (0,0),(0,1),(1,0),(1,1) with probability a,b,c,d.
 * One 64-bit draw serves two levels (32 bits each). No noise, no relabelling.
 */
void gg_rmat_pairs(int32_t scale, int64_t M, double a, double b, double c,
                   uint64_t seed, int32_t *src, int32_t *dst) {
  const uint64_t ta = (uint64_t)llround(a * 4294967296.0);
  const uint64_t tb = ta + (uint64_t)llround(b * 4294967296.0);
  const uint64_t tc = tb + (uint64_t)llround(c * 4294967296.0);
  const int64_t draws_per_edge = (scale + 1) / 2;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < M; ++e) {
    uint32_t r = 0, col = 0;
    uint64_t word = 0;
    for (int32_t lvl = 0; lvl < scale; ++lvl) {
      if ((lvl & 1) == 0) word = gg_draw(seed, 0, (uint64_t)e * draws_per_edge + lvl / 2);
      uint64_t u = (lvl & 1) ? (word >> 32) : (word & 0xFFFFFFFFULL);
      uint32_t rb, cb;
      if (u < ta) { rb = 0; cb = 0; }
      else if (u < tb) { rb = 0; cb = 1; }
      else if (u < tc) { rb = 1; cb = 0; }
      else { rb = 1; cb = 1; }
      r = (r << 1) | rb;
      col = (col << 1) | cb;
    }
    src[e] = (int32_t)r;
    dst[e] = (int32_t)col;
  }
}

/* G(n, M) with replacement: M pairs, each endpoint uniform on [0, n). */
void gg_gnm_pairs(int64_t n, int64_t M, uint64_t seed, int32_t *src, int32_t *dst) {
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < M; ++e) {
    uint64_t w = gg_draw(seed, 1, (uint64_t)e);
    src[e] = (int32_t)gg_below((uint32_t)(w >> 32), (uint32_t)n);
    dst[e] = (int32_t)gg_below((uint32_t)w, (uint32_t)n);
  }
}

/*
 * Chung-Lu expected-degree weights: w_i = min(wmax, C * (i+1)^(-1/(gamma-1))),
 * with C chosen (bisection) so that sum_i w_i = weight_sum. Returns C.
 */
double gg_chunglu_weights(int64_t n, double gamma, double wmax, double weight_sum,
                          double *w) {
  const double ex = -1.0 / (gamma - 1.0);
  /* w[] first holds the uncapped shape (i+1)^ex */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) w[i] = pow((double)(i + 1), ex);
  /* at C = wmax / w[n-1] every weight is capped, so the sum is n * wmax */
  double lo = 0.0, hi = wmax / w[n - 1];
  for (int it = 0; it < 64; ++it) {
    double mid = 0.5 * (lo + hi), s = 0.0;
    /* fixed chunking keeps the floating-point sum independent of threads */
    const int64_t nchunk = 64, step = (n + nchunk - 1) / nchunk;
    double part[64];
#pragma omp parallel for schedule(static)
    for (int64_t ch = 0; ch < nchunk; ++ch) {
      double acc = 0.0;
      int64_t end = (ch + 1) * step < n ? (ch + 1) * step : n;
      for (int64_t i = ch * step; i < end; ++i) {
        double x = mid * w[i];
        acc += x < wmax ? x : wmax;
      }
      part[ch] = acc;
    }
    for (int64_t ch = 0; ch < nchunk; ++ch) s += part[ch];
    if (s < weight_sum) lo = mid; else hi = mid;
  }
  const double C = 0.5 * (lo + hi);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double x = C * w[i];
    w[i] = x < wmax ? x : wmax;
  }
  return C;
}

/*
 * Vose's alias method (Vose 1991): prob[i] in 32-bit fixed point, alias[i].
 * Sampling: column i uniform, keep i if coin < prob[i], else alias[i].
 */
void gg_alias_build(int64_t n, const double *w, uint32_t *prob, int32_t *alias) {
  double total = 0.0;
  for (int64_t i = 0; i < n; ++i) total += w[i];
  double *scaled = (double *)malloc(sizeof(double) * (size_t)n);
  int32_t *small = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *large = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int64_t ns = 0, nl = 0;
  for (int64_t i = 0; i < n; ++i) {
    scaled[i] = w[i] * (double)n / total;
    if (scaled[i] < 1.0) small[ns++] = (int32_t)i; else large[nl++] = (int32_t)i;
  }
  while (ns > 0 && nl > 0) {
    int32_t s = small[--ns], l = large[--nl];
    double ps = scaled[s];
    prob[s] = ps >= 1.0 ? 0xFFFFFFFFu : (uint32_t)(ps * 4294967296.0);
    alias[s] = l;
    scaled[l] = (scaled[l] + ps) - 1.0;
    if (scaled[l] < 1.0) small[ns++] = l; else large[nl++] = l;
  }
  while (nl > 0) { int32_t l = large[--nl]; prob[l] = 0xFFFFFFFFu; alias[l] = l; }
  while (ns > 0) { int32_t s = small[--ns]; prob[s] = 0xFFFFFFFFu; alias[s] = s; }
  free(scaled); free(small); free(large);
}

static inline int32_t gg_alias_sample(uint64_t r, int64_t n, const uint32_t *prob,
                                      const int32_t *alias) {
  uint32_t col = gg_below((uint32_t)(r >> 32), (uint32_t)n);
  uint32_t coin = (uint32_t)r;
  return coin < prob[col] ? (int32_t)col : alias[col];
}

/* M Chung-Lu pairs: both endpoints drawn independently proportional to w. */
void gg_chunglu_pairs(int64_t n, int64_t M, const uint32_t *prob, const int32_t *alias,
                      uint64_t seed, int32_t *src, int32_t *dst) {
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < M; ++e) {
    src[e] = gg_alias_sample(gg_draw(seed, 2, 2 * (uint64_t)e), n, prob, alias);
    dst[e] = gg_alias_sample(gg_draw(seed, 2, 2 * (uint64_t)e + 1), n, prob, alias);
  }
}

static int gg_cmp_i32(const void *x, const void *y) {
  int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
  return (a > b) - (a < b);
}

/*
 * Symmetrised CSR of M pairs over n vertices: pair (a,b) lists b in row a and a
 * in row b (a self-loop lists a twice in row a). rowptr has n+1 entries and
 * colidx 2*M; each row is sorted ascending so the output does not depend on
 * the thread count. Duplicates and self-loops are kept.
 */
void gg_pairs_to_csr(int64_t n, int64_t M, const int32_t *src, const int32_t *dst,
                     int64_t *rowptr, int32_t *colidx) {
  int64_t *cursor = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < M; ++e) {
    __atomic_fetch_add(&cursor[src[e]], 1, __ATOMIC_RELAXED);
    __atomic_fetch_add(&cursor[dst[e]], 1, __ATOMIC_RELAXED);
  }
  int64_t acc = 0;
  for (int64_t v = 0; v < n; ++v) { rowptr[v] = acc; acc += cursor[v]; cursor[v] = rowptr[v]; }
  rowptr[n] = acc;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < M; ++e) {
    int64_t p = __atomic_fetch_add(&cursor[src[e]], 1, __ATOMIC_RELAXED);
    colidx[p] = dst[e];
    p = __atomic_fetch_add(&cursor[dst[e]], 1, __ATOMIC_RELAXED);
    colidx[p] = src[e];
  }
  free(cursor);
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t v = 0; v < n; ++v) {
    int64_t len = rowptr[v + 1] - rowptr[v];
    if (len > 1) qsort(colidx + rowptr[v], (size_t)len, sizeof(int32_t), gg_cmp_i32);
  }
}

/* OpenMP threads used by the calling thread's later generator calls. */
void gg_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int gg_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
