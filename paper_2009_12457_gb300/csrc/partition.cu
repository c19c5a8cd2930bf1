// partition.cu -- a5, probe-based symmetric partition (opts.partition = PBD).
//
// Sec. 4.1 asks for a symmetric rectilinear partition whose blocks stay
// small, and Sec. 4.4 measures it by the load imbalance lambda = m_max /
// m_avg over the p(p+1)/2 blocks G_ij, i <= j. The partition here bounds the
// largest block load m_max by probing and bisection:
//
//  1. Grains. The degree order is cut into G = min(2048, 64p) grains
//     balanced on undirected degree: b_t = min{ r : D(r) >= ceil(t*2m/G) },
//     D(r) = sum_{r' < r} (d+(r') + d-(r')) = rowptr[r] + (edges into
//     positions below r). Part boundaries are grain boundaries.
//  2. Loads. L[g][h] = oriented edges from grain g into grain h, and the
//     (G+1) x (G+1) prefix table S of L, so that the load of any rectangle
//     of grains is four reads.
//  3. Probe(B). Part i starts where part i-1 ended and takes the most
//     grains for which its diagonal block and every block above it in its
//     column (rows of parts k < i) hold at most B edges. Each load only
//     grows with the part's end, so the feasible ends form a prefix and are
//     searched 33-ary: 32 warps test 32 candidate ends at once, one lane per
//     block. The probe passes when the p parts cover all G grains.
//  4. Bisection on B in (ceil(m / (p(p+1)/2)) - 1, m]: the smallest B the
//     bisection reaches is B*, and the cuts are those of Probe(B*).
//
// Steps 1-2 read the oriented CSR once (in-degree histogram, grain loads);
// step 3-4 run in one CTA on the 33 MB table, which stays in L2.
#include "graph.cuh"
#include "primitives.cuh"

namespace bbtc {

namespace {

constexpr int MAXP = 64;
constexpr int PB_NT = 256;
constexpr int PB_HUB = 8192;   // top positions whose in-degree is counted on chip
constexpr int PB_MAXG = 2048;
constexpr int PB_SEARCH_NT = 1024;
constexpr int PB_WARPS = PB_SEARCH_NT / 32;

inline int pbd_grains(int p) { return 64 * p < PB_MAXG ? 64 * p : PB_MAXG; }

__device__ __forceinline__ void pb_share(int64_t e0, int64_t e1, int64_t *b0, int64_t *b1) {
  const int64_t per = (e1 - e0 + gridDim.x - 1) / gridDim.x;
  *b0 = e0 + (int64_t)blockIdx.x * per;
  *b1 = *b0 + per < e1 ? *b0 + per : e1;
}

// In-degree of every position. In degree order the top positions receive most
// edges, so each CTA counts its contiguous share of the columns for the top
// PB_HUB positions in shared memory and adds those once per CTA.
__global__ void __launch_bounds__(PB_NT) k_pbd_indeg(const int32_t *__restrict__ colidx,
                                                     int64_t m, int64_t n,
                                                     unsigned long long *__restrict__ indeg) {
  __shared__ unsigned sm[PB_HUB];
  const int64_t hub0 = n > PB_HUB ? n - PB_HUB : 0;
  for (int i = threadIdx.x; i < PB_HUB; i += PB_NT) sm[i] = 0;
  __syncthreads();
  int64_t b0, b1;
  pb_share(0, m, &b0, &b1);
  for (int64_t e = b0 + threadIdx.x; e < b1; e += PB_NT) {
    const int32_t v = colidx[e];
    if (v >= hub0) atomicAdd(&sm[v - hub0], 1u);
    else atomicAdd(&indeg[v], 1ull);
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n - hub0; i += PB_NT)
    if (sm[i]) atomicAdd(&indeg[hub0 + i], (unsigned long long)sm[i]);
}

// Grain boundaries b[0..G] from D(r) = rowptr[r] + in_below[r] (non-decreasing).
__global__ void k_pbd_bounds(const int64_t *__restrict__ rowptr,
                             const unsigned long long *__restrict__ in_below, int64_t n,
                             int64_t m, int G, int32_t *__restrict__ b) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > G) return;
  if (t == 0 || t == G) {
    b[t] = t == 0 ? 0 : (int32_t)n;
    return;
  }
  const int64_t target = ((int64_t)t * 2 * m + G - 1) / G;
  int64_t lo = 0, hi = n;  // the answer lies in [lo, hi]; D(n) = 2m >= target
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (rowptr[mid] + (int64_t)in_below[mid] < target) lo = mid + 1;
    else hi = mid;
  }
  b[t] = (int32_t)lo;
}

// Grain of position r: the g in [0, G) with b[g] <= r < b[g+1] (empty grains
// own nothing): one less than the first boundary above r.
__device__ __forceinline__ int grain_of(const int32_t *b, int G, int32_t r) {
  int lo = 0, hi = G + 1;  // first index with b[idx] > r lies in (0, G]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (b[mid] <= r) lo = mid + 1;
    else hi = mid;
  }
  return lo - 1;
}

// L[g*G + h] += oriented edges from grain g into grain h. Edges are sorted by
// (source, destination), so neighbouring lanes often hit one cell: lanes with
// equal cells add once.
__global__ void __launch_bounds__(PB_NT) k_pbd_loads(const int32_t *__restrict__ esrc,
                                                     const int32_t *__restrict__ colidx,
                                                     int64_t m, const int32_t *__restrict__ b_g,
                                                     int G, unsigned *__restrict__ L) {
  __shared__ int32_t b[PB_MAXG + 1];
  for (int i = threadIdx.x; i <= G; i += PB_NT) b[i] = b_g[i];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * PB_NT;
  // every lane of a warp runs the same number of iterations (for the match)
  const int64_t base0 = (int64_t)blockIdx.x * PB_NT + (threadIdx.x & ~31u);
  for (int64_t base = base0; base < m; base += stride) {
    const int64_t e = base + (threadIdx.x & 31u);
    const bool valid = e < m;
    const uint32_t cell = valid ? (uint32_t)(grain_of(b, G, esrc[e]) * G +
                                             grain_of(b, G, colidx[e]))
                                : 0xffffffffu;
    const unsigned peers = __match_any_sync(0xffffffffu, cell);
    if (valid && (threadIdx.x & 31u) == (unsigned)(__ffs(peers) - 1))
      atomicAdd(&L[cell], (unsigned)__popc(peers));
  }
}

// Column prefix of L into the interior of S: S[(r+1)*W + c+1] = sum_{r' <= r}
// L[r'*G + c]; row 0 and column 0 of S are zero. A CTA takes 32 columns;
// thread (ty, tx) sums rows [ty*R, (ty+1)*R) of column tx, the 32 partial sums
// of a column are scanned in shared memory, and each thread then writes its
// rows' prefixes.
constexpr int CS_ROWS = 32;
__global__ void __launch_bounds__(32 * CS_ROWS) k_pbd_colscan(const unsigned *__restrict__ L,
                                                              int G,
                                                              unsigned long long *__restrict__ S) {
  __shared__ unsigned long long part[CS_ROWS][33];
  const int W = G + 1;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + tx;
  const int R = (G + CS_ROWS - 1) / CS_ROWS;
  const int r0 = ty * R, r1 = r0 + R < G ? r0 + R : G;
  unsigned long long sum = 0;
  if (c < G)
#pragma unroll 8
    for (int r = r0; r < r1; ++r) sum += L[(int64_t)r * G + c];
  part[ty][tx] = sum;
  __syncthreads();
  if (ty == 0) {
    unsigned long long run = 0;
    for (int q = 0; q < CS_ROWS; ++q) {
      const unsigned long long x = part[q][tx];
      part[q][tx] = run;
      run += x;
    }
  }
  __syncthreads();
  if (c < G) {
    unsigned long long run = part[ty][tx];
#pragma unroll 8
    for (int r = r0; r < r1; ++r) {
      run += L[(int64_t)r * G + c];
      S[(int64_t)(r + 1) * W + c + 1] = run;
    }
    if (ty == 0) S[c + 1] = 0;  // row 0
  }
  if (blockIdx.x == 0 && tx == 0) {  // column 0
    for (int r = r0; r < r1; ++r) S[(int64_t)(r + 1) * W] = 0;
    if (ty == 0) S[0] = 0;
  }
}

// Row prefix of rows 1..G of S in place (one warp per row), after the column
// prefix: S[r][c] = edges from grains [0, r) into grains [0, c).
__global__ void k_pbd_rowscan(unsigned long long *__restrict__ S, int G) {
  const int W = G + 1;
  const int r = 1 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const unsigned lane = threadIdx.x & 31u;
  if (r > G) return;
  unsigned long long carry = 0;
  for (int c0 = 1; c0 <= G; c0 += 32) {
    const int c = c0 + (int)lane;
    const unsigned long long x = c <= G ? S[(int64_t)r * W + c] : 0ull;
    const unsigned long long inc = warp_inclusive_scan(x) + carry;
    if (c <= G) S[(int64_t)r * W + c] = inc;
    carry = __shfl_sync(0xffffffffu, inc, 31);
  }
}

__device__ __forceinline__ long long rect(const unsigned long long *__restrict__ S, int W, int r0,
                                          int r1, int c0, int c1) {
  return (long long)(S[(int64_t)r1 * W + c1] - S[(int64_t)r0 * W + c1] -
                     S[(int64_t)r1 * W + c0] + S[(int64_t)r0 * W + c0]);
}

struct SearchShared {
  int32_t x[MAXP + 1];
  int cand[PB_WARPS];
  int feas[PB_WARPS];
  int lo_t, hi_t;
  int ok;
};

// Probe(B) by the whole CTA: fills sh.x and returns whether it passed.
__device__ bool pbd_probe(const unsigned long long *__restrict__ S, int G, int p, long long B,
                          SearchShared &sh) {
  const int W = G + 1;
  const int warp = threadIdx.x >> 5;
  const unsigned lane = threadIdx.x & 31u;
  if (threadIdx.x == 0) {
    sh.x[0] = 0;
    sh.ok = 1;
  }
  __syncthreads();
  for (int i = 0; i < p; ++i) {
    const int xi = sh.x[i];
    if (xi == G) {
      if (threadIdx.x == 0) sh.x[i + 1] = G;
      __syncthreads();
      continue;
    }
    // feasible ends: a prefix of (xi, G]; lo_t is known feasible (xi stands for
    // "none yet"), hi_t known infeasible (G + 1 stands for "beyond the end")
    if (threadIdx.x == 0) {
      sh.lo_t = xi;
      sh.hi_t = G + 1;
    }
    __syncthreads();
    while (sh.hi_t - sh.lo_t > 1) {
      const int lo_t = sh.lo_t, hi_t = sh.hi_t;
      const int t = lo_t + (int)(((long long)(hi_t - lo_t) * (warp + 1)) / (PB_WARPS + 1));
      bool feasible = true;
      if (t > lo_t && t < hi_t) {
        // lane k checks the block of part k's rows (k < i), lane i the diagonal
        for (int k = (int)lane; k <= i; k += 32) {
          const long long load = k < i ? rect(S, W, sh.x[k], sh.x[k + 1], xi, t)
                                       : rect(S, W, xi, t, xi, t);
          if (load > B) feasible = false;
        }
      }
      feasible = __all_sync(0xffffffffu, feasible);
      if (lane == 0) {
        sh.cand[warp] = t;
        sh.feas[warp] = feasible ? 1 : 0;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int nlo = lo_t, nhi = hi_t;
        for (int w = 0; w < PB_WARPS; ++w) {
          const int c = sh.cand[w];
          if (c <= lo_t || c >= hi_t) continue;
          if (sh.feas[w]) nlo = c > nlo ? c : nlo;
          else nhi = c < nhi ? c : nhi;
        }
        // candidates can coincide when the range is small: step one grain then
        if (nlo == lo_t && nhi == hi_t) {
          const int c = lo_t + 1;
          bool f = true;
          for (int k = 0; k <= i && f; ++k) {
            const long long load = k < i ? rect(S, W, sh.x[k], sh.x[k + 1], xi, c)
                                         : rect(S, W, xi, c, xi, c);
            if (load > B) f = false;
          }
          if (f) nlo = c;
          else nhi = c;
        }
        sh.lo_t = nlo;
        sh.hi_t = nhi;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (sh.lo_t == xi) sh.ok = 0;
      sh.x[i + 1] = sh.lo_t;
    }
    __syncthreads();
    if (!sh.ok) break;
  }
  __syncthreads();
  const bool passed = sh.ok && sh.x[p] == G;
  __syncthreads();  // every thread has read the result before the next probe resets it
  return passed;
}

// Steps 3-4 in one CTA: bisection on B, then the cuts of Probe(B*).
__global__ void __launch_bounds__(PB_SEARCH_NT) k_pbd_search(
    const unsigned long long *__restrict__ S, int G, int p, int64_t m,
    const int32_t *__restrict__ b, int32_t *__restrict__ cuts, long long *__restrict__ bstar) {
  __shared__ SearchShared sh;
  const long long nblocks = (long long)p * (p + 1) / 2;
  long long lo = (m + nblocks - 1) / nblocks - 1, hi = m;
  while (hi - lo > 1) {
    const long long mid = lo + (hi - lo) / 2;
    if (pbd_probe(S, G, p, mid, sh)) hi = mid;
    else lo = mid;
  }
  pbd_probe(S, G, p, hi, sh);
  if (threadIdx.x <= p) cuts[threadIdx.x] = b[sh.x[threadIdx.x]];
  if (threadIdx.x == 0) *bstar = hi;
}

}  // namespace

bbtc_status pbd_partition(const bbtc_graph *g, int p, int32_t *d_cuts, int64_t *h_bstar,
                          cudaStream_t s) {
  if (p < 1 || p > MAXP) {
    set_error("pbd_partition: p = %d outside 1..%d", p, MAXP);
    return BBTC_EINVAL;
  }
  const int64_t n = g->n, m = g->m;
  const int G = pbd_grains(p);
  const int W = G + 1;
  Scratch scratch(s);
  unsigned long long *in_below = nullptr, *S = nullptr;
  unsigned *L = nullptr;
  int32_t *b = nullptr;
  long long *d_bstar = nullptr;
  BBTC_TRY(scratch.get(&in_below, n + 1));
  BBTC_TRY(scratch.get(&b, W));
  BBTC_TRY(scratch.get(&L, (int64_t)G * G));
  BBTC_TRY(scratch.get(&S, (int64_t)W * W));
  BBTC_TRY(scratch.get(&d_bstar, 1));
  // 1: in-degrees, their exclusive prefix (edges into positions below r), grains
  BBTC_CUDA(cudaMemsetAsync(in_below, 0, sizeof(unsigned long long) * (size_t)(n + 1), s));
  if (m > 0) {
    k_pbd_indeg<<<grid_for(m, PB_NT * 64, 4), PB_NT, 0, s>>>(g->colidx, m, n, in_below);
    BBTC_LAUNCH_CHECK();
  }
  BBTC_TRY(exclusive_scan_u64(reinterpret_cast<uint64_t *>(in_below),
                                reinterpret_cast<uint64_t *>(in_below), n + 1, s));
  k_pbd_bounds<<<(W + 255) / 256, 256, 0, s>>>(g->rowptr, in_below, n, m, G, b);
  BBTC_LAUNCH_CHECK();
  // 2: grain loads and their prefix table
  BBTC_CUDA(cudaMemsetAsync(L, 0, sizeof(unsigned) * (size_t)G * G, s));
  if (m > 0) {
    k_pbd_loads<<<grid_for(m, PB_NT, 16), PB_NT, 0, s>>>(g->esrc, g->colidx, m, b, G, L);
    BBTC_LAUNCH_CHECK();
  }
  k_pbd_colscan<<<(G + 31) / 32, 32 * CS_ROWS, 0, s>>>(L, G, S);
  BBTC_LAUNCH_CHECK();
  k_pbd_rowscan<<<(G * 32 + 255) / 256, 256, 0, s>>>(S, G);
  BBTC_LAUNCH_CHECK();
  // 3-4: search
  k_pbd_search<<<1, PB_SEARCH_NT, 0, s>>>(S, G, p, m, b, d_cuts, d_bstar);
  BBTC_LAUNCH_CHECK();
  long long hb = 0;
  BBTC_CUDA(cudaMemcpyAsync(&hb, d_bstar, sizeof(long long), cudaMemcpyDeviceToHost, s));
  BBTC_CUDA(cudaStreamSynchronize(s));
  *h_bstar = hb;
  return BBTC_OK;
}

}  // namespace bbtc
