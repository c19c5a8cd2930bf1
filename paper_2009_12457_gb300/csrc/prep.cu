// prep.cu -- graph-only steps of bbTC (run once per graph by bbtc_graph_create):
//   a1 canonical simple edge set  (Sec. 2: simple undirected graph, (u,v) with u<v)
//   a2 degree                     (Sec. 2, Sec. 4.1)
//   a3 order by degree            (Sec. 4.1: non-decreasing degree, ties by id)
//   a4 orientation                (Sec. 2: N(G,u) = {v : (u,v) in E, u < v})
#include <limits.h>

#include "graph.cuh"
#include "primitives.cuh"

namespace bbtc {

namespace {

constexpr int EK_NT = 256;
constexpr int EK_TILE = 2048;

// rowptr[0] == 0 and non-decreasing; error bit 1 otherwise.
__global__ void k_validate_rowptr(const int64_t *__restrict__ rowptr, int64_t n,
                                  int32_t *__restrict__ err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (rowptr[i] > rowptr[i + 1]) atomicOr(err, 1);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && rowptr[0] != 0) atomicOr(err, 1);
}

// a1: one 64-bit key (min << nb) | max per input entry joining two different
// vertices. Self-loops (and, for symmetric input, entries with u > v) emit
// nothing. Two passes over tiles of EK_TILE entries: count the keys of each
// tile, then (after a scan of the counts) write them compacted. Thread t of a
// tile owns entries [t*EK_ITEMS, (t+1)*EK_ITEMS) and walks their rows forward
// from one binary search inside the tile's row window.
constexpr int EK_ITEMS = EK_TILE / EK_NT;

// For a batch (voff != nullptr), graph g owns rows [voff[g], voff[g+1]) and
// its entries are local ids in [0, voff[g+1] - voff[g]), shifted by voff[g].
template <bool WRITE>
__global__ void __launch_bounds__(EK_NT) k_emit_keys(const int64_t *__restrict__ rowptr,
                                                     const int32_t *__restrict__ colidx,
                                                     int64_t n, int64_t nnz, int nb,
                                                     bool symmetric,
                                                     const int64_t *__restrict__ voff, int ng,
                                                     uint64_t *__restrict__ tile_count,
                                                     uint64_t *__restrict__ keys,
                                                     int32_t *__restrict__ err) {
  __shared__ int64_t win[2];
  __shared__ uint64_t tmp[EK_NT / 32 + 1];
  const int64_t ntiles = (nnz + EK_TILE - 1) / EK_TILE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t t0 = tile * EK_TILE;
    const int64_t t1 = t0 + EK_TILE < nnz ? t0 + EK_TILE : nnz;
    if (threadIdx.x < 2) {
      // last row r in [0, n) with rowptr[r] <= target
      int64_t target = threadIdx.x == 0 ? t0 : t1 - 1;
      int64_t lo = 0, hi = n;  // invariant: rowptr[lo] <= target
      while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (rowptr[mid] <= target) lo = mid; else hi = mid;
      }
      win[threadIdx.x] = lo;
    }
    __syncthreads();
    const int64_t rlo = win[0], rhi = win[1];
    const int64_t first = t0 + (int64_t)threadIdx.x * EK_ITEMS;
    uint64_t key[EK_ITEMS];
    uint64_t c = 0;
    int64_t u = rlo;
    if (first < t1) {
      int64_t lo = rlo, hi = rhi + 1;
      while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (rowptr[mid] <= first) lo = mid; else hi = mid;
      }
      u = lo;
    }
    int gi = 0;
    int64_t gbase = 0, gend = n;
    if (voff) {
      int lo = 0, hi = ng;  // last graph with voff[lo] <= u
      while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (voff[mid] <= u) lo = mid; else hi = mid;
      }
      gi = lo;
      gbase = voff[gi];
      gend = voff[gi + 1];
    }
#pragma unroll
    for (int i = 0; i < EK_ITEMS; ++i) {
      const int64_t idx = first + i;
      key[i] = ~0ull;
      if (idx < t1) {
        while (u < rhi && rowptr[u + 1] <= idx) ++u;
        if (voff) {
          while (u >= gend && gi + 1 < ng) {
            ++gi;
            gbase = voff[gi];
            gend = voff[gi + 1];
          }
        }
        int64_t v = colidx[idx];
        const bool in_range = voff ? (v >= 0 && v < gend - gbase) : (v >= 0 && v < n);
        v += gbase;
        if (!in_range) {
          if (!WRITE) atomicOr(err, 2);
        } else if (v != u && !(symmetric && u > v)) {
          uint64_t a = (uint64_t)(u < v ? u : v), b = (uint64_t)(u < v ? v : u);
          key[i] = (a << nb) | b;
          ++c;
        }
      }
    }
    uint64_t total;
    uint64_t pos = block_exclusive_scan<uint64_t, EK_NT>(c, tmp, &total);
    if (!WRITE) {
      if (threadIdx.x == 0) tile_count[tile] = total;
    } else {
      pos += tile_count[tile];
#pragma unroll
      for (int i = 0; i < EK_ITEMS; ++i)
        if (key[i] != ~0ull) keys[pos++] = key[i];
    }
  }
}

constexpr int UQ_NT = 512;
constexpr int UQ_ITEMS = 8;
constexpr int UQ_TILE = UQ_NT * UQ_ITEMS;

__device__ __forceinline__ bool is_head(const uint64_t *keys, int64_t i, uint64_t sentinel) {
  uint64_t k = keys[i];
  return k != sentinel && (i == 0 || keys[i - 1] != k);
}

__global__ void __launch_bounds__(UQ_NT) k_unique_count(const uint64_t *__restrict__ keys,
                                                        int64_t count, uint64_t sentinel,
                                                        uint64_t *__restrict__ block_counts) {
  __shared__ uint64_t tmp[UQ_NT / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * UQ_TILE + (int64_t)threadIdx.x * UQ_ITEMS;
  uint64_t c = 0;
#pragma unroll
  for (int i = 0; i < UQ_ITEMS; ++i)
    if (base + i < count && is_head(keys, base + i, sentinel)) ++c;
  uint64_t total;
  block_exclusive_scan<uint64_t, UQ_NT>(c, tmp, &total);
  if (threadIdx.x == 0) block_counts[blockIdx.x] = total;
}

// a1 + a2: compact the distinct keys and count each endpoint's degree. Keys
// are sorted by their first endpoint, so lanes holding equal endpoints add
// once per group (match_any) instead of once per edge.
__global__ void __launch_bounds__(UQ_NT) k_unique_write(const uint64_t *__restrict__ keys,
                                                        int64_t count, uint64_t sentinel,
                                                        const uint64_t *__restrict__ block_off,
                                                        int nb, uint64_t *__restrict__ ukeys,
                                                        int32_t *__restrict__ deg) {
  __shared__ uint64_t tmp[UQ_NT / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * UQ_TILE + (int64_t)threadIdx.x * UQ_ITEMS;
  const unsigned lane = threadIdx.x & 31u;
  bool head[UQ_ITEMS];
  uint64_t c = 0;
#pragma unroll
  for (int i = 0; i < UQ_ITEMS; ++i) {
    head[i] = base + i < count && is_head(keys, base + i, sentinel);
    c += head[i];
  }
  uint64_t total;
  uint64_t pos = block_exclusive_scan<uint64_t, UQ_NT>(c, tmp, &total) + block_off[blockIdx.x];
  const uint64_t mask = (1ull << nb) - 1ull;
#pragma unroll
  for (int i = 0; i < UQ_ITEMS; ++i) {
    uint64_t k = head[i] ? keys[base + i] : 0;
    if (head[i]) ukeys[pos++] = k;
    const int64_t a = head[i] ? (int64_t)(k >> nb) : -1;
    const int64_t b = head[i] ? (int64_t)(k & mask) : -1;
    unsigned peers = __match_any_sync(0xffffffffu, a);
    if (a >= 0 && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(&deg[a], __popc(peers));
    peers = __match_any_sync(0xffffffffu, b);
    if (b >= 0 && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(&deg[b], __popc(peers));
  }
}

// a3 keys: (degree << nb) | id, so ascending order is (degree, id).
__global__ void k_rank_keys(const int32_t *__restrict__ deg, int64_t n, int nb,
                            uint64_t *__restrict__ keys) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    keys[v] = ((uint64_t)deg[v] << nb) | (uint64_t)v;
}

__global__ void k_rank_finish(const uint64_t *__restrict__ sorted, int64_t n, int nb,
                              int32_t *__restrict__ perm, int32_t *__restrict__ rank) {
  const uint64_t mask = (1ull << nb) - 1ull;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = (int32_t)(sorted[r] & mask);
    perm[r] = v;
    rank[v] = (int32_t)r;
  }
}

// Batch handles: graph of each position (the graph owning perm[r]).
__global__ void k_graph_of_position(const int32_t *__restrict__ perm, int64_t n,
                                    const int64_t *__restrict__ voff, int ng,
                                    int32_t *__restrict__ gid) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = perm[r];
    int lo = 0, hi = ng;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (voff[mid] <= v) lo = mid; else hi = mid;
    }
    gid[r] = lo;
  }
}

// a4 keys: each edge {a,b} as (min(rank) << nb) | max(rank).
__global__ void k_orient_keys(const uint64_t *__restrict__ ukeys, int64_t m, int nb,
                              const int32_t *__restrict__ rank, uint64_t *__restrict__ okeys) {
  const uint64_t mask = (1ull << nb) - 1ull;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = ukeys[e];
    uint64_t ra = (uint64_t)rank[k >> nb], rb = (uint64_t)rank[k & mask];
    okeys[e] = ra < rb ? (ra << nb) | rb : (rb << nb) | ra;
  }
}

// Oriented CSR from the sorted oriented keys: colidx, the source of each
// edge, and the row lengths (counted into rowptr[src], warp-aggregated; a scan
// turns them into offsets).
__global__ void k_csr_finish(const uint64_t *__restrict__ okeys, int64_t m, int nb,
                             int32_t *__restrict__ colidx, int32_t *__restrict__ esrc,
                             unsigned long long *__restrict__ rowlen) {
  const uint64_t mask = (1ull << nb) - 1ull;
  const unsigned lane = threadIdx.x & 31u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m; base += stride) {
    const int64_t e = base + threadIdx.x;
    const bool valid = e < m;
    int64_t s = -1;
    if (valid) {
      uint64_t k = okeys[e];
      s = (int64_t)(k >> nb);
      colidx[e] = (int32_t)(k & mask);
      esrc[e] = (int32_t)s;
    }
    unsigned peers = __match_any_sync(0xffffffffu, s);
    if (valid && lane == (unsigned)(__ffs(peers) - 1))
      atomicAdd(&rowlen[s], (unsigned long long)__popc(peers));
  }
}

// ------------------------------------------------------------------------
// Symmetric input with sorted rows (every edge listed under both endpoints,
// each row ascending): the canonical edges of row u are its entries above u,
// each counted once, so no global sort is needed.

constexpr int SEG_CAP = 2048;  // longest oriented row sorted in shared memory

__device__ __forceinline__ int64_t row_of_first(const int64_t *rowptr, int64_t n, int64_t target,
                                                int64_t lo_hint, int64_t hi_hint) {
  int64_t lo = lo_hint, hi = hi_hint;  // rowptr[lo] <= target
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) >> 1;
    if (rowptr[mid] <= target) lo = mid; else hi = mid;
  }
  return lo;
}

constexpr int SP_NT = 256;
constexpr int SP_ITEMS = 8;
constexpr int SP_TILE = SP_NT * SP_ITEMS;

// Row of the first entry of every tile of SP_TILE entries (and of the last
// entry, in the final slot): the row windows of the per-entry passes.
__global__ void k_tile_rows(const int64_t *__restrict__ rowptr, int64_t n, int64_t nnz,
                            int64_t ntiles, int64_t *__restrict__ rows) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= ntiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t target = t < ntiles ? t * SP_TILE : nnz - 1;
    rows[t] = row_of_first(rowptr, n, target, 0, n);
  }
}

// Pass over the entries: thread t of a tile owns entries [t*8, t*8+8) and walks
// their rows forward from one search inside the tile's row window; the counts
// of a row are added once per thread. MODE 0:
// degree of u += first copies of v != u, flag unsorted rows and out-of-range
// ids. MODE 1: out-degree at rank(u) += first copies with rank(v) > rank(u).
// MODE 2: scatter rank(v) into row rank(u) (any order; rows are sorted after;
// the rows' sources are written afterwards by k_fill_esrc, with coalesced stores).
// When rr is given, MODE 1 also stores each entry's rank(v) when the entry is
// such an upward first copy (else -1), and MODE 2 reads it back in order
// instead of gathering rank(v) a second time.
// For a batch (voff != nullptr), the entries of a row of graph g are local ids
// in [0, voff[g+1] - voff[g]), shifted here by voff[g].
template <int MODE>
__global__ void __launch_bounds__(SP_NT) k_sym_pass(const int64_t *__restrict__ rowptr,
                                                    const int32_t *__restrict__ colidx, int64_t n,
                                                    int64_t nnz,
                                                    const int64_t *__restrict__ tile_rows,
                                                    int32_t *__restrict__ deg,
                                                    const int32_t *__restrict__ rank,
                                                    unsigned long long *__restrict__ dplus,
                                                    const int64_t *__restrict__ rowptr_o,
                                                    unsigned int *__restrict__ cursor,
                                                    int32_t *__restrict__ colidx_o,
                                                    int32_t *__restrict__ err,
                                                    const int64_t *__restrict__ voff, int ng,
                                                    int32_t *__restrict__ rr) {
  const unsigned lane = threadIdx.x & 31u;
  const int64_t ntiles = (nnz + SP_TILE - 1) / SP_TILE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t t0 = tile * SP_TILE;
    const int64_t t1 = t0 + SP_TILE < nnz ? t0 + SP_TILE : nnz;
    const int64_t rlo = tile_rows[tile], rhi = tile_rows[tile + 1];
    const int64_t first = t0 + (int64_t)threadIdx.x * SP_ITEMS;
    int64_t u = first < t1 ? row_of_first(rowptr, n, first, rlo, rhi + 1) : rlo;
    int64_t row_end = rowptr[u + 1];
    int32_t ru = MODE > 0 ? rank[u] : 0;
    int gi = 0;
    int64_t gbase = 0, gend = n;
    if (voff) {
      int lo = 0, hi = ng;  // last graph with voff[lo] <= u
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (voff[mid] <= u) lo = mid; else hi = mid;
      }
      gi = lo;
      gbase = voff[gi];
      gend = voff[gi + 1];
    }
    // key of each item: MODE 0 its row u when it is the first copy of a
    // neighbour != u; MODE 1/2 rank(u) when it is such a copy and points up;
    // else -1. Keys >= 0 never decrease along a thread's items (rows ascend), so
    // equal keys form one group per row and each group costs one atomic.
    int64_t key[SP_ITEMS];
    int32_t val[SP_ITEMS];  // MODE 2: rank(v)
    int32_t up[SP_ITEMS];   // MODE 1: the entry's upward rank, else -1 (stored in rr)
#pragma unroll
    for (int i = 0; i < SP_ITEMS; ++i) {
      const int64_t e = first + i;
      key[i] = -1;
      val[i] = 0;
      up[i] = -1;
      if (e < t1) {
        while (e >= row_end) {  // next non-empty row
          ++u;
          row_end = rowptr[u + 1];
          if (MODE > 0) ru = rank[u];
        }
        if (MODE == 2 && rr) {  // the upward rank stored by MODE 1
          const int32_t rv = rr[e];
          if (rv >= 0) {
            key[i] = ru;
            val[i] = rv;
          }
          continue;
        }
        if (voff) {
          while (u >= gend && gi + 1 < ng) {
            ++gi;
            gbase = voff[gi];
            gend = voff[gi + 1];
          }
        }
        const int32_t vl = colidx[e];  // local to the row's graph
        const bool first_in_row = e == rowptr[u];
        const int32_t prev = first_in_row ? -1 : colidx[e - 1];
        const bool in_range = vl >= 0 && (int64_t)vl < gend - gbase;
        if (MODE == 0) {
          if (!in_range) atomicOr(err, 2);
          else if (!first_in_row && prev > vl) atomicOr(err, 4);
        }
        const int32_t v = in_range ? (int32_t)(vl + gbase) : 0;
        const bool head = in_range && v != u && (first_in_row || prev != vl);
        if (MODE == 0) {
          key[i] = head ? u : -1;
        } else {
          const int32_t rv = head ? rank[v] : -1;
          if (head && rv > ru) key[i] = ru;
          val[i] = rv;
          if (MODE == 1) up[i] = head && rv > ru ? rv : -1;
        }
      }
    }
    if (MODE == 1 && rr) {
      // rr + first is 32-byte aligned (first is a multiple of 8 entries)
      if (first + SP_ITEMS <= t1) {
        int4 *d = reinterpret_cast<int4 *>(rr + first);
        d[0] = make_int4(up[0], up[1], up[2], up[3]);
        d[1] = make_int4(up[4], up[5], up[6], up[7]);
      } else {
#pragma unroll
        for (int i = 0; i < SP_ITEMS; ++i)
          if (first + i < t1) rr[first + i] = up[i];
      }
    }
    if (MODE < 2) {
      int64_t cur = -1;
      unsigned cnt = 0;
      int groups = 0;
#pragma unroll
      for (int i = 0; i < SP_ITEMS; ++i) {
        if (key[i] >= 0 && key[i] != cur) {
          if (cur >= 0) {
            if (MODE == 0) atomicAdd(&deg[cur], (int)cnt);
            else atomicAdd(&dplus[cur], (unsigned long long)cnt);
          }
          cur = key[i];
          cnt = 0;
          ++groups;
        }
        if (key[i] >= 0) ++cnt;
      }
      // a warp inside one long row (a hub's) adds once for all its lanes
      const int64_t cur0 = __shfl_sync(0xffffffffu, cur, 0);
      if (__all_sync(0xffffffffu, groups == 1 && cur == cur0)) {
        const unsigned tot = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) {
          if (MODE == 0) atomicAdd(&deg[cur0], (int)tot);
          else atomicAdd(&dplus[cur0], (unsigned long long)tot);
        }
      } else if (cur >= 0) {
        if (MODE == 0) atomicAdd(&deg[cur], (int)cnt);
        else atomicAdd(&dplus[cur], (unsigned long long)cnt);
      }
    } else {
      int64_t cur = -1, pos = 0;
#pragma unroll
      for (int i = 0; i < SP_ITEMS; ++i) {
        if (key[i] >= 0) {
          if (key[i] != cur) {  // first item of a group: reserve the group's slots
            cur = key[i];
            unsigned c = 0;
#pragma unroll
            for (int j = i; j < SP_ITEMS; ++j) c += key[j] == cur ? 1u : 0u;
            pos = rowptr_o[cur] + (int64_t)atomicAdd(&cursor[cur], c);
          }
          colidx_o[pos] = val[i];
          ++pos;
        }
      }
    }
  }
}

// esrc[x] = the row of position x, for every position of the oriented CSR.
// A warp takes 32 rows: lane j holds the start of row r0 + j, and each
// position of the rows' span finds its row by a search over the lanes, so
// the stores are coalesced whatever the row lengths.
__global__ void k_fill_esrc(const int64_t *__restrict__ rowptr, int64_t n,
                            int32_t *__restrict__ esrc) {
  const unsigned lane = threadIdx.x & 31u;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; r0 < n;
       r0 += nwarps * 32) {
    const int64_t rj = r0 + lane < n ? r0 + lane : n;
    const int64_t start_j = rowptr[rj];
    const int64_t span_end = rowptr[r0 + 32 < n ? r0 + 32 : n];
    const int64_t span_start = __shfl_sync(0xffffffffu, start_j, 0);
    for (int64_t x0 = span_start; x0 < span_end; x0 += 32) {
      const int64_t x = x0 + lane;
      int j = 0;  // last lane whose row starts at or before x
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int64_t sj = __shfl_sync(0xffffffffu, start_j, j + step);
        if (sj <= x) j += step;
      }
      if (x < span_end) esrc[x] = (int32_t)(r0 + j);
    }
  }
}

// Oriented keys from the scattered (source, destination) pairs, for graphs
// with rows too long for k_sort_rows: one global sort orders them instead.
__global__ void k_pair_keys(const int32_t *__restrict__ esrc, const int32_t *__restrict__ colidx,
                            int64_t m, int nb, uint64_t *__restrict__ keys) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    keys[e] = ((uint64_t)esrc[e] << nb) | (uint64_t)colidx[e];
}

__global__ void k_pair_unkey(const uint64_t *__restrict__ keys, int64_t m, int nb,
                             int32_t *__restrict__ colidx) {
  const uint64_t mask = (1ull << nb) - 1ull;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    colidx[e] = (int32_t)(keys[e] & mask);
}

// Bitonic sort of 32*K values held by a warp in registers: element i of the
// sequence is x[i / 32] of lane i % 32. Exchanges at distance j < 32 go
// through shuffles, those at distance j >= 32 stay within a lane (slots r and
// r ^ j/32).
template <int K>
__device__ __forceinline__ void warp_bitonic(int32_t (&x)[K], unsigned lane) {
  constexpr int S = 32 * K;
#pragma unroll
  for (int k = 2; k <= S; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
#pragma unroll
        for (int r = 0; r < K; ++r) {
          const int q = r ^ (j >> 5);
          if (q > r) {
            const bool up = (((int)lane + 32 * r) & k) == 0;
            const int32_t a = x[r], b = x[q];
            const bool swap = up ? (a > b) : (a < b);
            x[r] = swap ? b : a;
            x[q] = swap ? a : b;
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < K; ++r) {
          const int32_t y = __shfl_xor_sync(0xffffffffu, x[r], j);
          const bool up = (((int)lane + 32 * r) & k) == 0;
          const bool lower = (lane & (unsigned)j) == 0;
          x[r] = (lower == up) ? min(x[r], y) : max(x[r], y);
        }
      }
    }
  }
}

template <int K>
__device__ __forceinline__ void sort_row_regs(int32_t *__restrict__ row, int len, unsigned lane) {
  int32_t x[K];
#pragma unroll
  for (int r = 0; r < K; ++r) {
    const int i = (int)lane + 32 * r;
    x[r] = i < len ? row[i] : INT_MAX;
  }
  warp_bitonic<K>(x, lane);
#pragma unroll
  for (int r = 0; r < K; ++r) {
    const int i = (int)lane + 32 * r;
    if (i < len) row[i] = x[r];
  }
}

// Bitonic network over W values held by one thread (all indices are
// compile-time constants, so the values stay in registers).
template <int W>
__device__ __forceinline__ void thread_bitonic(int32_t (&x)[W]) {
#pragma unroll
  for (int k = 2; k <= W; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int i = 0; i < W; ++i) {
        const int l = i ^ j;
        if (l > i) {
          const int32_t a = x[i], b = x[l];
          if ((i & k) == 0) {
            x[i] = min(a, b);
            x[l] = max(a, b);
          } else {
            x[i] = max(a, b);
            x[l] = min(a, b);
          }
        }
      }
    }
  }
}

template <int W>
__device__ __forceinline__ void sort_row_thread(int32_t *__restrict__ row, int len) {
  int32_t x[W];
#pragma unroll
  for (int i = 0; i < W; ++i) x[i] = i < len ? row[i] : INT_MAX;
  thread_bitonic<W>(x);
#pragma unroll
  for (int i = 0; i < W; ++i)
    if (i < len) row[i] = x[i];
}

// Sort every oriented row ascending. A warp takes 32 rows at a time: each
// lane sorts its own row when it has at most 16 entries (a register network
// of 8 or 16), then the warp sorts the longer rows one at a time: up to 1024
// in registers (bitonic network over shuffles and register slots, padded to
// 32 * 2^t), longer ones (up to SEG_CAP) in the warp's shared memory.
constexpr int SR_WARPS = 4;
constexpr int SR_SMALL = 16;

__global__ void __launch_bounds__(SR_WARPS * 32) k_sort_rows(const int64_t *__restrict__ rowptr,
                                                             int64_t n,
                                                             int32_t *__restrict__ colidx) {
  __shared__ int32_t buf[SR_WARPS][SEG_CAP];
  const unsigned lane = threadIdx.x & 31u;
  const int warp = threadIdx.x >> 5;
  int32_t *sm = buf[warp];
  // rows are dealt round-robin over the warps (row r to warp r mod W), so that
  // runs of long rows, which the degree order keeps together, spread evenly
  const int64_t nwarps = (int64_t)gridDim.x * SR_WARPS;
  const int64_t gw = (int64_t)blockIdx.x * SR_WARPS + warp;
  for (int64_t t0 = 0; gw + nwarps * t0 < n; t0 += 32) {
    const int64_t r = gw + nwarps * (t0 + lane);
    int64_t b = 0;
    int len = 0;
    if (r < n) {
      b = rowptr[r];
      len = (int)(rowptr[r + 1] - b);
    }
    const bool small = len > 1 && len <= SR_SMALL;
    const int small_max = __reduce_max_sync(0xffffffffu, small ? len : 0);
    if (small_max > 0) {
      if (small_max <= 8) {
        if (small) sort_row_thread<8>(colidx + b, len);
      } else {
        if (small) sort_row_thread<16>(colidx + b, len);
      }
    }
    unsigned big = __ballot_sync(0xffffffffu, len > SR_SMALL);
    while (big) {
      const int src = __ffs(big) - 1;
      big &= big - 1;
      const int64_t bb = __shfl_sync(0xffffffffu, b, src);
      const int blen = __shfl_sync(0xffffffffu, len, src);
      int32_t *row = colidx + bb;
      if (blen <= 32) {
        sort_row_regs<1>(row, blen, lane);
      } else if (blen <= 64) {
        sort_row_regs<2>(row, blen, lane);
      } else if (blen <= 128) {
        sort_row_regs<4>(row, blen, lane);
      } else if (blen <= 256) {
        sort_row_regs<8>(row, blen, lane);
      } else if (blen <= 512) {
        sort_row_regs<16>(row, blen, lane);
      } else if (blen <= 1024) {
        sort_row_regs<32>(row, blen, lane);
      } else {
        int size = 64;
        while (size < blen) size <<= 1;
        for (int i = lane; i < size; i += 32) sm[i] = i < blen ? row[i] : INT_MAX;
        __syncwarp();
        for (int k = 2; k <= size; k <<= 1)
          for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < size; i += 32) {
              const int l = i ^ j;
              if (l > i) {
                const int32_t a = sm[i], c = sm[l];
                const bool up = (i & k) == 0;
                if ((a > c) == up) {
                  sm[i] = c;
                  sm[l] = a;
                }
              }
            }
            __syncwarp();
          }
        for (int i = lane; i < blen; i += 32) row[i] = sm[i];
        __syncwarp();
      }
    }
  }
}

}  // namespace

// a1-a4 for symmetric input with sorted rows. Sets *applied = false (and does
// nothing lasting) when some row turns out unsorted.
static bbtc_status prepare_sym_sorted(bbtc_graph *g, const int64_t *d_rowptr,
                                      const int32_t *d_colidx, int64_t nnz, int32_t *err,
                                      bool *applied) {
  cudaStream_t s = g->stream;
  const int64_t n = g->n;
  const int nb = g->nb;
  *applied = false;
  Scratch scratch(s);
  BBTC_TRY(dalloc_n(&g->deg, n, s));
  g->bytes += (uint64_t)(n > 0 ? n : 1) * sizeof(int32_t);
  BBTC_CUDA(cudaMemsetAsync(g->deg, 0, sizeof(int32_t) * (size_t)(n > 0 ? n : 1), s));
  const int64_t ntiles = (nnz + SP_TILE - 1) / SP_TILE;
  int64_t *tile_rows = nullptr;
  BBTC_TRY(scratch.get(&tile_rows, ntiles + 1));
  k_tile_rows<<<grid_for(ntiles + 1, 256, 16), 256, 0, s>>>(d_rowptr, n, nnz, ntiles, tile_rows);
  BBTC_LAUNCH_CHECK();
  const unsigned grid = grid_for(ntiles, 1, 32);
  k_sym_pass<0><<<grid, SP_NT, 0, s>>>(d_rowptr, d_colidx, n, nnz, tile_rows, g->deg, nullptr,
                                       nullptr, nullptr, nullptr, nullptr, err, g->voff, g->ng,
                                       nullptr);
  BBTC_LAUNCH_CHECK();
  int32_t herr = 0;
  BBTC_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  BBTC_CUDA(cudaStreamSynchronize(s));
  if (herr & 1) {
    set_error("bbtc_graph_create: rowptr[0] != 0 or rowptr decreases");
    return BBTC_EINVAL;
  }
  if (herr & 2) {
    set_error("bbtc_graph_create: colidx entry outside [0, n)");
    return BBTC_EINVAL;
  }
  if (herr & 4) return BBTC_OK;  // unsorted rows: the general path takes over
  *applied = true;

  // a3: order by (degree, id)
  int32_t *rank = nullptr, *dmax = nullptr;
  uint64_t *rk = nullptr, *rk_alt = nullptr;
  BBTC_TRY(scratch.get(&rank, n));
  BBTC_TRY(scratch.get(&dmax, 1));
  BBTC_TRY(scratch.get(&rk, n));
  BBTC_TRY(scratch.get(&rk_alt, n));
  BBTC_TRY(dalloc_n(&g->perm, n, s));
  g->bytes += (uint64_t)n * sizeof(int32_t);
  BBTC_TRY(reduce_max_i32(g->deg, n, dmax, s));
  int32_t hdmax = 0;
  BBTC_CUDA(cudaMemcpyAsync(&hdmax, dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  BBTC_CUDA(cudaStreamSynchronize(s));
  g->deg_max = hdmax;
  k_rank_keys<<<grid_for(n, 256, 16), 256, 0, s>>>(g->deg, n, nb, rk);
  BBTC_LAUNCH_CHECK();
  bool in_alt = false;
  BBTC_TRY(radix_sort(rk, rk_alt, nullptr, nullptr, n, 0, nb + ceil_log2_u64((uint64_t)hdmax + 1),
                      s, &in_alt));
  k_rank_finish<<<grid_for(n, 256, 16), 256, 0, s>>>(in_alt ? rk_alt : rk, n, nb, g->perm, rank);
  BBTC_LAUNCH_CHECK();
  if (g->voff) {
    BBTC_TRY(dalloc_n(&g->gid, n, s));
    g->bytes += (uint64_t)n * sizeof(int32_t);
    k_graph_of_position<<<grid_for(n, 256, 16), 256, 0, s>>>(g->perm, n, g->voff, g->ng, g->gid);
    BBTC_LAUNCH_CHECK();
  }

  // a4: out-degrees by rank, offsets, scatter, per-row sort
  BBTC_TRY(dalloc_n(&g->rowptr, n + 1, s));
  g->bytes += (uint64_t)(n + 1) * 8;
  BBTC_CUDA(cudaMemsetAsync(g->rowptr, 0, sizeof(int64_t) * (size_t)(n + 1), s));
  // each entry's upward rank, kept for the scatter pass (it is skipped, and the
  // scatter gathers the ranks again, when the nnz-entry array does not fit)
  int32_t *rr = nullptr;
  if (dalloc_n(&rr, nnz, s) != BBTC_OK) {
    clear_error();
    rr = nullptr;
  }
  struct FreeRR {
    int32_t *p;
    cudaStream_t s;
    ~FreeRR() { dfree(p, s); }
  } free_rr{rr, s};
  k_sym_pass<1><<<grid, SP_NT, 0, s>>>(d_rowptr, d_colidx, n, nnz, tile_rows, nullptr, rank,
                                       reinterpret_cast<unsigned long long *>(g->rowptr),
                                       nullptr, nullptr, nullptr, err, g->voff, g->ng, rr);
  BBTC_LAUNCH_CHECK();
  int64_t *stats = nullptr;
  BBTC_TRY(scratch.get(&stats, 2));
  BBTC_TRY(reduce_max_i64(g->rowptr, n, &stats[0], s));
  BBTC_TRY(exclusive_scan_u64(reinterpret_cast<uint64_t *>(g->rowptr),
                              reinterpret_cast<uint64_t *>(g->rowptr), n + 1, s));
  int64_t h[2] = {0, 0};
  BBTC_CUDA(cudaMemcpyAsync(&h[0], &stats[0], sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  BBTC_CUDA(cudaMemcpyAsync(&h[1], g->rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  BBTC_CUDA(cudaStreamSynchronize(s));
  g->dplus_max = h[0];
  const int64_t m = h[1];
  if (m > 0xFFFFFFFFLL) {
    set_error("bbtc_graph_create: %lld simple edges exceed 2^32 - 1", (long long)m);
    return BBTC_EINVAL;
  }
  g->m = m;
  BBTC_TRY(dalloc_n(&g->colidx, padded_columns(m), s));
  BBTC_TRY(dalloc_n(&g->esrc, m, s));
  g->bytes += (uint64_t)(m > 0 ? m : 1) * 8;
  unsigned int *cursor = nullptr;
  BBTC_TRY(scratch.get(&cursor, n));
  BBTC_CUDA(cudaMemsetAsync(cursor, 0, sizeof(unsigned int) * (size_t)(n > 0 ? n : 1), s));
  k_sym_pass<2><<<grid, SP_NT, 0, s>>>(d_rowptr, d_colidx, n, nnz, tile_rows, nullptr, rank,
                                       nullptr, g->rowptr, cursor, g->colidx, err, g->voff, g->ng,
                                       rr);
  BBTC_LAUNCH_CHECK();
  if (m > 0) {
    k_fill_esrc<<<grid_for((n + 31) / 32 * 32, 256, 16), 256, 0, s>>>(g->rowptr, n, g->esrc);
    BBTC_LAUNCH_CHECK();
  }
  if (m > 0) {
    if (g->dplus_max <= SEG_CAP) {
      k_sort_rows<<<grid_for((n + 31) / 32, SR_WARPS, 64), SR_WARPS * 32, 0, s>>>(g->rowptr, n,
                                                                                g->colidx);
      BBTC_LAUNCH_CHECK();
    } else {
      uint64_t *ok = nullptr, *ok_alt = nullptr;
      BBTC_TRY(scratch.get(&ok, m));
      BBTC_TRY(scratch.get(&ok_alt, m));
      k_pair_keys<<<grid_for(m, 256, 32), 256, 0, s>>>(g->esrc, g->colidx, m, nb, ok);
      BBTC_LAUNCH_CHECK();
      BBTC_TRY(radix_sort(ok, ok_alt, nullptr, nullptr, m, 0, 2 * nb, s, &in_alt));
      k_pair_unkey<<<grid_for(m, 256, 32), 256, 0, s>>>(in_alt ? ok_alt : ok, m, nb, g->colidx);
      BBTC_LAUNCH_CHECK();
    }
  }
  BBTC_CUDA(cudaStreamSynchronize(s));
  return BBTC_OK;
}

bbtc_status prepare_graph(bbtc_graph *g, const int64_t *d_rowptr, const int32_t *d_colidx,
                          int64_t nnz, bool symmetric) {
  cudaStream_t s = g->stream;
  const int64_t n = g->n;
  const int nb = ceil_log2_u64((uint64_t)n) < 1 ? 1 : ceil_log2_u64((uint64_t)n);
  g->nb = nb;
  Scratch scratch(s);
  int32_t *err = nullptr;
  int64_t *hstats = nullptr;  // device: [0]=m, [1]=deg_max, [2]=err
  BBTC_TRY(scratch.get(&err, 1));
  BBTC_TRY(scratch.get(&hstats, 3));
  BBTC_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), s));

  // ---- validation of rowptr (colidx range is checked while emitting keys)
  if (n > 0) {
    k_validate_rowptr<<<grid_for(n, 256, 8), 256, 0, s>>>(d_rowptr, n, err);
    BBTC_LAUNCH_CHECK();
  }

  // ---- symmetric input with sorted rows: per-row path, no global sort
  if (symmetric && nnz > 0) {
    bool applied = false;
    BBTC_TRY(prepare_sym_sorted(g, d_rowptr, d_colidx, nnz, err, &applied));
    if (applied) return BBTC_OK;
    BBTC_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), s));  // fall through: general path
  }

  // ---- a1: canonical keys (compacted), sort, unique; a2: degree
  // (no key equals the all-ones value: it would need min == max)
  const uint64_t sentinel = (nb * 2 >= 64) ? ~0ull : ((1ull << (2 * nb)) - 1ull);
  uint64_t *ka = nullptr, *kb = nullptr;
  int64_t nkeys = 0;
  if (nnz > 0) {
    const int64_t ntiles = (nnz + EK_TILE - 1) / EK_TILE;
    uint64_t *tile_count = nullptr;
    BBTC_TRY(scratch.get(&tile_count, ntiles + 1));
    const unsigned grid = grid_for(ntiles, 1, 64);
    k_emit_keys<false><<<grid, EK_NT, 0, s>>>(d_rowptr, d_colidx, n, nnz, nb, symmetric,
                                               g->voff, g->ng, tile_count, nullptr, err);
    BBTC_LAUNCH_CHECK();
    BBTC_TRY(exclusive_scan_u64(tile_count, tile_count, ntiles + 1, s));
    BBTC_CUDA(cudaMemcpyAsync(&hstats[0], &tile_count[ntiles], sizeof(int64_t),
                              cudaMemcpyDeviceToDevice, s));
    int64_t h[1] = {0};
    int32_t herr = 0;
    BBTC_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BBTC_CUDA(cudaMemcpyAsync(h, &hstats[0], sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BBTC_CUDA(cudaStreamSynchronize(s));
    if (herr & 1) {
      set_error("bbtc_graph_create: rowptr[0] != 0 or rowptr decreases");
      return BBTC_EINVAL;
    }
    if (herr & 2) {
      set_error("bbtc_graph_create: colidx entry outside [0, n)");
      return BBTC_EINVAL;
    }
    nkeys = h[0];
    const int64_t kcap = nkeys > n ? nkeys : n;  // the buffers also take the n rank keys
    BBTC_TRY(scratch.get(&ka, kcap));
    BBTC_TRY(scratch.get(&kb, kcap));
    k_emit_keys<true><<<grid, EK_NT, 0, s>>>(d_rowptr, d_colidx, n, nnz, nb, symmetric,
                                              g->voff, g->ng, tile_count, ka, err);
    BBTC_LAUNCH_CHECK();
  } else {
    int32_t herr = 0;
    BBTC_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BBTC_CUDA(cudaStreamSynchronize(s));
    if (herr & 1) {
      set_error("bbtc_graph_create: rowptr[0] != 0 or rowptr decreases");
      return BBTC_EINVAL;
    }
    BBTC_TRY(scratch.get(&ka, n));
    BBTC_TRY(scratch.get(&kb, n));
  }
  bool in_alt = false;
  BBTC_TRY(radix_sort(ka, kb, nullptr, nullptr, nkeys, 0, 2 * nb, s, &in_alt));
  uint64_t *sorted = in_alt ? kb : ka;
  uint64_t *ukeys = in_alt ? ka : kb;

  if (!g->deg) {
    BBTC_TRY(dalloc_n(&g->deg, n, s));
    g->bytes += (uint64_t)(n > 0 ? n : 1) * sizeof(int32_t);
  }
  BBTC_CUDA(cudaMemsetAsync(g->deg, 0, sizeof(int32_t) * (size_t)(n > 0 ? n : 1), s));
  int64_t m = 0;
  if (nkeys > 0) {
    const int64_t nblk = (nkeys + UQ_TILE - 1) / UQ_TILE;
    uint64_t *boff = nullptr;
    BBTC_TRY(scratch.get(&boff, nblk + 1));
    k_unique_count<<<(unsigned)nblk, UQ_NT, 0, s>>>(sorted, nkeys, sentinel, boff);
    BBTC_LAUNCH_CHECK();
    BBTC_TRY(exclusive_scan_u64(boff, boff, nblk + 1, s));  // boff[nblk] = total
    k_unique_write<<<(unsigned)nblk, UQ_NT, 0, s>>>(sorted, nkeys, sentinel, boff, nb, ukeys,
                                                     g->deg);
    BBTC_LAUNCH_CHECK();
    BBTC_CUDA(cudaMemcpyAsync(&hstats[0], &boff[nblk], sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  } else {
    BBTC_CUDA(cudaMemsetAsync(&hstats[0], 0, sizeof(int64_t), s));
  }
  int32_t *dmax = nullptr;
  BBTC_TRY(scratch.get(&dmax, 1));
  BBTC_TRY(reduce_max_i32(g->deg, n, dmax, s));
  int64_t stats[2] = {0, 0};
  int32_t hdmax = 0;
  BBTC_CUDA(cudaMemcpyAsync(&stats[0], &hstats[0], sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  BBTC_CUDA(cudaMemcpyAsync(&hdmax, dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  BBTC_CUDA(cudaStreamSynchronize(s));
  m = stats[0];
  if (m > 0xFFFFFFFFLL) {
    set_error("bbtc_graph_create: %lld simple edges exceed 2^32 - 1", (long long)m);
    return BBTC_EINVAL;
  }
  g->m = m;
  g->deg_max = hdmax;

  // ---- a3: order by (degree, id)
  int32_t *rank = nullptr;
  BBTC_TRY(scratch.get(&rank, n));
  BBTC_TRY(dalloc_n(&g->perm, n, s));
  g->bytes += (uint64_t)(n > 0 ? n : 1) * sizeof(int32_t);
  // ukeys (m) must survive the rank sort: rank keys go to the sort buffer that
  // does not hold ukeys, plus a separate alternate buffer.
  uint64_t *rk = sorted;  // free now (its distinct keys were copied to ukeys)
  uint64_t *rk_alt = nullptr;
  BBTC_TRY(scratch.get(&rk_alt, n));
  if (n > 0) {
    k_rank_keys<<<grid_for(n, 256, 16), 256, 0, s>>>(g->deg, n, nb, rk);
    BBTC_LAUNCH_CHECK();
    int dbits = ceil_log2_u64((uint64_t)hdmax + 1);
    BBTC_TRY(radix_sort(rk, rk_alt, nullptr, nullptr, n, 0, nb + dbits, s, &in_alt));
    k_rank_finish<<<grid_for(n, 256, 16), 256, 0, s>>>(in_alt ? rk_alt : rk, n, nb, g->perm,
                                                        rank);
    BBTC_LAUNCH_CHECK();
    if (g->voff) {
      BBTC_TRY(dalloc_n(&g->gid, n, s));
      g->bytes += (uint64_t)n * sizeof(int32_t);
      k_graph_of_position<<<grid_for(n, 256, 16), 256, 0, s>>>(g->perm, n, g->voff, g->ng,
                                                              g->gid);
      BBTC_LAUNCH_CHECK();
    }
  }

  // ---- a4: orient and build the oriented CSR
  BBTC_TRY(dalloc_n(&g->rowptr, n + 1, s));
  BBTC_TRY(dalloc_n(&g->colidx, padded_columns(m), s));
  BBTC_TRY(dalloc_n(&g->esrc, m, s));
  g->bytes += (uint64_t)(n + 1) * 8 + (uint64_t)(m > 0 ? m : 1) * 8;
  BBTC_CUDA(cudaMemsetAsync(g->rowptr, 0, sizeof(int64_t) * (size_t)(n + 1), s));
  if (m > 0) {
    uint64_t *ok = sorted;  // rank keys are consumed; reuse
    uint64_t *ok_alt = nullptr;
    BBTC_TRY(scratch.get(&ok_alt, m));
    k_orient_keys<<<grid_for(m, 256, 32), 256, 0, s>>>(ukeys, m, nb, rank, ok);
    BBTC_LAUNCH_CHECK();
    BBTC_TRY(radix_sort(ok, ok_alt, nullptr, nullptr, m, 0, 2 * nb, s, &in_alt));
    k_csr_finish<<<grid_for(m, 256, 32), 256, 0, s>>>(
        in_alt ? ok_alt : ok, m, nb, g->colidx, g->esrc,
        reinterpret_cast<unsigned long long *>(g->rowptr));
    BBTC_LAUNCH_CHECK();
  }
  // rowptr holds the row lengths: their maximum is d+_max, their scan the offsets
  BBTC_TRY(reduce_max_i64(g->rowptr, n, &hstats[1], s));
  BBTC_CUDA(cudaMemcpyAsync(&stats[1], &hstats[1], sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  BBTC_TRY(exclusive_scan_u64(reinterpret_cast<uint64_t *>(g->rowptr),
                              reinterpret_cast<uint64_t *>(g->rowptr), n + 1, s));
  BBTC_CUDA(cudaStreamSynchronize(s));
  g->dplus_max = n > 0 ? stats[1] : 0;
  return BBTC_OK;
}

}  // namespace bbtc
