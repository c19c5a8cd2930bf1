// plan.cu -- per-p planning steps of bbTC (run by bbtc_count, cached per p):
//   a5 partition: contiguous cuts of the degree order balanced on oriented
//      edges (Sec. 2 vertex partition V^p; Sec. 4.1 symmetric partition),
//      or the probe-based partition of partition.cu
//   a6 blocks G_ij = {(u,v) : u in V_i, v in V_j} (Sec. 2), materialised as
//      the in-edges of each v grouped by the part of their source, so that a
//      block's edges are one contiguous, destination-ordered range
//   a7 task composition: all (i,j,k), i <= j <= k (Sec. 4.2, Alg. 4)
//   a8 ExecTime estimate and non-increasing order (Sec. 5), split into work
//      items of at most `chunk` in-edges each
#include <new>

#include "graph.cuh"
#include "primitives.cuh"

namespace bbtc {

namespace {

constexpr int MAXP = 64;

// c_0 = 0, c_p = n, c_i = min{ r : rowptr[r] >= ceil(i*m/p) }.
__global__ void k_cuts(const int64_t *__restrict__ rowptr, int64_t n, int p,
                       int32_t *__restrict__ cuts) {
  const int i = threadIdx.x;
  if (i > p) return;
  const int64_t m = rowptr[n];
  int32_t c;
  if (i == 0) {
    c = 0;
  } else if (i == p) {
    c = (int32_t)n;
  } else {
    int64_t target = ((int64_t)i * m + p - 1) / p;
    c = (int32_t)lower_bound_dev<int64_t, int64_t>(rowptr, 0, n + 1, target);
  }
  cuts[i] = c;
}

// In-edges of part a (the edges of rows V_a, positions [rowptr[c_a],
// rowptr[c_a+1]) of the oriented CSR) grouped by destination v: a counting
// sort on v - c_a. In degree order the hubs hold the top positions and
// receive most in-edges (on R-MAT, the top 8192 of 2 M vertices receive 65%),
// so one global counter per hub would serialise. Each CTA takes a contiguous
// share of the part's edges and counts destinations in the top IE_HUB
// positions in shared memory, adding to the global counters once per CTA.
// Counters are 32-bit (positions relative to the part's first edge). The
// scatter can run over slabs of at most IE_SLAB destinations (each pass reads
// all of the part's columns); slabs small enough for their counters to stay in
// L2 (16 M positions) measured slower on the Friendster-shaped graph (105 ms
// in four passes against 99 ms in one), so one slab covers every position.
constexpr int IE_NT = 256;
constexpr int IE_NT_S = 512;  // scatter CTAs: more threads to keep position atomics in flight
constexpr int IE_HUB = 8192;
constexpr int64_t IE_SLAB = 1ll << 31;

__device__ __forceinline__ void ie_share(int64_t e0, int64_t e1, int64_t *b0, int64_t *b1) {
  const int64_t per = (e1 - e0 + gridDim.x - 1) / gridDim.x;
  *b0 = e0 + (int64_t)blockIdx.x * per;
  *b1 = *b0 + per < e1 ? *b0 + per : e1;
}

// Step 1: count the edges into each destination.
__global__ void __launch_bounds__(IE_NT) k_inedge_count(const int64_t *__restrict__ rowptr,
                                                        const int32_t *__restrict__ colidx,
                                                        const int32_t *__restrict__ cuts, int a,
                                                        int64_t n, unsigned *__restrict__ hist) {
  __shared__ unsigned sm[IE_HUB];
  const int32_t c_a = cuts[a];
  const int64_t e0 = rowptr[c_a], e1 = rowptr[cuts[a + 1]];
  const int64_t hub0 = n - IE_HUB > c_a ? n - IE_HUB : c_a;  // positions >= hub0 on chip
  for (int i = threadIdx.x; i < IE_HUB; i += IE_NT) sm[i] = 0;
  __syncthreads();
  int64_t b0, b1;
  ie_share(e0, e1, &b0, &b1);
  for (int64_t e = b0 + threadIdx.x; e < b1; e += IE_NT) {
    const int32_t v = colidx[e];
    if (v >= hub0) atomicAdd(&sm[v - hub0], 1u);
    else atomicAdd(&hist[v - c_a], 1u);
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n - hub0; i += IE_NT)
    if (sm[i]) atomicAdd(&hist[hub0 - c_a + i], sm[i]);
}

// With one part every edge of the oriented graph is an in-edge of the part,
// and the count of position r is its in-degree: the undirected degree of its
// vertex minus its out-degree (the rest of its edges point down to it).
__global__ void k_indegree(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ perm,
                           const int32_t *__restrict__ deg, int64_t n,
                           unsigned *__restrict__ hist) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x)
    hist[r] = (unsigned)(deg[perm[r]] - (int32_t)(rowptr[r + 1] - rowptr[r]));
}

// 32-bit counts to 64-bit (for the scan), and the scanned offsets back to the
// 32-bit cursors of the scatter (offsets within a part are below 2^32).
__global__ void k_widen(const unsigned *__restrict__ in, int64_t count, uint64_t *__restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}
__global__ void k_narrow(const uint64_t *__restrict__ in, int64_t count, unsigned *__restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (unsigned)in[i];
}

// Step 2 (after an exclusive scan of the counts): the block offsets of part a,
// boff[a*(p+1)+j] = first in-edge of part a whose destination is >= c_j.
__global__ void k_inedge_offsets(const int64_t *__restrict__ rowptr,
                                 const int32_t *__restrict__ cuts, int a, int p,
                                 const unsigned long long *__restrict__ scan, int64_t bins,
                                 int64_t *__restrict__ boff) {
  const int j = threadIdx.x;
  if (j > p) return;
  const int32_t c_a = cuts[a];
  const int64_t e0 = rowptr[c_a], e1 = rowptr[cuts[a + 1]];
  int64_t off;
  if (j <= a) {
    off = e0;
  } else {
    const int64_t idx = (int64_t)cuts[j] - c_a;  // scan has bins = n - c_a entries
    off = idx < bins ? e0 + (int64_t)scan[idx] : e1;
  }
  boff[a * (p + 1) + j] = off;
}

// Step 3: scatter each edge of part a whose destination lies in the slab
// [v_lo, v_hi) to its destination's run, as one 16-byte record (source u,
// destination v, CSR position e, end f of u's run in v's block, from the
// split table row of u) so that each random write touches one sector; within
// a run the order of the sources is whatever the atomics give (counts do not
// depend on it). For the slab's top IE_HUB destinations the CTA first counts
// its share, reserves one range per destination with a single global atomic,
// and hands out positions inside it from shared memory.
__global__ void __launch_bounds__(IE_NT_S) k_inedge_scatter(const int64_t *__restrict__ rowptr,
                                                            const int32_t *__restrict__ colidx,
                                                            const int32_t *__restrict__ esrc,
                                                            const int32_t *__restrict__ cuts_g,
                                                            int a, int p, int64_t v_lo,
                                                            int64_t v_hi,
                                                            const uint32_t *__restrict__ spl_a,
                                                            unsigned *__restrict__ offs,
                                                            InEdge *__restrict__ rec) {
  __shared__ unsigned sm[IE_HUB];
  __shared__ int32_t cuts[MAXP + 1];
  for (int i = threadIdx.x; i <= p; i += IE_NT_S) cuts[i] = cuts_g[i];
  const int32_t c_a = cuts_g[a];
  const int64_t e0 = rowptr[c_a], e1 = rowptr[cuts_g[a + 1]];
  const int64_t hub0 = v_hi - IE_HUB > v_lo ? v_hi - IE_HUB : v_lo;
  for (int i = threadIdx.x; i < IE_HUB; i += IE_NT_S) sm[i] = 0;
  __syncthreads();
  int64_t b0, b1;
  ie_share(e0, e1, &b0, &b1);
  for (int64_t e = b0 + threadIdx.x; e < b1; e += IE_NT_S) {
    const int32_t v = colidx[e];
    if (v >= hub0 && v < v_hi) atomicAdd(&sm[v - hub0], 1u);
  }
  __syncthreads();
  // positions are relative to e0 and below 2^32
  for (int64_t i = threadIdx.x; i < v_hi - hub0; i += IE_NT_S)
    if (sm[i]) sm[i] = atomicAdd(&offs[hub0 - c_a + i], sm[i]);
  __syncthreads();
  // IE_ILP edges per thread per step: their position atomics are in flight together
  constexpr int IE_ILP = 4;
  for (int64_t e = b0 + threadIdx.x; e < b1; e += (int64_t)IE_NT_S * IE_ILP) {
    int32_t v[IE_ILP];
    uint64_t x[IE_ILP];
#pragma unroll
    for (int r = 0; r < IE_ILP; ++r) {
      const int64_t idx = e + (int64_t)r * IE_NT_S;
      v[r] = idx < b1 ? colidx[idx] : -1;
      if (v[r] < v_lo || v[r] >= v_hi) v[r] = -1;  // outside the slab (or past the share)
    }
#pragma unroll
    for (int r = 0; r < IE_ILP; ++r)
      if (v[r] >= 0)
        x[r] = v[r] >= hub0 ? (uint64_t)atomicAdd(&sm[v[r] - hub0], 1u)
                            : (uint64_t)atomicAdd(&offs[v[r] - c_a], 1u);
#pragma unroll
    for (int r = 0; r < IE_ILP; ++r) {
      const int64_t idx = e + (int64_t)r * IE_NT_S;
      if (v[r] >= 0) {
        const int32_t u = esrc[idx];
        const int b = part_of_dev(cuts, p, v[r]);  // >= a: v > u
        const uint32_t f = spl_a[(int64_t)(u - c_a) * (p - a + 1) + (b - a + 1)];
        rec[e0 + (int64_t)x[r]] = make_int4(u, v[r], (int32_t)(uint32_t)idx, (int32_t)f);
      }
    }
  }
}

// Two-phase in-edge build for large parts. A direct scatter writes each
// 16-byte record to a random slot: half a 32-byte sector, read and written
// back whole, with a random counter per edge (on the Friendster-shaped graph
// the scatter moves 4x its algorithmic bytes). Instead:
//  1. partition: each CTA takes tiles of IEB_T edges, builds their records,
//     buckets them in shared memory into IEB_B destination ranges of about
//     equal record count, reserves each bucket's share with one atomic and
//     writes it as one contiguous run into the bucket's own range of the
//     output positions (in a temporary array);
//  2. place: a grid-stride pass reads the temporary array in order and puts
//     each record at its destination's cursor. The CTAs move through the
//     buckets together, so the bucket being filled (tens of MB) and its
//     cursors stay in L2 and its lines go to HBM once, whole; the temporary
//     array is streamed with evict-first loads so it does not displace them.
constexpr int IEB_T = 4096;   // edges per partition tile
constexpr int IEB_NT = 512;   // threads of a partition CTA (8 edges each)
constexpr int IEB_B = 512;    // buckets (one per partition thread in the scan)
constexpr int64_t IEB_MIN_EDGES = 16ll << 20;  // smaller parts use the direct scatter
constexpr int IEB_LUT = 4096;  // entries of the partition's bucket lookup table
static_assert(IEB_NT == IEB_B && IEB_T == 8 * IEB_NT, "partition layout");

// Bucket b of part a holds the destinations [bnd[b], bnd[b+1]) (relative to
// c_a) whose in-edge offsets start in [ceil(b M / B), ceil((b+1) M / B)), M the
// part's edge count; their records take the output offsets [bstart[b],
// bstart[b+1]). scan holds the exclusive scan of the bins destinations' counts.
__global__ void k_ieb_bounds(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ cuts,
                             int a, const uint64_t *__restrict__ scan, int64_t bins,
                             int32_t *__restrict__ bnd, unsigned *__restrict__ bstart,
                             unsigned *__restrict__ bcur) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b > IEB_B) return;
  const int64_t M = rowptr[cuts[a + 1]] - rowptr[cuts[a]];
  int64_t idx = bins;
  if (b == 0) {
    idx = 0;
  } else if (b < IEB_B) {
    const uint64_t target = (uint64_t)((M * b + IEB_B - 1) / IEB_B);
    idx = lower_bound_dev<uint64_t, int64_t>(scan, 0, bins, target);
  }
  bnd[b] = (int32_t)idx;
  bstart[b] = (unsigned)(idx < bins ? scan[idx] : (uint64_t)M);
  if (b < IEB_B) bcur[b] = 0;
}

__global__ void __launch_bounds__(IEB_NT, 2)
    k_ieb_partition(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                    const int32_t *__restrict__ esrc, const int32_t *__restrict__ cuts_g, int a,
                    int p, const uint32_t *__restrict__ spl_a, const int32_t *__restrict__ bnd_g,
                    const unsigned *__restrict__ bstart, unsigned *__restrict__ bcur,
                    InEdge *__restrict__ tmp) {
  __shared__ int32_t bnd[IEB_B + 1];
  __shared__ unsigned cnt[IEB_B], loff[IEB_B], gbase[IEB_B];
  __shared__ unsigned scan_tmp[IEB_NT / 32 + 1];
  __shared__ int32_t cuts[MAXP + 1];
  __shared__ uint16_t sb[IEB_T];  // bucket of each staged slot
  // lut[k]: the bucket holding destination offset k << shift; a destination
  // in [k << shift, (k + 1) << shift) lies in buckets lut[k] .. lut[k + 1]
  __shared__ uint16_t lut[IEB_LUT + 1];
  extern __shared__ __align__(16) unsigned char ieb_smem[];
  InEdge *stage = reinterpret_cast<InEdge *>(ieb_smem);  // IEB_T records
  for (int i = threadIdx.x; i <= IEB_B; i += IEB_NT) bnd[i] = bnd_g[i];
  for (int i = threadIdx.x; i <= p; i += IEB_NT) cuts[i] = cuts_g[i];
  const int32_t c_a = cuts_g[a];
  const int64_t e0 = rowptr[c_a], e1 = rowptr[cuts_g[a + 1]];
  __syncthreads();
  int shift = 0;
  while (((int64_t)IEB_LUT << shift) < (int64_t)bnd[IEB_B]) ++shift;
  for (int k = threadIdx.x; k <= IEB_LUT; k += IEB_NT) {
    const int64_t x = (int64_t)k << shift;
    int lo = 0, hi = IEB_B;  // last bucket with bnd[lo] <= x
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (bnd[mid] <= x) lo = mid; else hi = mid;
    }
    lut[k] = (uint16_t)lo;
  }
  __syncthreads();
  // the (v, u) of the next tile's edges are loaded while this tile is bucketed
  int32_t pv[8], pu[8];
  const int64_t tstep = (int64_t)gridDim.x * IEB_T;
  auto load_tile = [&](int64_t tt0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t idx = tt0 + (int)threadIdx.x + k * IEB_NT;
      pv[k] = 0;
      pu[k] = 0;
      if (idx < e1) {
        pv[k] = colidx[idx];
        pu[k] = esrc[idx];
      }
    }
  };
  load_tile(e0 + (int64_t)blockIdx.x * IEB_T);
  for (int64_t t0 = e0 + (int64_t)blockIdx.x * IEB_T; t0 < e1; t0 += tstep) {
    const int nv = (int)(e1 - t0 < IEB_T ? e1 - t0 : IEB_T);
    int32_t cv[8], cu[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      cv[k] = pv[k];
      cu[k] = pu[k];
    }
    load_tile(t0 + tstep);
    cnt[threadIdx.x] = 0;
    __syncthreads();
    uint32_t fk[8];
    int bk[8];
    unsigned lr[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = (int)threadIdx.x + k * IEB_NT;
      bk[k] = -1;
      if (i < nv) {
        const int32_t v = cv[k];
        const int32_t u = cu[k];
        const int b = part_of_dev(cuts, p, v);  // >= a: v > u
        const uint32_t f = spl_a[(int64_t)(u - c_a) * (p - a + 1) + (b - a + 1)];
        fk[k] = f;
        const int32_t x = v - c_a;
        int lo = lut[x >> shift], hi = lut[(x >> shift) + 1] + 1;  // last bucket with bnd[lo] <= x
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (bnd[mid] <= x) lo = mid; else hi = mid;
        }
        bk[k] = lo;
        lr[k] = atomicAdd(&cnt[lo], 1u);
      }
    }
    __syncthreads();
    unsigned total = 0;
    const unsigned c = cnt[threadIdx.x];
    loff[threadIdx.x] = block_exclusive_scan<unsigned, IEB_NT>(c, scan_tmp, &total);
    if (c) gbase[threadIdx.x] = bstart[threadIdx.x] + atomicAdd(&bcur[threadIdx.x], c);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (bk[k] >= 0) {
        const unsigned slot = loff[bk[k]] + lr[k];
        const int64_t idx = t0 + (int)threadIdx.x + k * IEB_NT;  // the edge's CSR position
        stage[slot] = make_int4(cu[k], cv[k], (int32_t)(uint32_t)idx, (int32_t)fk[k]);
        sb[slot] = (uint16_t)bk[k];
      }
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += IEB_NT) {
      const int b = sb[i];
      tmp[e0 + (int64_t)gbase[b] + (i - (int)loff[b])] = stage[i];
    }
    __syncthreads();
  }
}

__global__ void k_ieb_place(const InEdge *__restrict__ tmp, const int64_t *__restrict__ rowptr,
                            const int32_t *__restrict__ cuts, int a, unsigned *__restrict__ cursor,
                            InEdge *__restrict__ rec) {
  const int32_t c_a = cuts[a];
  const int64_t e0 = rowptr[c_a], e1 = rowptr[cuts[a + 1]];
  constexpr int ILP = 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t x = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < e1; x += stride * ILP) {
    InEdge r[ILP];
    unsigned pos[ILP];
#pragma unroll
    for (int k = 0; k < ILP; ++k)
      if (x + k * stride < e1) r[k] = __ldcs(tmp + x + k * stride);  // read once: evict first
#pragma unroll
    for (int k = 0; k < ILP; ++k)
      if (x + k * stride < e1) pos[k] = atomicAdd(&cursor[r[k].y - c_a], 1u);
#pragma unroll
    for (int k = 0; k < ILP; ++k)
      if (x + k * stride < e1) rec[e0 + (int64_t)pos[k]] = r[k];
  }
}

// The split table of the resident blocks: for row u of part a (sorted,
// every entry above u, so in blocks a..p-1), the CSR positions where its runs
// in blocks a, a+1, ..., p-1 start, then its end.
__global__ void k_splits(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                         int64_t n, const int32_t *__restrict__ cuts_g, int p,
                         const int64_t *__restrict__ off_g, uint32_t *__restrict__ spl) {
  __shared__ int32_t cuts[MAXP + 1];
  __shared__ int64_t off[MAXP + 1];
  for (int i = threadIdx.x; i <= p; i += blockDim.x) {
    cuts[i] = cuts_g[i];
    off[i] = off_g[i];
  }
  __syncthreads();
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int a = part_of_dev(cuts, p, (int32_t)u);
    const int64_t r0 = rowptr[u], r1 = rowptr[u + 1];
    uint32_t *row = spl + off[a] + (u - cuts[a]) * (int64_t)(p - a + 1);
    row[0] = (uint32_t)r0;
    int64_t lo = r0;
    for (int b = a + 1; b < p; ++b) {
      lo = lower_bound_dev<int32_t, int64_t>(colidx, lo, r1, cuts[b]);
      row[b - a] = (uint32_t)lo;
    }
    row[p - a] = (uint32_t)r1;
  }
}

// In-edge positions from CSR positions to physical block positions: e maps
// through pos_of_edge, and the run end f to one past the mapped position of
// the run's last edge (f - 1 >= e lies in the same run).
__global__ void k_remap_positions(InEdge *__restrict__ ie, int64_t m,
                                  const uint32_t *__restrict__ pos_of_edge) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < m;
       x += (int64_t)gridDim.x * blockDim.x) {
    InEdge r = ie[x];
    r.z = (int32_t)pos_of_edge[(uint32_t)r.z];
    r.w = (int32_t)(pos_of_edge[(uint32_t)r.w - 1u] + 1u);
    ie[x] = r;
  }
}

// BCSR, step 1 (one thread per oriented edge e = (u, v)): the edge falls in
// block (part(u), part(v)) at row slot rpb[part(u)*p + part(v)] + (u - c_a).
// Count the edges of every slot (warp-aggregated: consecutive edges share
// slots) and record where each slot's run starts in the oriented CSR (rows
// are sorted, so a slot's edges are consecutive).
__global__ void k_bcsr_count(const int32_t *__restrict__ esrc,
                             const int32_t *__restrict__ colidx, int64_t m,
                             const int32_t *__restrict__ cuts_g, int p,
                             const int64_t *__restrict__ rpb_g,
                             unsigned long long *__restrict__ cnt,
                             uint32_t *__restrict__ start) {
  __shared__ int32_t cuts[MAXP + 1];
  __shared__ int64_t rpb[MAXP * MAXP];
  for (int i = threadIdx.x; i <= p; i += blockDim.x) cuts[i] = cuts_g[i];
  for (int i = threadIdx.x; i < p * p; i += blockDim.x) rpb[i] = rpb_g[i];
  __syncthreads();
  const unsigned lane = threadIdx.x & 31u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m; base += stride) {
    const int64_t e = base + threadIdx.x;
    int64_t slot = -1;
    if (e < m) {
      const int32_t u = esrc[e], v = colidx[e];
      const int a = part_of_dev(cuts, p, u), b = part_of_dev(cuts, p, v);
      slot = rpb[a * p + b] + (u - cuts[a]);
      const bool run_head = e == 0 || esrc[e - 1] != u || part_of_dev(cuts, p, colidx[e - 1]) != b;
      if (run_head) start[slot] = (uint32_t)e;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, slot);
    if (slot >= 0 && lane == (unsigned)(__ffs(peers) - 1))
      atomicAdd(&cnt[slot], (unsigned long long)__popc(peers));
  }
}

// BCSR, step 2 (one thread per oriented edge): copy the column to its
// block-major position and record the position for the in-edges.
__global__ void k_bcsr_fill(const int32_t *__restrict__ esrc, const int32_t *__restrict__ colidx,
                            int64_t m, const int32_t *__restrict__ cuts_g, int p,
                            const int64_t *__restrict__ rpb_g, const uint64_t *__restrict__ pos,
                            const uint32_t *__restrict__ start, int32_t *__restrict__ ci,
                            uint32_t *__restrict__ pos_of_edge) {
  __shared__ int32_t cuts[MAXP + 1];
  __shared__ int64_t rpb[MAXP * MAXP];
  for (int i = threadIdx.x; i <= p; i += blockDim.x) cuts[i] = cuts_g[i];
  for (int i = threadIdx.x; i < p * p; i += blockDim.x) rpb[i] = rpb_g[i];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = esrc[e], v = colidx[e];
    const int a = part_of_dev(cuts, p, u), b = part_of_dev(cuts, p, v);
    const int64_t slot = rpb[a * p + b] + (u - cuts[a]);
    const uint64_t dest = pos[slot] + (uint64_t)(e - (int64_t)start[slot]);
    ci[dest] = v;
    pos_of_edge[e] = (uint32_t)dest;
  }
}

// BCSR, step 3: the row pointers are the scanned slot counts, narrowed.
__global__ void k_bcsr_rowptr(const uint64_t *__restrict__ pos, int64_t total,
                              uint32_t *__restrict__ rp) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x)
    rp[i] = (uint32_t)pos[i];
}

__device__ __forceinline__ int64_t block_nnz(const int64_t *boff, int p, int i, int j) {
  return boff[i * (p + 1) + j + 1] - boff[i * (p + 1) + j];
}

// Alg. 4 order: index of (i, j, j) is the number of tasks with a smaller first
// index plus those with first index i and a smaller second index.
__device__ __forceinline__ int64_t task_index(int p, int i, int j, int k) {
  int64_t t = 0;
  for (int a = 0; a < i; ++a) t += (int64_t)(p - a) * (p - a + 1) / 2;
  for (int b = i; b < j; ++b) t += p - b;
  return t + (k - j);
}

// a7 + a8: tasks, ExecTime (Sec. 5) and the sort keys of the order.
// est = |G_ij| * max(delta(G_ik), delta(G_jk)), delta(G_ab) = |G_ab| / |V_a|.
__global__ void k_tasks(const int64_t *__restrict__ boff, const int32_t *__restrict__ cuts,
                        int p, int32_t *__restrict__ tasks, double *__restrict__ est,
                        uint64_t *__restrict__ order_keys, uint32_t *__restrict__ order_vals) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // one thread per (i, j, k)
  if (idx >= p * p * p) return;
  const int i = idx / (p * p), j = (idx / p) % p, k = idx % p;
  if (!(i <= j && j <= k)) return;
  const int64_t t = task_index(p, i, j, k);
  tasks[3 * t + 0] = i;
  tasks[3 * t + 1] = j;
  tasks[3 * t + 2] = k;
  const int64_t vi = cuts[i + 1] - cuts[i], vj = cuts[j + 1] - cuts[j];
  const double dik = vi > 0 ? (double)block_nnz(boff, p, i, k) / (double)vi : 0.0;
  const double djk = vj > 0 ? (double)block_nnz(boff, p, j, k) / (double)vj : 0.0;
  const double e = (double)block_nnz(boff, p, i, j) * (dik > djk ? dik : djk);
  est[t] = e;
  // non-negative doubles order like their bit patterns; complement for
  // descending, and the stable sort keeps Alg. 4 order among equal estimates
  order_keys[t] = ~(uint64_t)__double_as_longlong(e);
  order_vals[t] = (uint32_t)t;
}

__global__ void k_order_finish(const uint32_t *__restrict__ vals, int64_t nt,
                               int32_t *__restrict__ order) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nt;
       x += (int64_t)gridDim.x * blockDim.x)
    order[x] = (int32_t)vals[x];
}

// Number of work items of the task at each position of the order. A task
// whose G_ij, G_ik or G_jk is empty holds no triangle and gets none.
__global__ void k_item_counts(const int32_t *__restrict__ order,
                              const int32_t *__restrict__ tasks, const int64_t *__restrict__ boff,
                              int p, int64_t nt, int64_t chunk, uint64_t *__restrict__ counts) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nt;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int t = order[x];
    const int i = tasks[3 * t], j = tasks[3 * t + 1], k = tasks[3 * t + 2];
    const int64_t nij = block_nnz(boff, p, i, j);
    const bool empty = nij == 0 || block_nnz(boff, p, i, k) == 0 || block_nnz(boff, p, j, k) == 0;
    counts[x] = empty ? 0 : (uint64_t)((nij + chunk - 1) / chunk);
  }
}

// One thread per work item q: the task at position x of the order with
// first[x] <= q < first[x + 1] (binary search), and its chunk q - first[x].
__global__ void k_item_fill(const int32_t *__restrict__ order, const int32_t *__restrict__ tasks,
                            const int64_t *__restrict__ boff, int p, int64_t nt, int64_t chunk,
                            const uint64_t *__restrict__ first, uint64_t nitems,
                            int kernel_mode, int32_t hash_threshold,
                            WorkItem *__restrict__ items) {
  // isDense (Alg. 7), decided per staged list N(G_jk, v) by the counting
  // kernel: bits 0-1 = 0 INTERSECT (sorted search), 1 HASHMAP, 2 AUTO;
  // bits 2.. = the AUTO length above which a list that does not fit a
  // bitmap is hashed rather than searched
  const int32_t flags = kernel_mode == BBTC_KERNEL_HASHMAP     ? 1
                        : kernel_mode == BBTC_KERNEL_INTERSECT ? 0
                                                               : 2 | (hash_threshold << 2);
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nitems;
       q += (uint64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = nt;  // last x with first[x] <= q
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (first[mid] <= q) lo = mid; else hi = mid;
    }
    const int t = order[lo];
    const int i = tasks[3 * t], j = tasks[3 * t + 1];
    const int64_t b0 = boff[i * (p + 1) + j], b1 = boff[i * (p + 1) + j + 1];
    WorkItem w;
    w.task = t;
    w.flags = flags;
    w.x0 = b0 + (int64_t)(q - first[lo]) * chunk;
    w.x1 = w.x0 + chunk < b1 ? w.x0 + chunk : b1;
    items[q] = w;
  }
}

}  // namespace

void free_plan(Plan *pl, cudaStream_t s) {
  dfree(pl->cuts, s);
  dfree(pl->ie, s);
  dfree(pl->boff, s);
  dfree(pl->tasks, s);
  dfree(pl->est, s);
  dfree(pl->order, s);
  dfree(pl->items, s);
  dfree(pl->scratch, s);
  dfree(pl->rp, s);
  dfree(pl->ci, s);
  dfree(pl->spl, s);
  dfree(pl->desc, s);
  free_plan_host(pl);
  *pl = Plan();
}

int default_p(const bbtc_graph *g, bool budgeted) {
  // Sec. 7.3 suggests p near the average degree for a CPU cache. On one GPU with
  // the whole graph resident nothing needs small blocks: fewer parts stage each
  // N(G_jk, v) once and probe it in longer runs (on the Friendster-shaped graph
  // the count takes 293 ms at p = 1, 472 ms at p = 8 and 654 ms at p = 16), so
  // resident counts take 2 parts (1 for small graphs). Under a device budget a
  // task's three blocks must fit in half the budget: p grows with m.
  if (g->m < (1 << 16)) return 1;
  if (!budgeted) return 2;
  if (g->m < (1 << 22)) return 2;
  if (g->m < (1 << 27)) return 4;
  return 8;
}

bbtc_status build_plan(bbtc_graph *g, int p, int kernel_mode, int hash_threshold, int chunk_req,
                       cudaStream_t s, int partition) {
  if (plan_matches(g->plan, p, kernel_mode, hash_threshold, chunk_req, partition)) return BBTC_OK;
  free_plan(&g->plan, s);
  Plan pl;
  pl.p = p;
  pl.kernel_mode = kernel_mode;
  pl.hash_threshold = hash_threshold;
  pl.chunk_req = chunk_req;
  pl.partition = partition;
  pl.ntasks = (int64_t)p * (p + 1) * (p + 2) / 6;
  const int64_t n = g->n, m = g->m;
  Scratch scratch(s);
  bbtc_status st = BBTC_OK;
#define PLAN_TRY(expr)          \
  do {                          \
    st = (expr);                \
    if (st != BBTC_OK) {        \
      free_plan(&pl, s);        \
      return st;                \
    }                           \
  } while (0)

  // a5: cuts
  PLAN_TRY(dalloc_n(&pl.cuts, p + 1, s));
  if (partition == 1) {
    PLAN_TRY(pbd_partition(g, p, pl.cuts, &pl.bstar, s));
  } else {
    k_cuts<<<1, MAXP + 1, 0, s>>>(g->rowptr, n, p, pl.cuts);
    PLAN_TRY(launch_status("build_plan"));
  }

  // a6: the blocks, read in place from the oriented CSR through the split
  // table (per part a: |V_a| rows of p - a + 1 positions)
  if (cudaMemcpyAsync(pl.h_cuts, pl.cuts, sizeof(int32_t) * (size_t)(p + 1),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("build_plan: reading the cuts failed");
    free_plan(&pl, s);
    return BBTC_ECUDA;
  }
  {
    int64_t off = 0;
    for (int a = 0; a < p; ++a) {
      pl.h_spl_off[a] = off;
      off += (int64_t)(pl.h_cuts[a + 1] - pl.h_cuts[a]) * (p - a + 1);
    }
    pl.h_spl_off[p] = off;
  }
  int64_t *d_spl_off = nullptr;
  PLAN_TRY(scratch.get(&d_spl_off, p + 1));
  PLAN_TRY(dalloc_n(&pl.spl, pl.h_spl_off[p] > 0 ? pl.h_spl_off[p] : 1, s));
  if (cudaMemcpyAsync(d_spl_off, pl.h_spl_off, sizeof(int64_t) * (size_t)(p + 1),
                      cudaMemcpyHostToDevice, s) != cudaSuccess) {
    set_error("build_plan: copying the split offsets failed");
    free_plan(&pl, s);
    return BBTC_ECUDA;
  }
  if (n > 0) {
    k_splits<<<grid_for(n, 256, 16), 256, 0, s>>>(g->rowptr, g->colidx, n, pl.cuts, p, d_spl_off,
                                                  pl.spl);
    PLAN_TRY(launch_status("build_plan"));
  }

  // in-edges grouped by (part(u), v), and the block offsets: one counting
  // sort on the destination per part
  PLAN_TRY(dalloc_n(&pl.ie, m, s));
  PLAN_TRY(dalloc_n(&pl.boff, (int64_t)p * (p + 1), s));
  {
    unsigned *hist = nullptr;  // counts, then the scatter's cursors
    uint64_t *scan = nullptr;
    PLAN_TRY(scratch.get(&hist, n + 1));
    PLAN_TRY(scratch.get(&scan, n + 1));
    // bucket tables of the two-phase build (large parts only)
    int32_t *ieb_bnd = nullptr;
    unsigned *ieb_bstart = nullptr, *ieb_bcur = nullptr;
    if (m / p >= IEB_MIN_EDGES) {
      PLAN_TRY(scratch.get(&ieb_bnd, IEB_B + 1));
      PLAN_TRY(scratch.get(&ieb_bstart, IEB_B + 1));
      PLAN_TRY(scratch.get(&ieb_bcur, IEB_B));
    }
    for (int a = 0; a < p; ++a) {
      const int64_t bins = n - pl.h_cuts[a];
      if (cudaMemsetAsync(hist, 0, sizeof(unsigned) * (size_t)(bins + 1), s) != cudaSuccess) {
        set_error("build_plan: cudaMemsetAsync failed");
        free_plan(&pl, s);
        return BBTC_ECUDA;
      }
      // a few CTAs per SM, each with a contiguous share of the part's edges
      const unsigned ie_grid = grid_for(m / p + 1, IE_NT * 64, 4);
      if (p == 1 && n > 0 && g->deg && g->perm) {  // a union of handles has no degrees
        k_indegree<<<grid_for(n, 256, 16), 256, 0, s>>>(g->rowptr, g->perm, g->deg, n, hist);
        PLAN_TRY(launch_status("build_plan"));
      } else if (m > 0) {
        k_inedge_count<<<ie_grid, IE_NT, 0, s>>>(g->rowptr, g->colidx, pl.cuts, a, n, hist);
        PLAN_TRY(launch_status("build_plan"));
      }
      if (bins > 0) {
        k_widen<<<grid_for(bins, 256, 16), 256, 0, s>>>(hist, bins, scan);
        PLAN_TRY(launch_status("build_plan"));
        PLAN_TRY(exclusive_scan_u64(scan, scan, bins, s));
        k_narrow<<<grid_for(bins, 256, 16), 256, 0, s>>>(scan, bins, hist);
        PLAN_TRY(launch_status("build_plan"));
      }
      k_inedge_offsets<<<1, MAXP + 1, 0, s>>>(g->rowptr, pl.cuts, a, p,
                                               reinterpret_cast<const unsigned long long *>(scan),
                                               bins, pl.boff);
      PLAN_TRY(launch_status("build_plan"));
      // large parts: partition into destination buckets, then place (the
      // temporary array takes 16 bytes per edge of the part); else, or when it
      // does not fit, one direct scatter
      InEdge *ieb_tmp = nullptr;
      const bool two_phase = m / p >= IEB_MIN_EDGES && bins > IEB_B && ieb_bnd &&
                             dalloc_n(&ieb_tmp, m, s) == BBTC_OK;
      if (!two_phase) clear_error();
      if (two_phase) {
        k_ieb_bounds<<<(IEB_B + 1 + 127) / 128, 128, 0, s>>>(g->rowptr, pl.cuts, a, scan, bins,
                                                            ieb_bnd, ieb_bstart, ieb_bcur);
        bbtc_status lst = launch_status("build_plan");
        if (lst == BBTC_OK &&
            cudaFuncSetAttribute(k_ieb_partition, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(InEdge) * IEB_T)) != cudaSuccess) {
          set_error("build_plan: configuring the in-edge partition kernel failed");
          lst = BBTC_ECUDA;
        }
        if (lst == BBTC_OK) {
          k_ieb_partition<<<(unsigned)num_sms() * 2, IEB_NT, sizeof(InEdge) * IEB_T, s>>>(
              g->rowptr, g->colidx, g->esrc, pl.cuts, a, p, pl.spl + pl.h_spl_off[a], ieb_bnd,
              ieb_bstart, ieb_bcur, ieb_tmp);
          lst = launch_status("build_plan");
        }
        if (lst == BBTC_OK) {
          k_ieb_place<<<grid_for(m / p + 1, 256, 8), 256, 0, s>>>(ieb_tmp, g->rowptr, pl.cuts, a,
                                                                  hist, pl.ie);
          lst = launch_status("build_plan");
        }
        dfree(ieb_tmp, s);
        PLAN_TRY(lst);
      } else if (m > 0) {
        for (int64_t v_lo = pl.h_cuts[a]; v_lo < n; v_lo += IE_SLAB) {
          const int64_t v_hi = v_lo + IE_SLAB < n ? v_lo + IE_SLAB : n;
          k_inedge_scatter<<<ie_grid, IE_NT_S, 0, s>>>(g->rowptr, g->colidx, g->esrc, pl.cuts, a,
                                                        p, v_lo, v_hi, pl.spl + pl.h_spl_off[a],
                                                        hist, pl.ie);
          PLAN_TRY(launch_status("build_plan"));
        }
      }
    }
  }

  // a7 + a8: tasks, estimates, order
  const int64_t nt = pl.ntasks;
  PLAN_TRY(dalloc_n(&pl.tasks, 3 * nt, s));
  PLAN_TRY(dalloc_n(&pl.est, nt, s));
  PLAN_TRY(dalloc_n(&pl.order, nt, s));
  uint64_t *okeys = nullptr, *okeys_alt = nullptr;
  uint32_t *ovals = nullptr, *ovals_alt = nullptr;
  PLAN_TRY(scratch.get(&okeys, nt));
  PLAN_TRY(scratch.get(&okeys_alt, nt));
  PLAN_TRY(scratch.get(&ovals, nt));
  PLAN_TRY(scratch.get(&ovals_alt, nt));
  bool in_alt = false;
  k_tasks<<<(p * p * p + 127) / 128, 128, 0, s>>>(pl.boff, pl.cuts, p, pl.tasks, pl.est, okeys,
                                                  ovals);
  PLAN_TRY(launch_status("build_plan"));
  PLAN_TRY(radix_sort(okeys, okeys_alt, ovals, ovals_alt, nt, 0, 64, s, &in_alt));
  k_order_finish<<<grid_for(nt, 256, 4), 256, 0, s>>>(in_alt ? ovals_alt : ovals, nt, pl.order);
  PLAN_TRY(launch_status("build_plan"));

  // task descriptors: every block of the resident BCSR
  {
    TaskDesc *h_desc = new (std::nothrow) TaskDesc[(size_t)nt];
    if (!h_desc) {
      set_error("build_plan: host allocation failed");
      free_plan(&pl, s);
      return BBTC_ENOMEM;
    }
    int64_t t = 0;
    for (int i = 0; i < p; ++i)
      for (int j = i; j < p; ++j)
        for (int k = j; k < p; ++k, ++t) {
          TaskDesc &d = h_desc[t];
          d.ie = pl.ie;
          d.ie_off = 0;
          d.rp_ik = pl.spl + pl.h_spl_off[i] + (k - i);
          d.rs_ik = p - i + 1;
          d.ci_ik = g->colidx;
          d.ci_ik_off = 0;
          d.rp_jk = pl.spl + pl.h_spl_off[j] + (k - j);
          d.rs_jk = p - j + 1;
          d.ci_jk = g->colidx;
          d.ci_jk_off = 0;
          d.c_i = pl.h_cuts[i];
          d.c_j = pl.h_cuts[j];
          d.diag = k == j;
          d.task = (int32_t)t;
        }
    bbtc_status dst = dalloc_n(&pl.desc, nt, s);
    if (dst == BBTC_OK &&
        (cudaMemcpyAsync(pl.desc, h_desc, sizeof(TaskDesc) * (size_t)nt, cudaMemcpyHostToDevice,
                         s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess)) {
      set_error("build_plan: copying the task descriptors failed");
      dst = BBTC_ECUDA;
    }
    delete[] h_desc;
    PLAN_TRY(dst);
  }

  // work items: about 64 per resident warp in total, 64..4096 in-edges each
  // (or the caller's choice)
  const int64_t warps = (int64_t)num_sms() * 24;
  int64_t chunk = (m * (int64_t)(p < 3 ? p : 3)) / (warps * 64);
  chunk = chunk < 64 ? 64 : (chunk > 4096 ? 4096 : chunk);
  if (chunk_req > 0) chunk = chunk_req;
  pl.chunk = chunk;
  uint64_t *first = nullptr;
  PLAN_TRY(scratch.get(&first, nt + 1));
  k_item_counts<<<grid_for(nt, 256, 4), 256, 0, s>>>(pl.order, pl.tasks, pl.boff, p, nt, chunk,
                                                     first);
  PLAN_TRY(launch_status("build_plan"));
  PLAN_TRY(exclusive_scan_u64(first, first, nt + 1, s));
  uint64_t nitems = 0;
  if (cudaMemcpyAsync(&nitems, first + nt, sizeof(uint64_t), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("build_plan: reading the work-item count failed");
    free_plan(&pl, s);
    return BBTC_ECUDA;
  }
  pl.nitems = (int64_t)nitems;
  PLAN_TRY(dalloc_n(&pl.items, pl.nitems, s));
  if (nitems > 0) {
    k_item_fill<<<grid_for((int64_t)nitems, 256, 8), 256, 0, s>>>(
        pl.order, pl.tasks, pl.boff, p, nt, chunk, first, nitems, kernel_mode, hash_threshold,
        pl.items);
    PLAN_TRY(launch_status("build_plan"));
  }
  // counting scratch and kernel configuration, so that a count only enqueues
  PLAN_TRY(dalloc_n(&pl.scratch, SCR_TASKS + nt + g->ng, s));
  PLAN_TRY(configure_count_kernels(&pl));
#undef PLAN_TRY
  pl.bytes = (uint64_t)m * sizeof(InEdge) + (uint64_t)pl.h_spl_off[p] * 4 + (uint64_t)nt * (24 + sizeof(TaskDesc)) +
             (uint64_t)pl.nitems * sizeof(WorkItem) + (uint64_t)(SCR_TASKS + nt + g->ng) * 8;
  g->plan = pl;
  return BBTC_OK;
}

bbtc_status plan_physical_blocks(const bbtc_graph *g, Plan &pl, cudaStream_t s) {
  if (pl.rp) return BBTC_OK;
  const int p = pl.p;
  const int64_t m = g->m;
  {
    int64_t off = 0;
    for (int a = 0; a < p; ++a)
      for (int b = a; b < p; ++b) {
        pl.h_rpb[a * p + b] = off;
        off += (int64_t)(pl.h_cuts[a + 1] - pl.h_cuts[a]) + 1;
      }
    pl.total_rp = off;
  }
  Scratch scratch(s);
  int64_t *d_rpb = nullptr;
  uint64_t *cnt = nullptr;
  uint32_t *start = nullptr, *pos_of_edge = nullptr;
  BBTC_TRY(scratch.get(&d_rpb, (int64_t)p * p));
  BBTC_TRY(scratch.get(&cnt, pl.total_rp));
  BBTC_TRY(scratch.get(&start, pl.total_rp));
  BBTC_TRY(scratch.get(&pos_of_edge, m > 0 ? m : 1));
  BBTC_TRY(dalloc_n(&pl.rp, pl.total_rp, s));
  BBTC_TRY(dalloc_n(&pl.ci, m > 0 ? m : 1, s));
  BBTC_CUDA(cudaMemcpyAsync(d_rpb, pl.h_rpb, sizeof(int64_t) * (size_t)p * p,
                            cudaMemcpyHostToDevice, s));
  BBTC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint64_t) * (size_t)pl.total_rp, s));
  if (m > 0) {
    k_bcsr_count<<<grid_for(m, 256, 32), 256, 0, s>>>(
        g->esrc, g->colidx, m, pl.cuts, p, d_rpb, reinterpret_cast<unsigned long long *>(cnt),
        start);
    BBTC_LAUNCH_CHECK();
  }
  BBTC_TRY(exclusive_scan_u64(cnt, cnt, pl.total_rp, s));
  if (m > 0) {
    k_bcsr_fill<<<grid_for(m, 256, 32), 256, 0, s>>>(g->esrc, g->colidx, m, pl.cuts, p, d_rpb,
                                                     cnt, start, pl.ci, pos_of_edge);
    BBTC_LAUNCH_CHECK();
    k_remap_positions<<<grid_for(m, 256, 32), 256, 0, s>>>(pl.ie, m, pos_of_edge);
    BBTC_LAUNCH_CHECK();
  }
  k_bcsr_rowptr<<<grid_for(pl.total_rp, 256, 32), 256, 0, s>>>(cnt, pl.total_rp, pl.rp);
  BBTC_LAUNCH_CHECK();
  dfree(pl.spl, s);
  pl.spl = nullptr;
  return BBTC_OK;
}

}  // namespace bbtc
