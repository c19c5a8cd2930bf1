// batch.cu -- union of separately created handles for bbtc_count_batch.
//
// The union of ng oriented CSRs is again an oriented CSR: positions of handle
// h are shifted by the vertices of the handles before it, edge lists by their
// edges. Each handle's orientation is kept, so every triangle of handle h is
// counted once, in h, and the counting kernel attributes it through the
// union's graph-of-position array.
#include <new>

#include "graph.cuh"
#include "primitives.cuh"

namespace bbtc {

namespace {

struct UnionSrc {
  const int64_t *rowptr;
  const int32_t *colidx;
  const int32_t *esrc;
  const int32_t *perm;
};

constexpr int SMEM_OFFSETS = 4096;  // offsets searched in shared memory up to this many graphs

// Last g in [0, ng) with off[g] <= x.
__device__ __forceinline__ int graph_of(const int64_t *off, int ng, int64_t x) {
  int lo = 0, hi = ng;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_union_vertices(const UnionSrc *__restrict__ src,
                                 const int64_t *__restrict__ voff_g,
                                 const int64_t *__restrict__ eoff_g, int ng, int64_t n,
                                 int64_t m, int64_t *__restrict__ rowptr,
                                 int32_t *__restrict__ perm, int32_t *__restrict__ gid) {
  __shared__ int64_t voff_s[SMEM_OFFSETS + 1];
  const bool in_smem = ng <= SMEM_OFFSETS;
  if (in_smem)
    for (int i = threadIdx.x; i <= ng; i += blockDim.x) voff_s[i] = voff_g[i];
  __syncthreads();
  const int64_t *voff = in_smem ? voff_s : voff_g;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int g = graph_of(voff, ng, r);
    const int64_t rr = r - voff[g];
    rowptr[r] = eoff_g[g] + src[g].rowptr[rr];
    perm[r] = (int32_t)(voff[g] + src[g].perm[rr]);
    gid[r] = g;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) rowptr[n] = m;
}

__global__ void k_union_edges(const UnionSrc *__restrict__ src,
                              const int64_t *__restrict__ voff_g,
                              const int64_t *__restrict__ eoff_g, int ng, int64_t m,
                              int32_t *__restrict__ colidx, int32_t *__restrict__ esrc) {
  __shared__ int64_t eoff_s[SMEM_OFFSETS + 1];
  const bool in_smem = ng <= SMEM_OFFSETS;
  if (in_smem)
    for (int i = threadIdx.x; i <= ng; i += blockDim.x) eoff_s[i] = eoff_g[i];
  __syncthreads();
  const int64_t *eoff = in_smem ? eoff_s : eoff_g;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int g = graph_of(eoff, ng, e);
    const int64_t ee = e - eoff[g];
    const int32_t shift = (int32_t)voff_g[g];
    colidx[e] = shift + src[g].colidx[ee];
    esrc[e] = shift + src[g].esrc[ee];
  }
}

}  // namespace

bbtc_status union_of(const bbtc_graph_t *gs, int32_t ng, cudaStream_t s, bbtc_graph **out) {
  *out = nullptr;
  int64_t *voff = new (std::nothrow) int64_t[(size_t)ng + 1];
  int64_t *eoff = new (std::nothrow) int64_t[(size_t)ng + 1];
  UnionSrc *tab = new (std::nothrow) UnionSrc[(size_t)ng];
  bbtc_graph *u = new (std::nothrow) bbtc_graph();
  bbtc_status st = BBTC_OK;
  if (!voff || !eoff || !tab || !u) {
    set_error("bbtc_count_batch: host allocation failed");
    st = BBTC_ENOMEM;
  }
  int64_t N = 0, M = 0;
  if (st == BBTC_OK) {
    voff[0] = eoff[0] = 0;
    for (int32_t i = 0; i < ng; ++i) {
      if (gs[i]->device != gs[0]->device) {
        set_error("bbtc_count_batch: handles live on different devices");
        st = BBTC_EINVAL;
        break;
      }
      tab[i] = UnionSrc{gs[i]->rowptr, gs[i]->colidx, gs[i]->esrc, gs[i]->perm};
      voff[i + 1] = voff[i] + gs[i]->n;
      eoff[i + 1] = eoff[i] + gs[i]->m;
    }
    N = voff[ng];
    M = eoff[ng];
    if (st == BBTC_OK && (N > 0x7fffffffLL || M > 0xFFFFFFFFLL)) {
      set_error("bbtc_count_batch: the union has %lld vertices and %lld edges, beyond the "
                "int32 id / uint32 edge limits", (long long)N, (long long)M);
      st = BBTC_EINVAL;
    }
  }
  UnionSrc *d_tab = nullptr;
  int64_t *d_eoff = nullptr;
  if (st == BBTC_OK) {
    u->n = N;
    u->m = M;
    u->nb = ceil_log2_u64((uint64_t)N) < 1 ? 1 : ceil_log2_u64((uint64_t)N);
    u->device = gs[0]->device;
    u->stream = s;
    u->own_stream = false;
    u->ng = ng;
    for (cudaEvent_t &e : u->ev)
      if (st == BBTC_OK && cudaEventCreate(&e) != cudaSuccess) {
        set_error("bbtc_count_batch: cudaEventCreate failed");
        st = BBTC_ECUDA;
      }
  }
  if (st == BBTC_OK) st = dalloc_n(&u->rowptr, N + 1, s);
  if (st == BBTC_OK) st = dalloc_n(&u->colidx, padded_columns(M), s);
  if (st == BBTC_OK) st = dalloc_n(&u->esrc, M, s);
  if (st == BBTC_OK) st = dalloc_n(&u->perm, N, s);
  if (st == BBTC_OK) st = dalloc_n(&u->gid, N, s);
  if (st == BBTC_OK) st = dalloc_n(&u->voff, ng + 1, s);
  if (st == BBTC_OK) st = dalloc_n(&d_eoff, ng + 1, s);
  if (st == BBTC_OK) st = dalloc_n(&d_tab, ng, s);
  if (st == BBTC_OK &&
      (cudaMemcpyAsync(u->voff, voff, sizeof(int64_t) * (size_t)(ng + 1), cudaMemcpyHostToDevice,
                       s) != cudaSuccess ||
       cudaMemcpyAsync(d_eoff, eoff, sizeof(int64_t) * (size_t)(ng + 1), cudaMemcpyHostToDevice,
                       s) != cudaSuccess ||
       cudaMemcpyAsync(d_tab, tab, sizeof(UnionSrc) * (size_t)ng, cudaMemcpyHostToDevice, s) !=
           cudaSuccess)) {
    set_error("bbtc_count_batch: copying the handle table failed");
    st = BBTC_ECUDA;
  }
  if (st == BBTC_OK) {
    k_union_vertices<<<grid_for(N + 1, 256, 16), 256, 0, s>>>(d_tab, u->voff, d_eoff, ng, N, M,
                                                              u->rowptr, u->perm, u->gid);
    st = launch_status("bbtc_count_batch");
  }
  if (st == BBTC_OK && M > 0) {
    k_union_edges<<<grid_for(M, 256, 32), 256, 0, s>>>(d_tab, u->voff, d_eoff, ng, M, u->colidx,
                                                       u->esrc);
    st = launch_status("bbtc_count_batch");
  }
  // the host tables must outlive the copies above
  if (cudaStreamSynchronize(s) != cudaSuccess && st == BBTC_OK) {
    set_error("bbtc_count_batch: %s", cudaGetErrorString(cudaGetLastError()));
    st = BBTC_ECUDA;
  }
  dfree(d_tab, s);
  dfree(d_eoff, s);
  delete[] voff;
  delete[] eoff;
  delete[] tab;
  if (st != BBTC_OK) {
    if (u) {
      free_plan(&u->plan, s);
      dfree(u->rowptr, s);
      dfree(u->colidx, s);
      dfree(u->esrc, s);
      dfree(u->perm, s);
      dfree(u->gid, s);
      dfree(u->voff, s);
      for (cudaEvent_t &e : u->ev)
        if (e) cudaEventDestroy(e);
      delete u;
    }
    return st;
  }
  *out = u;
  return BBTC_OK;
}

}  // namespace bbtc
