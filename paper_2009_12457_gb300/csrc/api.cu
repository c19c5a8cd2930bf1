// api.cu -- the extern "C" entry points declared in include/bbtc.h.
#include <stdarg.h>
#include <stdio.h>
#include <stddef.h>
#include <string.h>

#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "graph.cuh"
#include "primitives.cuh"

namespace bbtc {

namespace {
thread_local char g_error[1024] = "";
std::once_flag g_pool_once[64];
unsigned long long g_launches = 0;
}  // namespace

void note_launch() { __atomic_fetch_add(&g_launches, 1ull, __ATOMIC_RELAXED); }

bbtc_status launch_status(const char *where) {
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: kernel launch failed: %s", where, cudaGetErrorString(e));
    return BBTC_ECUDA;
  }
  return BBTC_OK;
}

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_error, sizeof(g_error), fmt, ap);
  va_end(ap);
}

void clear_error() { g_error[0] = '\0'; }

// Large blocks (at least kCacheMin bytes) are not returned to the pool when
// freed: an idle block is kept, with an event marking the end of its last use,
// and handed out again for a request of up to its size (and at least 4/5 of
// it) on a stream that first waits for that event. A repeated call with the
// same sizes then gets back the same blocks: taking a fresh block of tens of
// GB from the pool costs about a millisecond per GB of host time, during which
// the GPU runs dry. Idle blocks are released to the pool when an allocation
// fails, before a budgeted (streamed) count, and when they would exceed half
// of the device's memory.
namespace {
constexpr size_t kCacheMin = 64ull << 20;
struct IdleBlock {
  void *p;
  size_t bytes;
  cudaEvent_t ev;
};
struct BlockCache {
  std::mutex mu;
  std::vector<IdleBlock> idle[64];
  std::unordered_map<void *, size_t> live[64];  // large blocks handed out: bytes
  uint64_t idle_bytes[64] = {};
  uint64_t cap[64] = {};
};
BlockCache &block_cache() {
  static BlockCache *c = new BlockCache;  // never destroyed: blocks outlive static teardown
  return *c;
}

// frees the idle blocks of device dev (caller holds the lock), after s waits for
// their last use
void release_idle_locked(BlockCache &c, int dev, cudaStream_t s) {
  for (IdleBlock &b : c.idle[dev]) {
    cudaStreamWaitEvent(s, b.ev, 0);
    cudaFreeAsync(b.p, s);
    cudaEventDestroy(b.ev);
  }
  c.idle[dev].clear();
  c.idle_bytes[dev] = 0;
}
}  // namespace

void release_cached_blocks(int dev, cudaStream_t s) {
  if (dev < 0 || dev >= 64) return;
  BlockCache &c = block_cache();
  std::lock_guard<std::mutex> lk(c.mu);
  release_idle_locked(c, dev, s);
}

uint64_t cached_block_bytes(int dev) {
  if (dev < 0 || dev >= 64) return 0;
  BlockCache &c = block_cache();
  std::lock_guard<std::mutex> lk(c.mu);
  return c.idle_bytes[dev];
}

bbtc_status dalloc(void **p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_error("cudaGetDevice failed");
    return BBTC_ECUDA;
  }
  if (dev >= 0 && dev < 64)
    std::call_once(g_pool_once[dev], [dev] {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t threshold = ~0ull;  // keep freed blocks cached for the next call
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
      }
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) block_cache().cap[dev] = total_b / 2;
      cudaGetLastError();
    });
  const bool large = bytes >= kCacheMin && dev >= 0 && dev < 64;
  if (large) {
    BlockCache &c = block_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    std::vector<IdleBlock> &v = c.idle[dev];
    int best = -1;  // the smallest fitting block, one whose last use has ended first
    bool best_done = false;
    for (int i = 0; i < (int)v.size(); ++i) {
      if (v[i].bytes < bytes || v[i].bytes - bytes > v[i].bytes / 5) continue;
      const bool done = cudaEventQuery(v[i].ev) == cudaSuccess;
      if (best < 0 || (done && !best_done) ||
          (done == best_done && v[i].bytes < v[best].bytes)) {
        best = i;
        best_done = done;
      }
    }
    cudaGetLastError();
    if (best >= 0) {
      IdleBlock b = v[best];
      v.erase(v.begin() + best);
      c.idle_bytes[dev] -= b.bytes;
      cudaStreamWaitEvent(s, b.ev, 0);
      cudaEventDestroy(b.ev);
      c.live[dev][b.p] = b.bytes;
      *p = b.p;
      return BBTC_OK;
    }
  }
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e == cudaErrorMemoryAllocation && dev >= 0 && dev < 64) {
    cudaGetLastError();
    bool retry = false;
    {
      BlockCache &c = block_cache();
      std::lock_guard<std::mutex> lk(c.mu);
      retry = !c.idle[dev].empty();
      release_idle_locked(c, dev, s);
    }
    if (retry) e = cudaMallocAsync(p, bytes, s);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BBTC_ENOMEM : BBTC_ECUDA;
  }
  if (large) {
    BlockCache &c = block_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    c.live[dev][*p] = bytes;
  }
  return BBTC_OK;
}

void dfree(void *p, cudaStream_t s) {
  if (!p) return;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
    BlockCache &c = block_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.live[dev].find(p);
    if (it != c.live[dev].end()) {
      const size_t bytes = it->second;
      c.live[dev].erase(it);
      cudaEvent_t ev = nullptr;
      if (c.idle_bytes[dev] + bytes <= c.cap[dev] &&
          cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
          cudaEventRecord(ev, s) == cudaSuccess) {
        c.idle[dev].push_back(IdleBlock{p, bytes, ev});
        c.idle_bytes[dev] += bytes;
        return;
      }
      if (ev) cudaEventDestroy(ev);
      cudaGetLastError();
    }
  }
  cudaFreeAsync(p, s);
}

}  // namespace bbtc

namespace bbtc {
namespace {

// Makes the handle's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

void destroy_graph(bbtc_graph *g) {
  if (!g) return;
  cudaStream_t s = g->stream;
  free_plan(&g->plan, s);
  dfree(g->rowptr, s);
  dfree(g->colidx, s);
  dfree(g->esrc, s);
  dfree(g->perm, s);
  dfree(g->deg, s);
  dfree(g->voff, s);
  dfree(g->gid, s);
  cudaStreamSynchronize(s);
  for (cudaEvent_t &e : g->ev)
    if (e) cudaEventDestroy(e);
  if (g->own_stream) cudaStreamDestroy(s);
  delete g;
}

__global__ void k_scatter_by_perm(const unsigned long long *__restrict__ by_pos,
                                  const int32_t *__restrict__ perm, int64_t n,
                                  unsigned long long *__restrict__ by_id) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x)
    by_id[perm[r]] = by_pos[r];
}

bbtc_status check_opts(const bbtc_opts *opts, bbtc_opts *out) {
  bbtc_opts_init(out);
  if (opts) {
    if (opts->struct_size < sizeof(bbtc_opts)) {
      set_error("bbtc_opts.struct_size is %u, expected %zu (call bbtc_opts_init)",
                opts->struct_size, sizeof(bbtc_opts));
      return BBTC_EINVAL;
    }
    *out = *opts;
  }
  if (out->p < 0 || out->p > 64) {
    set_error("p = %d is outside 0..64", out->p);
    return BBTC_EINVAL;
  }
  if (out->kernel < BBTC_KERNEL_AUTO || out->kernel > BBTC_KERNEL_HASHMAP) {
    set_error("kernel = %d is not a bbtc_kernel", out->kernel);
    return BBTC_EINVAL;
  }
  if (out->hash_threshold < 0 || out->hash_threshold > (1 << 28)) {
    set_error("hash_threshold = %d is outside 0..2^28", out->hash_threshold);
    return BBTC_EINVAL;
  }
  if (out->hash_threshold == 0) out->hash_threshold = 16;
  if (out->chunk < 0) {
    set_error("chunk = %d must be >= 0", out->chunk);
    return BBTC_EINVAL;
  }
  if (out->partition != BBTC_PARTITION_EDGES && out->partition != BBTC_PARTITION_PROBE) {
    set_error("partition = %d is not a bbtc_partition", out->partition);
    return BBTC_EINVAL;
  }
  return BBTC_OK;
}

// Shared body of bbtc_graph_create_async and bbtc_graph_create_batch.
bbtc_status create_common(int64_t n, const int64_t *rowptr, const int32_t *colidx,
                          uint32_t flags, void *stream, int32_t ng, const int64_t *voff_host,
                          bbtc_graph_t *out);

}  // namespace
}  // namespace bbtc

using namespace bbtc;

extern "C" {

void bbtc_opts_init(bbtc_opts *opts) {
  if (!opts) return;
  memset(opts, 0, sizeof(*opts));
  opts->struct_size = sizeof(bbtc_opts);
  opts->kernel = BBTC_KERNEL_AUTO;
}

const char *bbtc_last_error(void) { return g_error; }

uint64_t bbtc_num_tasks(int32_t p) {
  if (p < 1) return 0;
  return (uint64_t)p * (uint64_t)(p + 1) * (uint64_t)(p + 2) / 6;
}

}  // extern "C"

namespace bbtc {
namespace {

bbtc_status create_common(int64_t n, const int64_t *rowptr, const int32_t *colidx,
                          uint32_t flags, void *stream, int32_t ng, const int64_t *voff_host,
                          bbtc_graph_t *out) {
  if (!out) {
    set_error("bbtc_graph_create: out is NULL");
    return BBTC_EINVAL;
  }
  if (n < 0 || n > 0x7fffffffLL) {
    set_error("bbtc_graph_create: n = %lld is outside [0, 2^31 - 1]", (long long)n);
    return BBTC_EINVAL;
  }
  if (flags & ~(BBTC_INPUT_DEVICE | BBTC_INPUT_SYMMETRIC)) {
    set_error("bbtc_graph_create: unknown flags 0x%x", flags);
    return BBTC_EINVAL;
  }
  if (!rowptr) {
    set_error("bbtc_graph_create: rowptr is NULL");
    return BBTC_EINVAL;
  }
  const bool on_device = (flags & BBTC_INPUT_DEVICE) != 0;
  bbtc_graph *g = new (std::nothrow) bbtc_graph();
  if (!g) {
    set_error("bbtc_graph_create: host allocation failed");
    return BBTC_ENOMEM;
  }
  cudaGetDevice(&g->device);
  g->n = n;
  g->ng = ng;
  if (stream) {
    g->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("bbtc_graph_create: cudaStreamCreate failed");
      delete g;
      return BBTC_ECUDA;
    }
    g->own_stream = true;
  }
  cudaStream_t s = g->stream;
  for (cudaEvent_t &e : g->ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      set_error("bbtc_graph_create: cudaEventCreate failed");
      destroy_graph(g);
      return BBTC_ECUDA;
    }
  }
  bbtc_status st = BBTC_OK;
  if (voff_host) {
    if (dalloc_n(&g->voff, ng + 1, s) != BBTC_OK ||
        cudaMemcpyAsync(g->voff, voff_host, sizeof(int64_t) * (size_t)(ng + 1),
                        cudaMemcpyHostToDevice, s) != cudaSuccess) {
      set_error("bbtc_graph_create_batch: copying the vertex offsets failed");
      destroy_graph(g);
      return BBTC_ENOMEM;
    }
    g->bytes += (uint64_t)(ng + 1) * 8;
  }
  int64_t nnz = 0;
  int64_t *d_rowptr = nullptr;
  int32_t *d_colidx = nullptr;
  bool copied = false;
  do {
    if (on_device) {
      if (cudaMemcpyAsync(&nnz, rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
              cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("bbtc_graph_create: reading rowptr[n] from the device failed");
        st = BBTC_ECUDA;
        break;
      }
    } else {
      nnz = rowptr[n];
    }
    if (nnz < 0) {
      set_error("bbtc_graph_create: rowptr[n] = %lld is negative", (long long)nnz);
      st = BBTC_EINVAL;
      break;
    }
    if (nnz > 0 && !colidx) {
      set_error("bbtc_graph_create: colidx is NULL with %lld entries", (long long)nnz);
      st = BBTC_EINVAL;
      break;
    }
    if (on_device) {
      d_rowptr = const_cast<int64_t *>(rowptr);
      d_colidx = const_cast<int32_t *>(colidx);
    } else {
      copied = true;
      if ((st = dalloc_n(&d_rowptr, n + 1, s)) != BBTC_OK) break;
      if ((st = dalloc_n(&d_colidx, nnz, s)) != BBTC_OK) break;
      if (cudaMemcpyAsync(d_rowptr, rowptr, sizeof(int64_t) * (size_t)(n + 1),
                          cudaMemcpyHostToDevice, s) != cudaSuccess ||
          (nnz > 0 && cudaMemcpyAsync(d_colidx, colidx, sizeof(int32_t) * (size_t)nnz,
                                      cudaMemcpyHostToDevice, s) != cudaSuccess)) {
        set_error("bbtc_graph_create: host-to-device copy failed");
        st = BBTC_ECUDA;
        break;
      }
    }
    if (cudaEventRecord(g->ev[0], s) != cudaSuccess) {
      set_error("bbtc_graph_create: cudaEventRecord failed");
      st = BBTC_ECUDA;
      break;
    }
    st = prepare_graph(g, d_rowptr, d_colidx, nnz, (flags & BBTC_INPUT_SYMMETRIC) != 0);
    if (st == BBTC_OK && cudaEventRecord(g->ev[1], s) != cudaSuccess) {
      set_error("bbtc_graph_create: cudaEventRecord failed");
      st = BBTC_ECUDA;
    }
  } while (0);
  if (copied) {
    dfree(d_rowptr, s);
    dfree(d_colidx, s);
  }
  if (st == BBTC_OK && cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("bbtc_graph_create: %s", cudaGetErrorString(cudaGetLastError()));
    st = BBTC_ECUDA;
  }
  if (st != BBTC_OK) {
    destroy_graph(g);
    return st;
  }
  *out = g;
  return BBTC_OK;
}

}  // namespace
}  // namespace bbtc

extern "C" {

bbtc_status bbtc_graph_create_async(int64_t n, const int64_t *rowptr, const int32_t *colidx,
                                    uint32_t flags, void *stream, bbtc_graph_t *out) {
  clear_error();
  return create_common(n, rowptr, colidx, flags, stream, 1, nullptr, out);
}

bbtc_status bbtc_graph_create_batch(int32_t ng, const int64_t *vertex_offsets,
                                    const int64_t *rowptr, const int32_t *colidx, uint32_t flags,
                                    void *stream, bbtc_graph_t *out) {
  clear_error();
  if (ng < 1 || !vertex_offsets) {
    set_error("bbtc_graph_create_batch: ng = %d must be >= 1 with vertex offsets", ng);
    return BBTC_EINVAL;
  }
  if (vertex_offsets[0] != 0) {
    set_error("bbtc_graph_create_batch: vertex_offsets[0] must be 0");
    return BBTC_EINVAL;
  }
  for (int32_t i = 0; i < ng; ++i)
    if (vertex_offsets[i + 1] < vertex_offsets[i]) {
      set_error("bbtc_graph_create_batch: vertex_offsets decrease at graph %d", i);
      return BBTC_EINVAL;
    }
  return create_common(vertex_offsets[ng], rowptr, colidx, flags, stream, ng, vertex_offsets,
                       out);
}

bbtc_status bbtc_graph_create(int64_t n, const int64_t *rowptr, const int32_t *colidx,
                              uint32_t flags, bbtc_graph_t *out) {
  return bbtc_graph_create_async(n, rowptr, colidx, flags, nullptr, out);
}

void bbtc_graph_destroy(bbtc_graph_t g) {
  if (!g) return;
  DeviceGuard dg(g->device);
  destroy_graph(g);
}

bbtc_status bbtc_count(bbtc_graph_t g, const bbtc_opts *opts_in, uint64_t *count) {
  clear_error();
  if (!g || !count) {
    set_error("bbtc_count: NULL handle or count");
    return BBTC_EINVAL;
  }
  bbtc_opts opts;
  BBTC_TRY(check_opts(opts_in, &opts));
  DeviceGuard dg(g->device);
  const bool budgeted = opts.device_budget_bytes != 0;
  const int p = opts.p == 0 ? default_p(g, budgeted) : opts.p;
  cudaStream_t s = opts.stream ? (cudaStream_t)opts.stream : g->stream;
  if (budgeted && opts.per_edge_out) {
    set_error("bbtc_count: per_edge_out needs a resident count (device_budget_bytes = 0)");
    return BBTC_EINVAL;
  }
  // a resident count needs the block arrays on the device: a plan that was
  // streamed (its arrays now in host memory) is rebuilt
  if (!budgeted && g->plan.streamed) free_plan(&g->plan, s);
  const bool rebuild =
      !plan_matches(g->plan, p, opts.kernel, opts.hash_threshold, opts.chunk, opts.partition);
  if (rebuild) BBTC_CUDA(cudaEventRecord(g->ev[2], s));
  BBTC_TRY(build_plan(g, p, opts.kernel, opts.hash_threshold, opts.chunk, s, opts.partition));
  if (rebuild) BBTC_CUDA(cudaEventRecord(g->ev[3], s));
  g->plan_timed = rebuild;
  const Plan &pl = g->plan;
  Scratch scratch(s);
  unsigned long long *vertex_count = nullptr;
  if (opts.per_vertex_out) BBTC_TRY(scratch.get(&vertex_count, g->n));
  unsigned long long *task_cycles = nullptr;
  if (opts.per_task_cycles_out) {
    BBTC_TRY(scratch.get(&task_cycles, pl.ntasks));
    BBTC_CUDA(cudaMemsetAsync(task_cycles, 0, sizeof(uint64_t) * (size_t)pl.ntasks, s));
  }
  unsigned *edge_sup = nullptr;
  if (opts.per_edge_out) {
    BBTC_TRY(scratch.get(&edge_sup, g->m > 0 ? g->m : 1));
    BBTC_CUDA(cudaMemsetAsync(edge_sup, 0, sizeof(unsigned) * (size_t)(g->m > 0 ? g->m : 1), s));
  }
  const bool per_graph = opts.per_graph_out != nullptr;
  uint8_t *task_mask = nullptr;  // this caller's share of the tasks, on the device
  if (opts.task_mask) {
    BBTC_TRY(scratch.get(&task_mask, pl.ntasks));
    BBTC_CUDA(cudaMemcpyAsync(task_mask, opts.task_mask, (size_t)pl.ntasks,
                              cudaMemcpyHostToDevice, s));
  }
  if (budgeted) {
    StreamStats st;
    BBTC_TRY(run_count_streamed(g, g->plan, opts.device_budget_bytes, vertex_count, per_graph,
                                opts.timeout_ms, s, &st, task_cycles, task_mask));
    g->stream_stats.rounds = st.rounds;
    g->stream_stats.h2d_bytes = st.h2d_bytes;
    g->stream_stats.copy_ms = st.copy_ms;
    g->stream_stats.block_bytes = st.block_bytes;
    g->stream_stats.device_peak = st.device_peak;
    g->stream_stats.mode = st.mode;
    g->stream_stats_total_ms = st.total_ms;
  } else {
    BBTC_TRY(run_count(g, pl, vertex_count, per_graph, opts.timeout_ms, s, g->ev[4], g->ev[5],
                       task_cycles, edge_sup, task_mask));
    g->stream_stats_total_ms = -1.0;
  }
  unsigned long long head[SCR_TASKS] = {0, 0, 0};
  BBTC_CUDA(cudaMemcpyAsync(head, pl.scratch, sizeof(head), cudaMemcpyDeviceToHost, s));
  BBTC_CUDA(cudaStreamSynchronize(s));
  if ((int32_t)head[SCR_STATUS] != 0) return count_status_error("bbtc_count", (int32_t)head[SCR_STATUS], opts.timeout_ms);
  const bool out_dev = (opts.flags & BBTC_OUT_DEVICE) != 0;
  const cudaMemcpyKind kind = out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (opts.per_task_out)
    BBTC_CUDA(cudaMemcpyAsync(opts.per_task_out, pl.scratch + SCR_TASKS,
                              sizeof(uint64_t) * (size_t)pl.ntasks, kind, s));
  if (per_graph)
    BBTC_CUDA(cudaMemcpyAsync(opts.per_graph_out, pl.scratch + SCR_TASKS + pl.ntasks,
                              sizeof(uint64_t) * (size_t)g->ng, kind, s));
  if (task_cycles)
    BBTC_CUDA(cudaMemcpyAsync(opts.per_task_cycles_out, task_cycles,
                              sizeof(uint64_t) * (size_t)pl.ntasks, kind, s));
  if (edge_sup && g->m > 0)  // resident plans index the oriented CSR directly
    BBTC_CUDA(cudaMemcpyAsync(opts.per_edge_out, edge_sup, sizeof(uint32_t) * (size_t)g->m, kind,
                              s));
  if (opts.per_vertex_out && g->n > 0) {
    unsigned long long *by_id = nullptr;
    BBTC_TRY(scratch.get(&by_id, g->n));
    k_scatter_by_perm<<<grid_for(g->n, 256, 16), 256, 0, s>>>(vertex_count, g->perm, g->n,
                                                              by_id);
    BBTC_LAUNCH_CHECK();
    BBTC_CUDA(cudaMemcpyAsync(opts.per_vertex_out, by_id, sizeof(uint64_t) * (size_t)g->n, kind,
                              s));
  }
  BBTC_CUDA(cudaStreamSynchronize(s));
  *count = head[SCR_TOTAL];
  return BBTC_OK;
}

bbtc_status bbtc_count_async(bbtc_graph_t g, const bbtc_opts *opts_in, uint64_t *total_dev) {
  clear_error();
  if (!g || !total_dev) {
    set_error("bbtc_count_async: NULL handle or total_dev");
    return BBTC_EINVAL;
  }
  bbtc_opts opts;
  BBTC_TRY(check_opts(opts_in, &opts));
  const int p = opts.p == 0 ? default_p(g) : opts.p;
  if (!plan_matches(g->plan, p, opts.kernel, opts.hash_threshold, opts.chunk, opts.partition) ||
      g->plan.streamed) {
    set_error("bbtc_count_async: no resident plan for these options on the handle; build it "
              "with bbtc_count (without a device budget) or bbtc_graph_get_plan first");
    return BBTC_EINVAL;
  }
  if (opts.per_vertex_out || opts.per_task_cycles_out || opts.per_edge_out || opts.task_mask ||
      ((opts.per_task_out || opts.per_graph_out) && !(opts.flags & BBTC_OUT_DEVICE))) {
    set_error("bbtc_count_async: outputs must be device pointers (BBTC_OUT_DEVICE) and "
              "per_vertex_out / per_task_cycles_out / per_edge_out / task_mask must be NULL");
    return BBTC_EINVAL;
  }
  DeviceGuard dg(g->device);
  cudaStream_t s = opts.stream ? (cudaStream_t)opts.stream : g->stream;
  const Plan &pl = g->plan;
  const bool per_graph = opts.per_graph_out != nullptr;
  BBTC_TRY(run_count(g, pl, nullptr, per_graph, 0, s, nullptr, nullptr));
  BBTC_CUDA(cudaMemcpyAsync(total_dev, pl.scratch + SCR_TOTAL, sizeof(uint64_t),
                            cudaMemcpyDeviceToDevice, s));
  if (opts.per_task_out)
    BBTC_CUDA(cudaMemcpyAsync(opts.per_task_out, pl.scratch + SCR_TASKS,
                              sizeof(uint64_t) * (size_t)pl.ntasks, cudaMemcpyDeviceToDevice, s));
  if (per_graph)
    BBTC_CUDA(cudaMemcpyAsync(opts.per_graph_out, pl.scratch + SCR_TASKS + pl.ntasks,
                              sizeof(uint64_t) * (size_t)g->ng, cudaMemcpyDeviceToDevice, s));
  return BBTC_OK;
}

bbtc_status bbtc_graph_plan(bbtc_graph_t g, const bbtc_opts *opts_in) {
  clear_error();
  if (!g) {
    set_error("bbtc_graph_plan: NULL handle");
    return BBTC_EINVAL;
  }
  bbtc_opts opts;
  BBTC_TRY(check_opts(opts_in, &opts));
  DeviceGuard dg(g->device);
  const int p = opts.p == 0 ? default_p(g) : opts.p;
  cudaStream_t s = opts.stream ? (cudaStream_t)opts.stream : g->stream;
  if (g->plan.streamed) free_plan(&g->plan, s);
  BBTC_TRY(build_plan(g, p, opts.kernel, opts.hash_threshold, opts.chunk, s, opts.partition));
  BBTC_CUDA(cudaStreamSynchronize(s));
  return BBTC_OK;
}

bbtc_status bbtc_count_batch(const bbtc_graph_t *gs, int32_t ng, const bbtc_opts *opts,
                             uint64_t *counts, bbtc_status *per_graph) {
  clear_error();
  if (ng < 0 || (ng > 0 && (!gs || !counts))) {
    set_error("bbtc_count_batch: invalid arguments");
    return BBTC_EINVAL;
  }
  if (ng == 0) return BBTC_OK;
  bbtc_opts o;
  BBTC_TRY(check_opts(opts, &o));
  // NULL handles are reported and skipped; the rest are counted together
  bbtc_graph_t *valid = new (std::nothrow) bbtc_graph_t[(size_t)ng];
  int32_t *where = new (std::nothrow) int32_t[(size_t)ng];
  if (!valid || !where) {
    delete[] valid;
    delete[] where;
    set_error("bbtc_count_batch: host allocation failed");
    return BBTC_ENOMEM;
  }
  int32_t nv = 0;
  bbtc_status first = BBTC_OK;
  for (int32_t i = 0; i < ng; ++i) {
    if (gs[i]) {
      where[nv] = i;
      valid[nv++] = gs[i];
      if (per_graph) per_graph[i] = BBTC_OK;
    } else {
      if (per_graph) per_graph[i] = BBTC_EINVAL;
      if (first == BBTC_OK) {
        first = BBTC_EINVAL;
        set_error("bbtc_count_batch: handle %d is NULL", i);
      }
    }
  }
  bbtc_status st = BBTC_OK;
  for (int32_t x = 1; x < nv && st == BBTC_OK; ++x)
    if (valid[x]->device != valid[0]->device) {
      set_error("bbtc_count_batch: handles %d and %d live on different devices", where[0],
                where[x]);
      st = BBTC_EINVAL;
    }
  if (nv > 0 && st == BBTC_OK && o.device_budget_bytes == 0) {
    // resident: every handle keeps (or first builds) its own plan, and one
    // launch drains the work items of all of them
    DeviceGuard dg(valid[0]->device);
    cudaStream_t s = o.stream ? (cudaStream_t)o.stream : valid[0]->stream;
    for (int32_t x = 0; x < nv && st == BBTC_OK; ++x) {
      bbtc_graph *h = valid[x];
      const int p = o.p == 0 ? default_p(h) : o.p;
      if (h->plan.streamed) free_plan(&h->plan, s);
      st = build_plan(h, p, o.kernel, o.hash_threshold, o.chunk, s, o.partition);
    }
    uint64_t *sub = st == BBTC_OK ? new (std::nothrow) uint64_t[(size_t)nv] : nullptr;
    if (st == BBTC_OK && !sub) st = BBTC_ENOMEM;
    if (st == BBTC_OK) st = count_plans(valid, nv, o.timeout_ms, s, sub);
    if (st == BBTC_OK)
      for (int32_t x = 0; x < nv; ++x) counts[where[x]] = sub[x];
    if (st != BBTC_OK && per_graph)
      for (int32_t x = 0; x < nv; ++x) per_graph[where[x]] = st;
    delete[] sub;
  } else if (nv > 0 && st == BBTC_OK) {
    // under a device budget: count the union of the handles, streamed
    DeviceGuard dg(valid[0]->device);
    cudaStream_t s = o.stream ? (cudaStream_t)o.stream : valid[0]->stream;
    bbtc_graph *u = nullptr;
    st = union_of(valid, nv, s, &u);
    uint64_t *sub = st == BBTC_OK ? new (std::nothrow) uint64_t[(size_t)nv] : nullptr;
    if (st == BBTC_OK && !sub) st = BBTC_ENOMEM;
    if (st == BBTC_OK) {
      bbtc_opts uo = o;
      uo.per_task_out = nullptr;
      uo.per_vertex_out = nullptr;
      uo.per_task_cycles_out = nullptr;
      uo.per_edge_out = nullptr;
      uo.task_mask = nullptr;  // the union's tasks are not the caller's
      uo.per_graph_out = sub;
      uo.flags = 0;
      uo.stream = s;
      uint64_t total = 0;
      st = bbtc_count(u, &uo, &total);
      if (st == BBTC_OK)
        for (int32_t x = 0; x < nv; ++x) counts[where[x]] = sub[x];
    }
    if (st != BBTC_OK && per_graph)
      for (int32_t x = 0; x < nv; ++x) per_graph[where[x]] = st;
    delete[] sub;
    if (u) destroy_graph(u);
  }
  delete[] valid;
  delete[] where;
  return st != BBTC_OK ? st : first;
}

bbtc_status bbtc_graph_get_info(bbtc_graph_t g, bbtc_graph_info *info) {
  clear_error();
  if (!g || !info) {
    set_error("bbtc_graph_get_info: NULL argument");
    return BBTC_EINVAL;
  }
  info->n = g->n;
  info->m = g->m;
  info->dplus_max = g->dplus_max;
  info->deg_max = g->deg_max;
  info->device_bytes = g->bytes + g->plan.bytes;
  if (!g->wedges_known) {
    DeviceGuard dg(g->device);
    BBTC_TRY(wedge_sums(g, &g->wedges_in, &g->wedges_out, g->stream));
    g->wedges_known = true;
  }
  info->wedges_in = g->wedges_in;
  info->wedges_out = g->wedges_out;
  info->num_graphs = g->ng;
  return BBTC_OK;
}

bbtc_status bbtc_device_memory(int32_t device, uint64_t *available, uint64_t *total,
                               uint64_t *pool_reserved, uint64_t *pool_used) {
  clear_error();
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    set_error("bbtc_device_memory: no device %d", device);
    return BBTC_EINVAL;
  }
  DeviceGuard dg(device);
  size_t free_b = 0, total_b = 0;
  BBTC_CUDA(cudaMemGetInfo(&free_b, &total_b));
  cudaMemPool_t pool;
  BBTC_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
  uint64_t reserved = 0, used = 0;
  BBTC_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
  BBTC_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
  // idle blocks kept by the library's cache are part of the pool's used bytes
  // but are handed out again (or released) on demand
  const uint64_t idle = cached_block_bytes(device);
  if (idle <= used) used -= idle;
  if (available) *available = (uint64_t)free_b + (reserved > used ? reserved - used : 0);
  if (total) *total = (uint64_t)total_b;
  if (pool_reserved) *pool_reserved = reserved;
  if (pool_used) *pool_used = used;
  return BBTC_OK;
}

bbtc_status bbtc_graph_get_timings(bbtc_graph_t g, bbtc_timings *t) {
  clear_error();
  if (!g || !t) {
    set_error("bbtc_graph_get_timings: NULL argument");
    return BBTC_EINVAL;
  }
  DeviceGuard dg(g->device);
  auto elapsed = [](cudaEvent_t a, cudaEvent_t b) -> double {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
      cudaGetLastError();
      return 0.0;
    }
    return (double)ms;
  };
  t->prep_ms = elapsed(g->ev[0], g->ev[1]);
  t->plan_ms = g->plan_timed ? elapsed(g->ev[2], g->ev[3]) : 0.0;
  t->count_ms = g->stream_stats_total_ms >= 0 ? g->stream_stats_total_ms
                                              : elapsed(g->ev[4], g->ev[5]);
  t->work_items = g->plan.nitems;
  t->stream_rounds = g->stream_stats.rounds;
  t->stream_h2d_bytes = g->stream_stats.h2d_bytes;
  t->stream_copy_ms = g->stream_stats.copy_ms;
  t->stream_block_bytes = g->stream_stats.block_bytes;
  t->stream_device_peak_bytes = g->stream_stats.device_peak;
  t->stream_mode = g->stream_stats.mode;
  return BBTC_OK;
}

uint64_t bbtc_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

bbtc_status bbtc_graph_get_oriented(bbtc_graph_t g, int64_t *rowptr, int32_t *colidx,
                                    int32_t *perm, int64_t *degree) {
  clear_error();
  if (!g) {
    set_error("bbtc_graph_get_oriented: NULL handle");
    return BBTC_EINVAL;
  }
  DeviceGuard dg(g->device);
  cudaStream_t s = g->stream;
  if (rowptr)
    BBTC_CUDA(cudaMemcpyAsync(rowptr, g->rowptr, sizeof(int64_t) * (size_t)(g->n + 1),
                              cudaMemcpyDeviceToHost, s));
  if (colidx && g->m > 0)
    BBTC_CUDA(cudaMemcpyAsync(colidx, g->colidx, sizeof(int32_t) * (size_t)g->m,
                              cudaMemcpyDeviceToHost, s));
  if (perm && g->n > 0)
    BBTC_CUDA(cudaMemcpyAsync(perm, g->perm, sizeof(int32_t) * (size_t)g->n,
                              cudaMemcpyDeviceToHost, s));
  int32_t *deg32 = nullptr;
  if (degree && g->n > 0) {
    deg32 = new (std::nothrow) int32_t[(size_t)g->n];
    if (!deg32) {
      set_error("bbtc_graph_get_oriented: host allocation failed");
      return BBTC_ENOMEM;
    }
    if (cudaMemcpyAsync(deg32, g->deg, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToHost,
                        s) != cudaSuccess) {
      delete[] deg32;
      set_error("bbtc_graph_get_oriented: copy failed");
      return BBTC_ECUDA;
    }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (deg32) {
    for (int64_t v = 0; v < g->n; ++v) degree[v] = deg32[v];
    delete[] deg32;
  }
  if (e != cudaSuccess) {
    set_error("bbtc_graph_get_oriented: %s", cudaGetErrorString(e));
    return BBTC_ECUDA;
  }
  return BBTC_OK;
}

bbtc_status bbtc_graph_get_plan(bbtc_graph_t g, int32_t p, int32_t *cuts, int64_t *block_nnz,
                                int32_t *tasks, double *estimate, int32_t *order) {
  clear_error();
  if (!g || p < 1 || p > 64) {
    set_error("bbtc_graph_get_plan: NULL handle or p outside 1..64");
    return BBTC_EINVAL;
  }
  DeviceGuard dg(g->device);
  cudaStream_t s = g->stream;
  const int kmode = g->plan.p == p ? g->plan.kernel_mode : BBTC_KERNEL_AUTO;
  const int thr = g->plan.p == p ? g->plan.hash_threshold : 16;
  const int chunk = g->plan.p == p ? g->plan.chunk_req : 0;
  const int part = g->plan.p == p ? g->plan.partition : BBTC_PARTITION_EDGES;
  BBTC_TRY(build_plan(g, p, kmode, thr, chunk, s, part));
  const Plan &pl = g->plan;
  if (cuts)
    BBTC_CUDA(cudaMemcpyAsync(cuts, pl.cuts, sizeof(int32_t) * (size_t)(p + 1),
                              cudaMemcpyDeviceToHost, s));
  int64_t *boff = nullptr;
  if (block_nnz) {
    boff = new (std::nothrow) int64_t[(size_t)p * (p + 1)];
    if (!boff) {
      set_error("bbtc_graph_get_plan: host allocation failed");
      return BBTC_ENOMEM;
    }
    if (cudaMemcpyAsync(boff, pl.boff, sizeof(int64_t) * (size_t)p * (p + 1),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess) {
      delete[] boff;
      set_error("bbtc_graph_get_plan: copy failed");
      return BBTC_ECUDA;
    }
  }
  if (tasks)
    BBTC_CUDA(cudaMemcpyAsync(tasks, pl.tasks, sizeof(int32_t) * 3 * (size_t)pl.ntasks,
                              cudaMemcpyDeviceToHost, s));
  if (estimate)
    BBTC_CUDA(cudaMemcpyAsync(estimate, pl.est, sizeof(double) * (size_t)pl.ntasks,
                              cudaMemcpyDeviceToHost, s));
  if (order)
    BBTC_CUDA(cudaMemcpyAsync(order, pl.order, sizeof(int32_t) * (size_t)pl.ntasks,
                              cudaMemcpyDeviceToHost, s));
  cudaError_t e = cudaStreamSynchronize(s);
  if (boff) {
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j)
        block_nnz[i * p + j] = boff[i * (p + 1) + j + 1] - boff[i * (p + 1) + j];
    delete[] boff;
  }
  if (e != cudaSuccess) {
    set_error("bbtc_graph_get_plan: %s", cudaGetErrorString(e));
    return BBTC_ECUDA;
  }
  return BBTC_OK;
}

}  // extern "C"
