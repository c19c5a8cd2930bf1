// stream.cu -- a11: counting with the blocks streamed from pinned host memory.
//
// When a caller gives bbtc_count a device budget, the plan's block arrays
// (each block G_ab's row pointers and columns, and each block's in-edge
// records) move to pinned host memory, and the plan's work items are put in
// Alg. 4's task order, so that the tasks (i, j, k), k >= j, which share the
// in-edge block of G_ij, are consecutive. The counting step then holds at
// most `budget` bytes of blocks on the device, in one pool, in one of two
// ways:
//  1. When every block CSR fits in the pool beside two in-edge buffers, the
//     block CSRs are copied once and stay, and the in-edge blocks are copied
//     once each, group by group (one group = the tasks of one G_ij): the next
//     group's in-edges are copied on a copy stream into the other buffer
//     while the current group counts (the paper's prefetch of the next task's
//     blocks, Alg. 7). Every block crosses to the device exactly once.
//  2. Otherwise, tasks are taken in that order in rounds: a round is the
//     longest run of consecutive tasks whose blocks are either already in the
//     pool or fit beside the blocks of the round still being counted. Blocks
//     sit at fixed offsets; one still in the pool when a later round needs it
//     is used in place, and one that was overwritten is copied again. Round
//     r+1's copies overlap round r's count.
// Each task's descriptor is rewritten to point at its blocks in the pool.
// Counts accumulate across rounds exactly as in one launch.
#include <stdio.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "graph.cuh"

namespace bbtc {

namespace {

constexpr size_t ALIGN = 256;

inline size_t align_up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }

// Pinned host buffers are kept for reuse once a streamed plan lets them go:
// pinning tens of GB costs seconds (page by page), far more than the copies,
// and a caller that streams one graph after another needs buffers of the
// same sizes again. A request takes the smallest cached buffer that holds it
// and is at most twice its size; released buffers stay cached up to
// PINNED_KEEP bytes in total, and the rest are freed.
constexpr size_t PINNED_KEEP = 64ull << 30;

struct PinnedCache {
  std::mutex mu;
  std::multimap<size_t, void *> free_by_size;
  std::map<void *, size_t> size_of;
  size_t cached = 0;
};

PinnedCache &pinned_cache() {
  static PinnedCache *c = new PinnedCache;  // never destroyed: safe during exit
  return *c;
}

cudaError_t pinned_alloc(void **ptr, size_t bytes) {
  PinnedCache &c = pinned_cache();
  {
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.free_by_size.lower_bound(bytes);
    if (it != c.free_by_size.end() && it->first <= 2 * bytes) {
      *ptr = it->second;
      c.cached -= it->first;
      c.free_by_size.erase(it);
      return cudaSuccess;
    }
  }
  cudaError_t e = cudaHostAlloc(ptr, bytes, cudaHostAllocDefault);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(c.mu);
    c.size_of[*ptr] = bytes;
  }
  return e;
}

void pinned_release(void *ptr) {
  if (!ptr) return;
  PinnedCache &c = pinned_cache();
  std::lock_guard<std::mutex> lk(c.mu);
  auto it = c.size_of.find(ptr);
  if (it == c.size_of.end()) return;
  const size_t bytes = it->second;
  if (c.cached + bytes <= PINNED_KEEP) {
    c.free_by_size.emplace(bytes, ptr);
    c.cached += bytes;
  } else {
    c.size_of.erase(it);
    cudaFreeHost(ptr);
  }
}

template <typename T>
bbtc_status to_pinned(T **host, T **dev, int64_t count, cudaStream_t s) {
  const size_t bytes = sizeof(T) * (size_t)(count > 0 ? count : 1);
  BBTC_CUDA(pinned_alloc(reinterpret_cast<void **>(host), bytes));
  if (count > 0) BBTC_CUDA(cudaMemcpyAsync(*host, *dev, sizeof(T) * (size_t)count,
                                           cudaMemcpyDeviceToHost, s));
  return BBTC_OK;
}

// Moves the block arrays of a resident plan to pinned host memory, as
// physical per-block copies.
bbtc_status plan_to_host(const bbtc_graph *g, Plan &pl, int64_t m, cudaStream_t s) {
  if (pl.streamed) return BBTC_OK;
  BBTC_TRY(plan_physical_blocks(g, pl, s));
  BBTC_TRY(to_pinned(&pl.h_rp, &pl.rp, pl.total_rp, s));
  BBTC_TRY(to_pinned(&pl.h_ci, &pl.ci, m, s));
  BBTC_TRY(to_pinned(&pl.h_ie, &pl.ie, m, s));
  BBTC_CUDA(cudaStreamSynchronize(s));
  dfree(pl.rp, s);
  dfree(pl.ci, s);
  dfree(pl.ie, s);
  pl.rp = nullptr;
  pl.ci = nullptr;
  pl.ie = nullptr;
  // work items in Alg. 4 task order (a task's items stay together and keep
  // their order), so that the tasks sharing an in-edge block are consecutive
  if (pl.nitems > 0) {
    std::vector<WorkItem> items((size_t)pl.nitems);
    BBTC_CUDA(cudaMemcpyAsync(items.data(), pl.items, sizeof(WorkItem) * items.size(),
                              cudaMemcpyDeviceToHost, s));
    BBTC_CUDA(cudaStreamSynchronize(s));
    std::stable_sort(items.begin(), items.end(),
                     [](const WorkItem &a, const WorkItem &b) { return a.task < b.task; });
    BBTC_CUDA(cudaMemcpyAsync(pl.items, items.data(), sizeof(WorkItem) * items.size(),
                              cudaMemcpyHostToDevice, s));
    BBTC_CUDA(cudaStreamSynchronize(s));
  }
  pl.streamed = true;
  return BBTC_OK;
}

// A block in the pool: kind 0 = BCSR block (a, b) (row pointers, then
// columns), kind 1 = in-edge records of block (a, b).
struct BlockKey {
  int kind, a, b;
  bool operator<(const BlockKey &o) const {
    return kind != o.kind ? kind < o.kind : (a != o.a ? a < o.a : b < o.b);
  }
};

struct Run {  // the work items of one task, in plan order
  int32_t task;
  int64_t item0, item1;
};

}  // namespace

void free_plan_host(Plan *pl) {
  pinned_release(pl->h_rp);
  pinned_release(pl->h_ci);
  pinned_release(pl->h_ie);
  pl->h_rp = nullptr;
  pl->h_ci = nullptr;
  pl->h_ie = nullptr;
}

bbtc_status run_count_streamed(bbtc_graph *g, Plan &pl, uint64_t budget,
                               unsigned long long *vertex_count, bool per_graph,
                               uint32_t timeout_ms, cudaStream_t s, StreamStats *stats,
                               unsigned long long *task_cycles, const uint8_t *task_mask) {
  const int p = pl.p;
  const int64_t nt = pl.ntasks;
  BBTC_TRY(plan_to_host(g, pl, g->m, s));
  // a budgeted count holds no idle cached blocks: the device memory it uses,
  // and the high-water mark it reports, are its own
  release_cached_blocks(g->device, s);

  // small plan tables on the host
  std::vector<WorkItem> items((size_t)pl.nitems);
  std::vector<int64_t> boff((size_t)p * (p + 1));
  if (pl.nitems > 0)
    BBTC_CUDA(cudaMemcpyAsync(items.data(), pl.items, sizeof(WorkItem) * (size_t)pl.nitems,
                              cudaMemcpyDeviceToHost, s));
  BBTC_CUDA(cudaMemcpyAsync(boff.data(), pl.boff, sizeof(int64_t) * boff.size(),
                            cudaMemcpyDeviceToHost, s));
  BBTC_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> ti((size_t)nt), tj((size_t)nt), tk((size_t)nt);
  {
    int64_t t = 0;
    for (int i = 0; i < p; ++i)
      for (int j = i; j < p; ++j)
        for (int k = j; k < p; ++k, ++t) {
          ti[(size_t)t] = i;
          tj[(size_t)t] = j;
          tk[(size_t)t] = k;
        }
  }
  std::vector<Run> runs;
  for (int64_t x = 0; x < pl.nitems; ++x) {
    if (runs.empty() || runs.back().task != items[(size_t)x].task)
      runs.push_back(Run{items[(size_t)x].task, x, x});
    runs.back().item1 = x + 1;
  }

  auto vsize = [&](int a) -> int64_t { return (int64_t)(pl.h_cuts[a + 1] - pl.h_cuts[a]); };
  auto col0 = [&](int a, int b) -> int64_t { return (int64_t)pl.h_rp[pl.h_rpb[a * p + b]]; };
  auto col1 = [&](int a, int b) -> int64_t {
    return (int64_t)pl.h_rp[pl.h_rpb[a * p + b] + vsize(a)];
  };
  auto ie0 = [&](int a, int b) -> int64_t { return boff[(size_t)(a * (p + 1) + b)]; };
  auto ie1 = [&](int a, int b) -> int64_t { return boff[(size_t)(a * (p + 1) + b + 1)]; };
  auto block_bytes = [&](const BlockKey &k) -> size_t {
    if (k.kind == 0)
      return align_up(4 * (size_t)(vsize(k.a) + 1)) + align_up(4 * (size_t)(col1(k.a, k.b) - col0(k.a, k.b)));
    return align_up(sizeof(InEdge) * (size_t)(ie1(k.a, k.b) - ie0(k.a, k.b)));
  };

  // totals: every block once (exact bytes, as counted in h2d_bytes)
  uint64_t csr_exact = 0, ie_exact = 0;
  size_t csr_total = 0, ie_max = 0;
  for (int a = 0; a < p; ++a)
    for (int b = a; b < p; ++b) {
      csr_exact += 4 * (uint64_t)(vsize(a) + 1 + col1(a, b) - col0(a, b));
      ie_exact += sizeof(InEdge) * (uint64_t)(ie1(a, b) - ie0(a, b));
      csr_total += block_bytes(BlockKey{0, a, b});
      ie_max = std::max(ie_max, block_bytes(BlockKey{1, a, b}));
    }
  stats->block_bytes = csr_exact + ie_exact;

  // The pool holds blocks at fixed offsets. A round's blocks that are already
  // in the pool (copied for an earlier round and not overwritten since) are
  // used in place; the others go to free space, where a block may overwrite
  // only blocks that neither the round in flight nor this round uses. The
  // copies of round r wait for the kernel of round r-2 (every kernel that may
  // have read what they overwrite), so they overlap the kernel of round r-1.
  const size_t pool_bytes = (size_t)budget & ~(ALIGN - 1);
  Scratch scratch(s);
  unsigned char *pool = nullptr;
  BBTC_TRY(scratch.get(&pool, (int64_t)pool_bytes));
  struct Slot {
    size_t off, size;
    int64_t round;  // last round that uses the block
  };
  const bool csr_resident = csr_total + 2 * ie_max <= pool_bytes;
  stats->mode = csr_resident ? 1 : 2;
  cudaMemPool_t mem_pool = nullptr;
  {
    int dev = 0;
    uint64_t zero = 0;  // resets the high-water mark to the memory in use now
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetDefaultMemPool(&mem_pool, dev) == cudaSuccess)
      cudaMemPoolSetAttribute(mem_pool, cudaMemPoolAttrUsedMemHigh, &zero);
    else
      mem_pool = nullptr;
  }
  std::map<BlockKey, Slot> placed;
  cudaStream_t cs = nullptr;
  cudaEvent_t copy_done[2] = {nullptr, nullptr}, kern_done[2] = {nullptr, nullptr};
  cudaEvent_t t_begin = nullptr, t_end = nullptr;
  TaskDesc *stage[2] = {nullptr, nullptr};  // pinned staging of descriptors, by round parity
  bbtc_status st = BBTC_OK;
  bool used_parity[2] = {false, false};
  int64_t round = 0;
  float copy_ms_total = 0.f;
  do {
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&copy_done[0]) != cudaSuccess ||
        cudaEventCreate(&copy_done[1]) != cudaSuccess ||
        cudaEventCreate(&kern_done[0]) != cudaSuccess ||
        cudaEventCreate(&kern_done[1]) != cudaSuccess || cudaEventCreate(&t_begin) != cudaSuccess ||
        cudaEventCreate(&t_end) != cudaSuccess ||
        pinned_alloc(reinterpret_cast<void **>(&stage[0]),
                     sizeof(TaskDesc) * (size_t)(nt > 0 ? nt : 1)) != cudaSuccess ||
        pinned_alloc(reinterpret_cast<void **>(&stage[1]),
                     sizeof(TaskDesc) * (size_t)(nt > 0 ? nt : 1)) != cudaSuccess) {
      set_error("streamed count: creating streams, events or staging buffers failed");
      st = BBTC_ECUDA;
      break;
    }
    if ((st = count_reset(g, pl, vertex_count, per_graph, s)) != BBTC_OK) break;
    if (cudaEventRecord(t_begin, s) != cudaSuccess) { st = BBTC_ECUDA; break; }
    if (csr_resident) {
      // mode 1: every block CSR once, then the in-edge blocks group by group
      // into two alternating buffers after them
      std::map<std::pair<int, int>, size_t> csr_off;
      size_t off = 0;
      // event pairs around each batch of copies (not around the waits), summed at the end
      std::vector<std::pair<cudaEvent_t, cudaEvent_t>> copy_ev;
      auto copy_begin = [&]() {
        cudaEvent_t a = nullptr, b = nullptr;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, cs);
        copy_ev.emplace_back(a, b);
      };
      auto copy_end = [&]() { cudaEventRecord(copy_ev.back().second, cs); };
      copy_begin();
      for (int a = 0; a < p && st == BBTC_OK; ++a)
        for (int b = a; b < p; ++b) {
          csr_off[{a, b}] = off;
          const int64_t nrp = vsize(a) + 1, c0i = col0(a, b), nci = col1(a, b) - c0i;
          if (cudaMemcpyAsync(pool + off, pl.h_rp + pl.h_rpb[a * p + b], 4 * (size_t)nrp,
                              cudaMemcpyHostToDevice, cs) != cudaSuccess ||
              (nci > 0 && cudaMemcpyAsync(pool + off + align_up(4 * (size_t)nrp), pl.h_ci + c0i,
                                          4 * (size_t)nci, cudaMemcpyHostToDevice,
                                          cs) != cudaSuccess)) {
            set_error("streamed count: host-to-device block copy failed");
            st = BBTC_ECUDA;
            break;
          }
          stats->h2d_bytes += 4 * (uint64_t)(nrp + nci);
          off += block_bytes(BlockKey{0, a, b});
        }
      copy_end();
      const size_t slot[2] = {csr_total, csr_total + ie_max};
      size_t gpos = 0;
      while (gpos < runs.size() && st == BBTC_OK) {
        // one group: the consecutive tasks that share (i, j), hence G_ij's in-edges
        const int t0 = runs[gpos].task;
        const int i = ti[t0], j = tj[t0];
        size_t gend = gpos;
        while (gend < runs.size() && ti[runs[gend].task] == i && tj[runs[gend].task] == j) ++gend;
        const int h = (int)(round & 1);
        if (used_parity[h]) {  // the kernel of round - 2 read this buffer and stage[h]
          if (cudaStreamWaitEvent(cs, kern_done[h], 0) != cudaSuccess ||
              cudaEventSynchronize(copy_done[h]) != cudaSuccess) {
            st = BBTC_ECUDA;
            break;
          }
        }
        const int64_t x0 = ie0(i, j), len = ie1(i, j) - x0;
        copy_begin();
        if (len > 0 && cudaMemcpyAsync(pool + slot[h], pl.h_ie + x0, sizeof(InEdge) * (size_t)len,
                                       cudaMemcpyHostToDevice, cs) != cudaSuccess) {
          set_error("streamed count: host-to-device block copy failed");
          st = BBTC_ECUDA;
          break;
        }
        stats->h2d_bytes += sizeof(InEdge) * (uint64_t)len;
        for (size_t r = gpos; r < gend && st == BBTC_OK; ++r) {
          const int t = runs[r].task;
          const int k = tk[t];
          const size_t o_ik = csr_off[{i, k}], o_jk = csr_off[{j, k}];
          TaskDesc &d = stage[h][t];
          d.ie = reinterpret_cast<const InEdge *>(pool + slot[h]);
          d.ie_off = x0;
          d.rp_ik = reinterpret_cast<const uint32_t *>(pool + o_ik);
          d.rs_ik = 1;
          d.rs_jk = 1;
          d.ci_ik = reinterpret_cast<const int32_t *>(pool + o_ik +
                                                      align_up(4 * (size_t)(vsize(i) + 1)));
          d.ci_ik_off = col0(i, k);
          d.rp_jk = reinterpret_cast<const uint32_t *>(pool + o_jk);
          d.ci_jk = reinterpret_cast<const int32_t *>(pool + o_jk +
                                                      align_up(4 * (size_t)(vsize(j) + 1)));
          d.ci_jk_off = col0(j, k);
          d.c_i = pl.h_cuts[i];
          d.c_j = pl.h_cuts[j];
          d.diag = k == j;
          d.task = t;
          if (cudaMemcpyAsync(pl.desc + t, &stage[h][t], sizeof(TaskDesc), cudaMemcpyHostToDevice,
                              cs) != cudaSuccess) {
            set_error("streamed count: descriptor copy failed");
            st = BBTC_ECUDA;
          }
        }
        copy_end();
        if (st != BBTC_OK) break;
        if (cudaEventRecord(copy_done[h], cs) != cudaSuccess ||
            cudaStreamWaitEvent(s, copy_done[h], 0) != cudaSuccess) {
          st = BBTC_ECUDA;
          break;
        }
        st = count_launch(g, pl, runs[gpos].item0, runs[gend - 1].item1 - runs[gpos].item0,
                          vertex_count, per_graph, timeout_ms, s, task_cycles, nullptr,
                          task_mask);
        if (st != BBTC_OK) break;
        if (cudaEventRecord(kern_done[h], s) != cudaSuccess) {
          st = BBTC_ECUDA;
          break;
        }
        used_parity[h] = true;
        ++round;
        gpos = gend;
      }
      cudaStreamSynchronize(cs);
      for (auto &ev : copy_ev) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev.first, ev.second) == cudaSuccess) copy_ms_total += ms;
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
      }
    }
    size_t pos = csr_resident ? runs.size() : 0;
    while (pos < runs.size() && st == BBTC_OK) {
      // place blocks for the longest run of tasks that fits next to the
      // blocks of the round in flight (round - 1)
      std::vector<std::pair<BlockKey, Slot>> fresh;  // blocks to copy this round
      auto busy_until = [&](const Slot &sl) { return sl.round >= round - 1; };
      auto find_gap = [&](size_t need, size_t *off) -> bool {
        std::vector<std::pair<size_t, size_t>> used;  // protected intervals
        for (const auto &kv : placed)
          if (busy_until(kv.second)) used.emplace_back(kv.second.off, kv.second.off + kv.second.size);
        for (const auto &f : fresh) used.emplace_back(f.second.off, f.second.off + f.second.size);
        std::sort(used.begin(), used.end());
        size_t at = 0;
        for (const auto &iv : used) {
          if (iv.first >= at + need) break;
          if (iv.second > at) at = iv.second;
        }
        if (at + need > pool_bytes) return false;
        *off = at;
        return true;
      };
      const size_t first = pos;
      while (pos < runs.size()) {
        const int t = runs[pos].task;
        const BlockKey need[3] = {{1, ti[t], tj[t]}, {0, ti[t], tk[t]}, {0, tj[t], tk[t]}};
        const size_t nfresh0 = fresh.size();
        bool ok = true;
        for (int q = 0; q < 3 && ok; ++q) {
          bool have = false;
          for (const auto &f : fresh)
            have = have || (!(f.first < need[q]) && !(need[q] < f.first));
          if (have) continue;
          auto it = placed.find(need[q]);
          if (it != placed.end()) {
            it->second.round = round;  // used in place: protected from now on
            continue;
          }
          size_t off = 0;
          const size_t bytes = block_bytes(need[q]);
          if (!find_gap(bytes, &off)) {
            ok = false;
            break;
          }
          // the new copy overwrites the (unprotected) blocks it overlaps
          for (auto pit = placed.begin(); pit != placed.end();) {
            const Slot &sl = pit->second;
            if (sl.off < off + bytes && off < sl.off + sl.size)
              pit = placed.erase(pit);
            else
              ++pit;
          }
          fresh.push_back({need[q], Slot{off, bytes, round}});
        }
        if (!ok) {
          fresh.resize(nfresh0);
          break;
        }
        ++pos;
      }
      if (pos == first) {
        const int t = runs[pos].task;
        if (round > 0 && !placed.empty()) {
          // nothing fits beside the round in flight: let this round's copies
          // wait for it, then plan with the whole pool
          if (cudaStreamWaitEvent(cs, kern_done[(round - 1) & 1], 0) != cudaSuccess) {
            st = BBTC_ECUDA;
            break;
          }
          placed.clear();
          continue;
        }
        set_error("streamed count: the blocks of task (%d,%d,%d) do not fit in a %llu-byte "
                  "device budget", ti[t], tj[t], tk[t], (unsigned long long)budget);
        st = BBTC_ENOMEM;
        break;
      }
      for (const auto &f : fresh) placed[f.first] = f.second;

      const int h = (int)(round & 1);
      // kernel round-2 read the regions now overwritten and used stage[h]
      if (used_parity[h]) {
        if (cudaStreamWaitEvent(cs, kern_done[h], 0) != cudaSuccess ||
            cudaEventSynchronize(copy_done[h]) != cudaSuccess) {
          st = BBTC_ECUDA;
          break;
        }
      }
      cudaEvent_t c0 = nullptr, c1 = nullptr;
      cudaEventCreate(&c0);
      cudaEventCreate(&c1);
      cudaEventRecord(c0, cs);
      for (const auto &f : fresh) {
        const BlockKey &k = f.first;
        unsigned char *dst = pool + f.second.off;
        cudaError_t e1 = cudaSuccess, e2 = cudaSuccess, e3 = cudaSuccess;
        if (k.kind == 0) {
          const int64_t nrp = vsize(k.a) + 1, c0i = col0(k.a, k.b), nci = col1(k.a, k.b) - c0i;
          e1 = cudaMemcpyAsync(dst, pl.h_rp + pl.h_rpb[k.a * p + k.b], 4 * (size_t)nrp,
                               cudaMemcpyHostToDevice, cs);
          if (nci > 0)
            e2 = cudaMemcpyAsync(dst + align_up(4 * (size_t)nrp), pl.h_ci + c0i, 4 * (size_t)nci,
                                 cudaMemcpyHostToDevice, cs);
          stats->h2d_bytes += 4 * (uint64_t)(nrp + nci);
        } else {
          const int64_t x0 = ie0(k.a, k.b), len = ie1(k.a, k.b) - x0;
          if (len > 0)
            e1 = cudaMemcpyAsync(dst, pl.h_ie + x0, sizeof(InEdge) * (size_t)len,
                                 cudaMemcpyHostToDevice, cs);
          stats->h2d_bytes += sizeof(InEdge) * (uint64_t)len;
        }
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
          set_error("streamed count: host-to-device block copy failed");
          st = BBTC_ECUDA;
          break;
        }
      }
      if (st != BBTC_OK) break;
      // descriptors of the round's tasks, pointing at their blocks in the pool
      for (size_t r = first; r < pos; ++r) {
        const int t = runs[r].task;
        const int i = ti[t], j = tj[t], k = tk[t];
        const size_t o_ie = placed[BlockKey{1, i, j}].off;
        const size_t o_ik = placed[BlockKey{0, i, k}].off;
        const size_t o_jk = placed[BlockKey{0, j, k}].off;
        TaskDesc &d = stage[h][t];
        d.ie = reinterpret_cast<const InEdge *>(pool + o_ie);
        d.ie_off = ie0(i, j);
        d.rp_ik = reinterpret_cast<const uint32_t *>(pool + o_ik);
        d.rs_ik = 1;
        d.rs_jk = 1;
        d.ci_ik = reinterpret_cast<const int32_t *>(pool + o_ik + align_up(4 * (size_t)(vsize(i) + 1)));
        d.ci_ik_off = col0(i, k);
        d.rp_jk = reinterpret_cast<const uint32_t *>(pool + o_jk);
        d.ci_jk = reinterpret_cast<const int32_t *>(pool + o_jk + align_up(4 * (size_t)(vsize(j) + 1)));
        d.ci_jk_off = col0(j, k);
        d.c_i = pl.h_cuts[i];
        d.c_j = pl.h_cuts[j];
        d.diag = k == j;
        d.task = t;
        if (cudaMemcpyAsync(pl.desc + t, &stage[h][t], sizeof(TaskDesc), cudaMemcpyHostToDevice,
                            cs) != cudaSuccess) {
          set_error("streamed count: descriptor copy failed");
          st = BBTC_ECUDA;
          break;
        }
      }
      if (st != BBTC_OK) break;
      cudaEventRecord(c1, cs);
      if (cudaEventRecord(copy_done[h], cs) != cudaSuccess ||
          cudaStreamWaitEvent(s, copy_done[h], 0) != cudaSuccess) {
        st = BBTC_ECUDA;
        break;
      }
      st = count_launch(g, pl, runs[first].item0, runs[pos - 1].item1 - runs[first].item0,
                        vertex_count, per_graph, timeout_ms, s, task_cycles, nullptr, task_mask);
      if (st != BBTC_OK) break;
      if (cudaEventRecord(kern_done[h], s) != cudaSuccess) {
        st = BBTC_ECUDA;
        break;
      }
      used_parity[h] = true;
      ++round;
      // copy time of this round (host waits only for the copy, not the kernel)
      if (cudaEventSynchronize(c1) == cudaSuccess) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c0, c1) == cudaSuccess) copy_ms_total += ms;
      }
      cudaEventDestroy(c0);
      cudaEventDestroy(c1);
    }
    if (st != BBTC_OK) break;
    st = count_finish(pl, s);
    if (st == BBTC_OK && cudaEventRecord(t_end, s) != cudaSuccess) st = BBTC_ECUDA;
  } while (0);
  cudaStreamSynchronize(s);
  if (cs) {
    cudaStreamSynchronize(cs);
    cudaStreamDestroy(cs);
  }
  if (st == BBTC_OK) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t_begin, t_end) == cudaSuccess) stats->total_ms = ms;
  }
  stats->rounds = round;
  stats->copy_ms = copy_ms_total;
  if (mem_pool) {
    uint64_t peak = 0;
    if (cudaMemPoolGetAttribute(mem_pool, cudaMemPoolAttrUsedMemHigh, &peak) == cudaSuccess)
      stats->device_peak = peak;
  }
  for (cudaEvent_t e : {copy_done[0], copy_done[1], kern_done[0], kern_done[1], t_begin, t_end})
    if (e) cudaEventDestroy(e);
  for (TaskDesc *d : stage) pinned_release(d);
  return st;
}

}  // namespace bbtc
