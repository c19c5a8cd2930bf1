// count.cu -- per-task triangle counting (a9) and the reduction of the
// per-task counts (a10).
//
// A task t = (i, j, k) counts, for every edge (u, v) of G_ij, the common
// elements of N(G_ik, u) and N(G_jk, v) (Sec. 4.3, Alg. 5 / Alg. 6). The
// kernel walks G_ij's edges grouped by their destination v (the in-edges of
// each v in V_j that come from V_i, one contiguous range per block) and, for
// each, looks up the elements of N(G_ik, u) that lie above v in N(G_jk, v).
// Elements of N(G_ik, u) at or below v cannot be in N(G_jk, v) (every entry
// of N(v) is above v), so the count equals Alg. 5's |N(G_ik,u) ∩ N(G_jk,v)|.
//
// Work: a persistent grid; each warp takes work items (task, in-edge range)
// from a global counter, heaviest task first, until none remain.
#include <algorithm>
#include <mutex>
#include <vector>

#include "graph.cuh"
#include "primitives.cuh"

namespace bbtc {

namespace {

constexpr int CT_NT = 256;

constexpr int32_t STATUS_TIMEOUT = 1, STATUS_COPY_WAIT = 2;

struct CountParams {
  const TaskDesc *desc;  // per task (Alg. 4 order): where its three blocks live
  const WorkItem *items;
  int64_t nitems;
  unsigned long long *head;
  unsigned long long *task_count;
  unsigned long long *vcount;       // per-vertex counts by position (MODE & 1)
  const int32_t *gid;               // graph of each position (MODE & 2)
  unsigned long long *graph_count;  // per-graph counts (MODE & 2)
  unsigned long long *task_cycles;  // nullable: SM cycles spent on each task's items
  unsigned *edge_sup;               // per-edge support by position in the block columns (MODE & 4)
  const uint8_t *task_mask;         // nullable: items of tasks whose byte is 0 are skipped
  int32_t *status;
  uint64_t timeout_ns;
};

constexpr int MODE_VERTEX = 1, MODE_GRAPH = 2, MODE_EDGE = 4;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Per-warp shared staging area for N(G_jk, v) (int32 slots).
constexpr int STAGE = 2048;
static_assert(STAGE % 4 == 0, "the bitmap is cleared with 16-byte stores");
// largest power of two <= STAGE: the biggest hash table the stage holds
constexpr int STAGE_POW2 = STAGE >= 2048 ? 2048 : STAGE >= 1024 ? 1024 : STAGE >= 512 ? 512 : 256;
static_assert(STAGE_POW2 <= STAGE && STAGE >= 256, "stage too small");
constexpr int MIN_STAGE = 8;
// lists at least this long are staged through one bulk copy (TMA)
constexpr int BULK_STAGE_MIN = 64;
constexpr int ST_NONE = 0, ST_SORTED = 1, ST_HASH = 2, ST_BITMAP = 3, ST_FILTER = 4;
// ST_FILTER: an open-addressed table of up to FILTER_SLOTS slots in the upper
// half of the stage, with a bit filter over a second hash of the keys in the
// lower half. A probe reads one filter word and looks in the table only when
// its bit is set: for a key not in the list that happens with probability at
// most blen / FILTER_BITS (below 1/64 for blen <= 512).
constexpr int FILTER_WORDS = STAGE / 2;
constexpr int FILTER_BITS_LOG2 = 15;
constexpr int FILTER_SLOTS = STAGE - FILTER_WORDS;
static_assert(FILTER_WORDS * 32 == 1 << FILTER_BITS_LOG2, "filter size");
static_assert((FILTER_SLOTS & (FILTER_SLOTS - 1)) == 0 && FILTER_WORDS % 4 == 0, "filter table");
constexpr int32_t EMPTY = -1;

__device__ __forceinline__ uint32_t hash_slot(int32_t w, int log2h) {
  return ((uint32_t)w * 2654435761u) >> (32 - log2h);
}

__device__ __forceinline__ uint32_t filter_bit(int32_t w) {
  return ((uint32_t)w * 0x85EBCA6Bu) >> (32 - FILTER_BITS_LOG2);
}

// Membership of w in the sorted list stage[0, len): lower bound by a fixed
// number of halvings (the same for every lane, since len is warp-uniform).
__device__ __forceinline__ bool sorted_contains(const int32_t *stage, int len, int32_t w) {
  int pos = 0;
  for (int step = len > 0 ? 1 << (31 - __clz(len)) : 0; step > 0; step >>= 1)
    if (pos + step <= len && stage[pos + step - 1] < w) pos += step;
  return pos < len && stage[pos] == w;
}

// Membership of w in the open-addressed table stage[0, 2^log2h) (linear
// probing, at most half full). The probe reads four slots per 16-byte load,
// starting at the 4-slot group of w's hash slot, so nearly every lookup ends
// after one load and the lanes of a warp stay together.
__device__ __forceinline__ bool hash_contains(const int32_t *stage, int log2h, int32_t w) {
  const uint32_t gmask = (1u << (log2h - 2)) - 1u;
  uint32_t g = hash_slot(w, log2h) >> 2;
  const int4 *groups = reinterpret_cast<const int4 *>(stage);
  for (uint32_t n = 0; n <= gmask; ++n) {
    const int4 q = groups[g];
    if (q.x == w || q.y == w || q.z == w || q.w == w) return true;
    if (q.x == EMPTY || q.y == EMPTY || q.z == EMPTY || q.w == EMPTY) return false;
    g = (g + 1) & gmask;
  }
  return false;
}

// The table half of an ST_FILTER stage, reached only when the filter bit is set.
__device__ __forceinline__ bool filter_verify(const int32_t *table, int log2h, int32_t w) {
  return hash_contains(table, log2h, w);
}

__device__ __forceinline__ uint32_t filter_lookup(const int32_t *stage, int log2h, int32_t w) {
  const uint32_t h = filter_bit(w);
  const uint32_t word = reinterpret_cast<const uint32_t *>(stage)[h >> 5];
  if (((word >> (h & 31u)) & 1u) == 0u) return 0u;
  return filter_verify(stage + FILTER_WORDS, log2h, w) ? 1u : 0u;
}

// ------------------------------------------------ bulk copies (TMA, PTX)

__device__ __forceinline__ uint32_t smem_addr(const void *ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(unsigned long long *m) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(m)) : "memory");
}
// Makes an initialised barrier visible to the bulk-copy unit.
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// The one arrival of the barrier's current phase, announcing `bytes` of copies.
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *m, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(m)), "r"(parity)
      : "memory");
  return done != 0;
}
// limit of one wait on a bulk copy (copies of valid addresses take microseconds)
constexpr uint64_t COPY_WAIT_NS = 200ull * 1000 * 1000;
// Waits for the barrier's phase of the given parity, for at most COPY_WAIT_NS.
__device__ __noinline__ bool mbar_wait_bounded(unsigned long long *m, uint32_t parity) {
  if (mbar_try_wait(m, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(m, parity))
    if (global_ns() - t0 > COPY_WAIT_NS) return false;
  return true;
}
// TMA bulk copy global -> shared of `bytes` (a multiple of 16, both addresses
// 16-byte aligned), completing on barrier m.
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes,
                                          unsigned long long *m) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(m))
      : "memory");
}
// Orders this thread's earlier plain shared-memory accesses before later bulk
// copies into the same memory.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Starts one bulk copy of list[e0, e1) into `dst` (e0, e1 multiples of 4:
// whole 16-byte quads of a 16-byte aligned, quad-padded column array; dst
// 16-byte aligned), issued by lane 0 on barrier mbar. Warp-uniform call.
__device__ __forceinline__ void bulk_issue(int32_t *dst, const int32_t *list, int64_t e0,
                                           int64_t e1, unsigned long long *mbar, unsigned lane) {
  fence_proxy_async();  // earlier plain accesses to the stage before the copy
  __syncwarp();
  if (lane == 0) {
    const uint32_t bytes = (uint32_t)(4 * (e1 - e0));
    mbar_expect_tx(mbar, bytes);
    bulk_copy(dst, list + e0, bytes, mbar);
  }
}

// Waits (bounded) for the copy of bulk_issue; true on every lane when it
// arrived. On false the copy is awaited once more and the caller stops.
__device__ __forceinline__ bool bulk_wait(unsigned long long *mbar, uint32_t &parity) {
  const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(mbar, parity));
  if (!ok) {
    mbar_wait_bounded(mbar, parity);
    return false;
  }
  parity ^= 1u;
  return true;
}

// Per-batch lane records, shared by the warp: where each in-edge's probes
// start in the flattened probe sequence and where they come from.
struct LaneRec {
  int64_t b0[32];     // N(G_jk, v) range of each lane (mixed batches only)
  int64_t b1[32];
  uint32_t s0[32];    // first probe element (local column index) of each lane's in-edge
  uint32_t s1[32];    // one past its last probe element (quad probes only)
  uint32_t incl[32];  // inclusive prefix of the probe counts (quad counts for quad probes)
  int32_t u[32];
  int32_t v[32];
  unsigned long long mbar;  // completion of bulk copies into the warp's stage
};

// Runs the flattened probes of one batch: probe q (0 <= q < total) belongs to
// the lane-record o whose inclusive prefix first exceeds q and reads column
// rec.s0[o] + q - (prefix before o). Lane l takes q = l, l + 32, ...; U probes
// per lane per round have their loads issued before any lookup, so each lane
// keeps U global loads in flight (4 suits the one-load lookups; the halving
// searches, which keep more registers live, take 3). Column indices are local
// to the block arrays and below 2^32.
template <int U, typename OnHit, typename Lookup>
__device__ __forceinline__ void probe_batch(const int32_t *__restrict__ ci_ik, const LaneRec &rec,
                                            uint32_t total, unsigned lane, OnHit &on_hit,
                                            Lookup lookup) {
  int o = 0;
  uint32_t o_end = rec.incl[0];
  uint32_t addr = rec.s0[0];  // column of probe q is addr + q (mod 2^32)
  uint32_t qb = lane;
  // full rounds: every lane's U probes exist (the test is warp-uniform)
  for (; qb - lane + 32u * U <= total; qb += 32u * U) {
    int32_t wv[U];
    int own[U];
    uint32_t qpos[U];
#pragma unroll
    for (int r = 0; r < U; ++r) {
      const uint32_t q = qb + 32u * r;
      while (q >= o_end) {
        ++o;
        const uint32_t prev_end = o_end;
        o_end = rec.incl[o];
        addr = rec.s0[o] - prev_end;
      }
      qpos[r] = addr + q;
      wv[r] = ci_ik[qpos[r]];
      own[r] = o;
    }
#pragma unroll
    for (int r = 0; r < U; ++r)
      if (lookup(wv[r], own[r])) on_hit(wv[r], own[r], qpos[r]);
  }
  // the last, partial round
  if (qb - lane < total) {
    int32_t wv[U];
    int own[U];
    uint32_t qpos[U];
#pragma unroll
    for (int r = 0; r < U; ++r) {
      const uint32_t q = qb + 32u * r;
      own[r] = -1;
      if (q < total) {
        while (q >= o_end) {
          ++o;
          const uint32_t prev_end = o_end;
          o_end = rec.incl[o];
          addr = rec.s0[o] - prev_end;
        }
        qpos[r] = addr + q;
        wv[r] = ci_ik[qpos[r]];
        own[r] = o;
      }
    }
#pragma unroll
    for (int r = 0; r < U; ++r)
      if (own[r] >= 0 && lookup(wv[r], own[r])) on_hit(wv[r], own[r], qpos[r]);
  }
}

// Quad probes (plain counts against a bitmap-staged list): the probe range
// [s0, s1) of each in-edge is widened down to a multiple of four, cut into
// aligned groups of four columns ("quads"), and the quads of the batch are
// flattened like single probes: lane l takes quads l, l + 32, ... and loads
// each with one 16-byte load. A 4-bit mask per quad keeps the columns inside
// [s0, s1). Column arrays are 16-byte aligned and padded by whole quads, so
// the widened reads stay inside them. UQ quads per lane are in flight.
__device__ __forceinline__ uint32_t quad_mask(uint32_t q, uint32_t lo, uint32_t hi) {
  // columns q + c, 0 <= c < 4, with lo <= q + c < hi (q <= hi - 1, q >= lo - 3)
  const uint32_t first = lo > q ? lo - q : 0u;
  const uint32_t last = hi - q < 4u ? hi - q : 4u;
  return ((1u << last) - 1u) & ~((1u << first) - 1u);
}

template <int UQ, typename Lookup>
__device__ __forceinline__ uint32_t probe_quads(const int32_t *__restrict__ ci,
                                                const LaneRec &rec, uint32_t totalq,
                                                unsigned lane, Lookup lookup) {
  uint32_t hits = 0;
  int o = 0;
  uint32_t o_end = rec.incl[0];
  uint32_t lo = rec.s0[0], hi = rec.s1[0];
  uint32_t base = lo & ~3u;  // column of quad j is base + 4 * j (mod 2^32)
  uint32_t jb = lane;
  for (; jb - lane < totalq; jb += 32u * UQ) {
    int4 wq[UQ];
    uint32_t msk[UQ];
#pragma unroll
    for (int r = 0; r < UQ; ++r) {
      const uint32_t j = jb + 32u * r;
      msk[r] = 0u;
      wq[r] = make_int4(0, 0, 0, 0);
      if (j < totalq) {
        while (j >= o_end) {
          ++o;
          const uint32_t prev_end = o_end;
          o_end = rec.incl[o];
          lo = rec.s0[o];
          hi = rec.s1[o];
          base = (lo & ~3u) - 4u * prev_end;
        }
        const uint32_t q = base + 4u * j;
        wq[r] = *reinterpret_cast<const int4 *>(ci + q);
        msk[r] = quad_mask(q, lo, hi);
      }
    }
#pragma unroll
    for (int r = 0; r < UQ; ++r) {
      hits += lookup(wq[r].x) & msk[r];
      hits += lookup(wq[r].y) & (msk[r] >> 1);
      hits += lookup(wq[r].z) & (msk[r] >> 2);
      hits += lookup(wq[r].w) & (msk[r] >> 3);
    }
  }
  return hits;
}

constexpr int UNIFORM_MIN = 4;  // a run of >= 4 in-edges into one v is a uniform batch

template <int MODE>
__global__ void __launch_bounds__(CT_NT, 3) k_count(CountParams P) {
  constexpr bool PER_VERTEX = (MODE & MODE_VERTEX) != 0;
  constexpr bool PER_GRAPH = (MODE & MODE_GRAPH) != 0;
  constexpr bool PER_EDGE = (MODE & MODE_EDGE) != 0;
  extern __shared__ __align__(16) unsigned char count_smem_raw[];
  const unsigned lane = threadIdx.x & 31u;
  const int warp = threadIdx.x >> 5;
  int32_t *stage = reinterpret_cast<int32_t *>(count_smem_raw) + warp * (STAGE + 4);
  LaneRec &rec = reinterpret_cast<LaneRec *>(count_smem_raw + (size_t)(CT_NT / 32) * (STAGE + 4) *
                                                                  sizeof(int32_t))[warp];
  if (lane == 0) {
    stage[STAGE] = 0;  // zero guard word after the stage
    mbar_init(&rec.mbar);
    mbar_init_fence();
  }
  __syncwarp();
  uint32_t mbar_parity = 0;  // parity of rec.mbar's next phase
  const uint64_t t_start = P.timeout_ns ? global_ns() : 0;
  // (task, v) whose N(G_jk, v) is in `stage`, and how it is stored
  unsigned long long staged_tag = ~0ull;
  int staged_len = 0, staged_log2h = 0, staged_mode = ST_NONE, staged_off = 0;
  int32_t staged_first = 0;
  uint32_t staged_gw = STAGE;  // bitmap: index of its zero guard word
  bool failed = false;

  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(P.head, 1ull);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= (unsigned long long)P.nitems) break;
    if (P.timeout_ns && global_ns() - t_start > P.timeout_ns) {
      if (lane == 0) atomicExch(P.status, STATUS_TIMEOUT);
      break;
    }
    const WorkItem w = P.items[it];
    const int t = w.task;
    if (P.task_mask && P.task_mask[t] == 0) continue;  // another rank's task
    const long long t_item = P.task_cycles ? clock64() : 0;
    const int kflag = w.flags & 3;  // 0 INTERSECT, 1 HASHMAP, 2 AUTO (per list)
    const int hash_min = w.flags >> 2;  // AUTO: longer lists hash, shorter ones sorted
    const TaskDesc &d = P.desc[t];
    // block arrays are indexed locally: in-edge x at [x - ie_off], column
    // position q at [q - ci_*_off] (the offsets are 0 when the plan is resident)
    const InEdge *__restrict__ ie = d.ie;
    const int64_t ie_off = d.ie_off;
    const uint32_t *__restrict__ rp_ik = d.rp_ik;
    const uint32_t *__restrict__ rp_jk = d.rp_jk;
    const int32_t *__restrict__ ci_ik = d.ci_ik;
    const int32_t *__restrict__ ci_jk = d.ci_jk;
    const int64_t ik_off = d.ci_ik_off, jk_off = d.ci_jk_off;
    const int64_t rs_ik = d.rs_ik, rs_jk = d.rs_jk;
    const int32_t c_i = d.c_i, c_j = d.c_j;
    const bool diag = d.diag != 0;
    unsigned long long acc = 0;

    int64_t base = w.x0;
    // the records (u, v, e, f) of the current window of 32 in-edges; lanes past
    // the item hold v = -1
    InEdge r = base + lane < w.x1 ? ie[base + lane - ie_off] : make_int4(0, -1, 0, 0);
    while (base < w.x1) {
      const int64_t batch_x0 = base;  // in-edge of lane 0; lane l's is batch_x0 + l
      const int32_t v = r.y;
      const bool valid = v >= 0;
      // in-edges are sorted by destination: lanes equal to lane 0's v form a prefix
      const int32_t v0 = __shfl_sync(0xffffffffu, v, 0);
      const unsigned eq = __ballot_sync(0xffffffffu, valid && v == v0);
      const unsigned vmask = __ballot_sync(0xffffffffu, valid);
      const int run0 = __popc(eq);
      const int nvalid = __popc(vmask);
      const bool uniform = run0 >= UNIFORM_MIN || run0 == nvalid;
      int nb;  // in-edges handled by this batch
      if (uniform) {
        nb = run0;
      } else {
        // cut before the last run, which may continue past the batch
        const int32_t vprev = __shfl_up_sync(0xffffffffu, v, 1);
        const unsigned heads = __ballot_sync(0xffffffffu, valid && (lane == 0 || v != vprev));
        const int last_head = 31 - __clz(heads);
        nb = (base + 32 < w.x1 && last_head > 0) ? last_head : nvalid;
      }
      base += nb;
      // the next window's records into registers while this batch runs, and the
      // one after it into L2
      const InEdge rn = base + lane < w.x1 ? ie[base + lane - ie_off] : make_int4(0, -1, 0, 0);
      if (base + 32 + lane < w.x1)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(ie + (base + 32 + lane - ie_off)));
      const bool active = (int)lane < nb;
      const int32_t u = r.x;
      const int64_t e = (int64_t)(uint32_t)r.z;
      const int64_t f = (int64_t)(uint32_t)r.w;
      r = rn;
      // N(G_jk, v): direct row pointers of block (j, k); [b0, b1) local to ci_jk
      int64_t b0 = 0, b1 = 0;
      if (uniform) {
        if (lane == 0) {
          b0 = (int64_t)rp_jk[(v0 - c_j) * rs_jk] - jk_off;
          b1 = (int64_t)rp_jk[(v0 - c_j) * rs_jk + 1] - jk_off;
        }
        b0 = __shfl_sync(0xffffffffu, b0, 0);
        b1 = __shfl_sync(0xffffffffu, b1, 0);
      } else if (active) {
        b0 = (int64_t)rp_jk[(v - c_j) * rs_jk] - jk_off;
        b1 = (int64_t)rp_jk[(v - c_j) * rs_jk + 1] - jk_off;
      }
      // N(G_ik, u) restricted to entries above v: for k == j the entries of u's
      // run in G_ij after (u, v) itself, [e + 1, f) from the record; else u's
      // run in G_ik from the split table. [s0, s1) local to ci_ik
      int64_t s0 = 0, s1 = 0;
      if (active && b1 > b0) {
        if (diag) {
          s0 = e + 1 - ik_off;
          s1 = f - ik_off;
        } else {
          s0 = (int64_t)rp_ik[(u - c_i) * rs_ik] - ik_off;
          s1 = (int64_t)rp_ik[(u - c_i) * rs_ik + 1] - ik_off;
        }
      }
      const uint32_t len = (uint32_t)(s1 - s0);
      const uint32_t total = __reduce_add_sync(0xffffffffu, len);
      if (total == 0) continue;

      // stage N(G_jk, v) once per (task, v) in one of three forms:
      //  - bitmap over [first, last] of the list (Alg. 6's direct-address
      //    table H, windowed to the list's value range) when that range has at
      //    most STAGE * 32 values;
      //  - open-addressed hash table (at most half full) otherwise;
      //  - sorted copy (bbTC-Intersect, Alg. 5), searched by halving.
      // The item's kernel flag picks sorted (INTERSECT), bitmap-else-hash
      // (HASHMAP), or, per list, bitmap, then hash for long lists, then sorted
      // (AUTO).
      const int blen = (int)(b1 - b0);
      bool staged = false;
      if (uniform && blen >= MIN_STAGE) {
        const unsigned long long tag =
            ((unsigned long long)(uint32_t)t << 33) | ((unsigned long long)(uint32_t)v0 << 2);
        if (tag == staged_tag) {
          staged = true;
        } else if (nb == 32 || total >= (uint32_t)blen / 2) {
          // the list's first 32 entries, one per lane, and its last entry, in
          // one round of loads: the value range comes from them
          const int32_t x0 = (int)lane < blen ? ci_jk[b0 + lane] : 0;
          int32_t lastv = 0;
          if (lane == 0 && blen > 32) lastv = ci_jk[b1 - 1];
          const int32_t first = __shfl_sync(0xffffffffu, x0, 0);
          const int32_t last = blen > 32 ? __shfl_sync(0xffffffffu, lastv, 0)
                                         : __shfl_sync(0xffffffffu, x0, blen - 1);
          const int64_t span = (int64_t)last - first + 1;
          int mode = ST_NONE;
          if (kflag == 0) {
            if (blen <= STAGE) mode = ST_SORTED;
          } else if (span <= (int64_t)STAGE * 32) {
            mode = ST_BITMAP;
          } else if (2 * blen <= FILTER_SLOTS && (kflag == 1 || blen > hash_min)) {
            mode = ST_FILTER;
          } else if (2 * blen <= STAGE_POW2 && (kflag == 1 || blen > hash_min)) {
            mode = ST_HASH;
          } else if (kflag == 2 && blen <= STAGE) {
            mode = ST_SORTED;
          }
          if (mode != ST_NONE) {
            __syncwarp();
            // A list of at least BULK_STAGE_MIN entries arrives by one bulk
            // copy (TMA) of its aligned 16-byte span: a sorted copy straight
            // into the stage, for the tables into the free words beside them,
            // from which the table is then built. Shorter lists, and lists
            // with no room beside their table, are read with plain loads.
            const int64_t e0 = b0 & ~int64_t(3), e1 = (b1 + 3) & ~int64_t(3);
            const bool long_list = blen >= BULK_STAGE_MIN;
            const int32_t *src = ci_jk + b0;  // where the table build reads the list
            if (mode == ST_BITMAP) {
              // words [0, nw) hold the window, word nw is its zero guard; only
              // these are cleared (4-word groups up to `land`)
              const uint32_t nw = (uint32_t)((span + 31) >> 5);
              const int64_t land = (int64_t)((nw + 4u) & ~3u);
              const bool bulk = long_list && land + (e1 - e0) <= STAGE;
              if (bulk) bulk_issue(stage + land, ci_jk, e0, e1, &rec.mbar, lane);
              int4 *s4 = reinterpret_cast<int4 *>(stage);
              for (int i = lane; i < (int)(land >> 2); i += 32) s4[i] = make_int4(0, 0, 0, 0);
              if (bulk) {
                failed = !bulk_wait(&rec.mbar, mbar_parity);
                src = stage + land + (b0 - e0);
              }
              __syncwarp();
              if (!failed)
                for (int i = lane; i < blen; i += 32) {
                  const uint32_t d = (uint32_t)((i < 32 ? x0 : src[i]) - first);
                  atomicOr(reinterpret_cast<unsigned *>(stage) + (d >> 5), 1u << (d & 31u));
                }
              staged_first = first;
              staged_len = (int)span;
              staged_gw = nw;
            } else if (mode == ST_FILTER || mode == ST_HASH) {
              int log2h = 5;
              while ((1 << log2h) < 2 * blen) ++log2h;
              const int hsize = 1 << log2h;
              const int tab0 = mode == ST_FILTER ? FILTER_WORDS : 0;
              int32_t *table = stage + tab0;
              const int64_t land = tab0 + hsize;
              const bool bulk = long_list && land + (e1 - e0) <= STAGE;
              if (bulk) bulk_issue(stage + land, ci_jk, e0, e1, &rec.mbar, lane);
              if (mode == ST_FILTER) {
                int4 *f4 = reinterpret_cast<int4 *>(stage);
                for (int i = lane; i < FILTER_WORDS / 4; i += 32) f4[i] = make_int4(0, 0, 0, 0);
              }
              for (int i = lane; i < hsize; i += 32) table[i] = EMPTY;
              if (bulk) {
                failed = !bulk_wait(&rec.mbar, mbar_parity);
                src = stage + land + (b0 - e0);
              }
              __syncwarp();
              const uint32_t hmask = (uint32_t)hsize - 1u;
              if (!failed)
                for (int i = lane; i < blen; i += 32) {
                  const int32_t key = i < 32 ? x0 : src[i];
                  if (mode == ST_FILTER) {
                    const uint32_t fb = filter_bit(key);
                    atomicOr(reinterpret_cast<unsigned *>(stage) + (fb >> 5), 1u << (fb & 31u));
                  }
                  // linear probing from the first slot of the key's 4-slot
                  // group, the order in which hash_contains reads the table
                  uint32_t h = hash_slot(key, log2h) & ~3u;
                  for (int n = 0; n < hsize; ++n) {
                    if (atomicCAS(&table[h], EMPTY, key) == EMPTY) break;
                    h = (h + 1) & hmask;
                  }
                }
              staged_log2h = log2h;
              staged_len = blen;
            } else {
              staged_off = 0;
              if (long_list && e1 - e0 <= STAGE) {
                bulk_issue(stage, ci_jk, e0, e1, &rec.mbar, lane);
                failed = !bulk_wait(&rec.mbar, mbar_parity);
                staged_off = (int)(b0 - e0);
              } else {
                for (int i = lane; i < blen; i += 32) stage[i] = i < 32 ? x0 : ci_jk[b0 + i];
              }
              staged_len = blen;
            }
            __syncwarp();
            staged_tag = failed ? ~0ull : tag;
            staged_mode = mode;
            staged = !failed;
          }
        }
      }
      if (failed) break;

      if (diag && r.y >= 0) {
        // the start of the next window's probe run, [e + 1, f) of its record,
        // into L2 while this batch is looked up (the rows of the sources of
        // one destination lie anywhere in the column array)
        const uint32_t e_next = (uint32_t)r.z + 1u, f_next = (uint32_t)r.w;
        if (f_next > e_next) {
          const int32_t *q = ci_ik + ((int64_t)e_next - ik_off);
          asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
          if (f_next - e_next > 32u) asm volatile("prefetch.global.L2 [%0];" ::"l"(q + 32));
        }
      }

      if (MODE == 0 && staged && (staged_mode == ST_BITMAP || staged_mode == ST_FILTER)) {
        // quad probes (see probe_quads) against a bitmap or a filtered table;
        // plain hash-table and sorted lookups keep the single-probe loop below,
        // which measured faster for them
        const uint32_t a0 = (uint32_t)s0 & ~3u;
        const uint32_t nq = len ? ((uint32_t)s1 - a0 + 3u) >> 2 : 0u;
        const uint32_t inclq = warp_inclusive_scan(nq);
        const uint32_t totalq = __shfl_sync(0xffffffffu, inclq, 31);
        rec.s0[lane] = (uint32_t)s0;
        rec.s1[lane] = (uint32_t)s1;
        rec.incl[lane] = inclq;
        __syncwarp();
        if (staged_mode == ST_BITMAP) {
          const unsigned *__restrict__ bm = reinterpret_cast<const unsigned *>(stage);
          const int32_t first = staged_first;
          const uint32_t gw = staged_gw;
          acc += probe_quads<2>(ci_ik, rec, totalq, lane, [&](int32_t w) -> uint32_t {
            const uint32_t dlt = (uint32_t)(w - first);
            // values outside the window [first, first + 32 * gw) read the zero
            // guard word gw
            const uint32_t word = bm[min(dlt >> 5, gw)];
            return (word >> (dlt & 31u)) & 1u;
          });
        } else {
          const int log2h = staged_log2h;
          acc += probe_quads<2>(ci_ik, rec, totalq, lane, [&](int32_t w) -> uint32_t {
            return filter_lookup(stage, log2h, w);
          });
        }
        __syncwarp();
        continue;
      }

      // flattened probes, interleaved over the lanes (lanes that share an
      // in-edge read consecutive elements); each lane's owner only moves
      // forward, at most 31 steps per batch
      const uint32_t incl = warp_inclusive_scan(len);
      rec.s0[lane] = (uint32_t)s0;
      rec.incl[lane] = incl;
      if (!uniform) {
        rec.b0[lane] = b0;
        rec.b1[lane] = b1;
      }
      if (PER_VERTEX || PER_GRAPH) {
        rec.u[lane] = u;
        rec.v[lane] = uniform ? v0 : v;
      }
      __syncwarp();
      uint32_t hits = 0;
      unsigned long long batch_hits = 0;  // one graph per uniform batch
      auto on_hit = [&](int32_t wv, int o, uint32_t qpos) {
        ++hits;
        if (PER_VERTEX) {
          atomicAdd(&P.vcount[rec.u[o]], 1ull);
          atomicAdd(&P.vcount[rec.v[o]], 1ull);
          atomicAdd(&P.vcount[wv], 1ull);
        }
        if (PER_EDGE) {
          // the triangle's three edges, by position in the block columns:
          // (u,v) from the in-edge record, (u,w) from the probe, (v,w) found
          // in N(G_jk, v)
          const int64_t lo = uniform ? b0 : rec.b0[o];
          const int64_t hi = uniform ? b1 : rec.b1[o];
          const int64_t pvw = lower_bound_dev<int32_t, int64_t>(ci_jk, lo, hi, wv);
          atomicAdd(&P.edge_sup[(uint32_t)ie[batch_x0 + o - ie_off].z], 1u);
          atomicAdd(&P.edge_sup[(int64_t)qpos + ik_off], 1u);
          atomicAdd(&P.edge_sup[pvw + jk_off], 1u);
        }
        if (PER_GRAPH) {
          // every in-edge into v comes from v's own graph
          if (uniform) ++batch_hits;
          else atomicAdd(&P.graph_count[P.gid[rec.v[o]]], 1ull);
        }
      };
      // the probe loop, specialised by how N(G_jk, v) is looked up
      if (staged && staged_mode == ST_BITMAP) {
        const unsigned *__restrict__ bm = reinterpret_cast<const unsigned *>(stage);
        const int32_t first = staged_first;
        const uint32_t span = (uint32_t)staged_len;
        probe_batch<4>(ci_ik, rec, total, lane, on_hit, [&](int32_t w, int) {
          // branch-free: the word index is clamped into the bitmap, and the
          // range test masks the bit
          const uint32_t dlt = (uint32_t)(w - first);
          const uint32_t word = bm[min(dlt >> 5, (uint32_t)(STAGE - 1))];
          return ((dlt < span) & (word >> (dlt & 31u))) & 1u;
        });
      } else if (staged && staged_mode == ST_FILTER) {
        const int log2h = staged_log2h;
        probe_batch<4>(ci_ik, rec, total, lane, on_hit,
                       [&](int32_t w, int) { return filter_lookup(stage, log2h, w) != 0u; });
      } else if (staged && staged_mode == ST_HASH) {
        const int log2h = staged_log2h;
        probe_batch<4>(ci_ik, rec, total, lane, on_hit,
                       [&](int32_t w, int) { return hash_contains(stage, log2h, w); });
      } else if (staged) {
        const int slen = staged_len;
        const int32_t *sl = stage + staged_off;
        probe_batch<3>(ci_ik, rec, total, lane, on_hit,
                       [&](int32_t w, int) { return sorted_contains(sl, slen, w); });
      } else {
        probe_batch<3>(ci_ik, rec, total, lane, on_hit, [&](int32_t w, int o) {
          const int64_t lo = uniform ? b0 : rec.b0[o];
          const int64_t hi = uniform ? b1 : rec.b1[o];
          const int64_t pos = lower_bound_dev<int32_t, int64_t>(ci_jk, lo, hi, w);
          return pos < hi && ci_jk[pos] == w;
        });
      }
      acc += hits;
      if (PER_GRAPH && uniform) {
        batch_hits = warp_sum(batch_hits);
        if (lane == 0 && batch_hits) atomicAdd(&P.graph_count[P.gid[v0]], batch_hits);
      }
      __syncwarp();
    }
    acc = warp_sum(acc);
    if (lane == 0 && acc) atomicAdd(&P.task_count[t], acc);
    if (P.task_cycles && lane == 0)
      atomicAdd(&P.task_cycles[t], (unsigned long long)(clock64() - t_item));
    if (failed) break;
  }
  if (failed && lane == 0) atomicExch(P.status, STATUS_COPY_WAIT);
}

__global__ void k_sum_u64(const unsigned long long *__restrict__ in, int64_t count,
                          unsigned long long *__restrict__ out) {
  unsigned long long s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    s += in[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

__global__ void k_wedges(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                         const int32_t *__restrict__ esrc, int64_t m, int64_t n,
                         unsigned long long *__restrict__ sums) {
  unsigned long long win = 0, wout = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const int32_t v = colidx[e];
    win += (unsigned long long)(rowptr[v + 1] - rowptr[v]);
  }
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
    const unsigned long long d = (unsigned long long)(rowptr[u + 1] - rowptr[u]);
    wout += d * (d > 0 ? d - 1 : 0) / 2;
  }
  win = warp_sum(win);
  wout = warp_sum(wout);
  if ((threadIdx.x & 31) == 0) {
    if (win) atomicAdd(&sums[0], win);
    if (wout) atomicAdd(&sums[1], wout);
  }
}

size_t count_smem_bytes() {
  return (size_t)(CT_NT / 32) * ((STAGE + 4) * sizeof(int32_t) + sizeof(LaneRec));
}

template <int MODE>
bbtc_status configure_mode(int *blocks_per_sm) {
  const size_t smem = count_smem_bytes();
  BBTC_CUDA(cudaFuncSetAttribute(k_count<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  BBTC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_count<MODE>, CT_NT,
                                                          smem));
  if (*blocks_per_sm < 1) *blocks_per_sm = 1;
  return BBTC_OK;
}

}  // namespace

bbtc_status configure_count_kernels(Plan *pl) {
  // the attributes and occupancies are per device: set and query them once
  static std::mutex mu;
  static int cached[64][8];
  static bool done[64] = {false};
  int dev = 0;
  BBTC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range", dev);
    return BBTC_EINVAL;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!done[dev]) {
    BBTC_TRY(configure_mode<0>(&cached[dev][0]));
    BBTC_TRY(configure_mode<1>(&cached[dev][1]));
    BBTC_TRY(configure_mode<2>(&cached[dev][2]));
    BBTC_TRY(configure_mode<3>(&cached[dev][3]));
    BBTC_TRY(configure_mode<4>(&cached[dev][4]));
    BBTC_TRY(configure_mode<5>(&cached[dev][5]));
    BBTC_TRY(configure_mode<6>(&cached[dev][6]));
    BBTC_TRY(configure_mode<7>(&cached[dev][7]));
    done[dev] = true;
  }
  for (int i = 0; i < 8; ++i) pl->blocks_per_sm[i] = cached[dev][i];
  return BBTC_OK;
}

bbtc_status wedge_sums(const bbtc_graph *g, uint64_t *in_sum, uint64_t *out_sum,
                       cudaStream_t s) {
  Scratch scratch(s);
  unsigned long long *sums = nullptr;
  BBTC_TRY(scratch.get(&sums, 2));
  BBTC_CUDA(cudaMemsetAsync(sums, 0, 2 * sizeof(unsigned long long), s));
  const int64_t work = g->m > g->n ? g->m : g->n;
  if (work > 0) {
    k_wedges<<<grid_for(work, 256, 16), 256, 0, s>>>(g->rowptr, g->colidx, g->esrc, g->m, g->n,
                                                     sums);
    BBTC_LAUNCH_CHECK();
  }
  unsigned long long h[2] = {0, 0};
  BBTC_CUDA(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s));
  BBTC_CUDA(cudaStreamSynchronize(s));
  *in_sum = h[0];
  *out_sum = h[1];
  return BBTC_OK;
}

bbtc_status count_reset(bbtc_graph *g, const Plan &pl, unsigned long long *vertex_count,
                        bool per_graph, cudaStream_t s) {
  const int ng = per_graph ? g->ng : 0;
  BBTC_CUDA(cudaMemsetAsync(pl.scratch, 0,
                            sizeof(unsigned long long) * (size_t)(SCR_TASKS + pl.ntasks + ng), s));
  if (vertex_count)
    BBTC_CUDA(cudaMemsetAsync(vertex_count, 0,
                              sizeof(unsigned long long) * (size_t)(g->n > 0 ? g->n : 1), s));
  return BBTC_OK;
}

bbtc_status count_launch(bbtc_graph *g, const Plan &pl, int64_t item0, int64_t nitems,
                         unsigned long long *vertex_count, bool per_graph, uint32_t timeout_ms,
                         cudaStream_t s, unsigned long long *task_cycles, unsigned *edge_sup,
                         const uint8_t *task_mask) {
  if (nitems <= 0) return BBTC_OK;
  unsigned long long *scr = pl.scratch;
  BBTC_CUDA(cudaMemsetAsync(scr + SCR_HEAD, 0, sizeof(unsigned long long), s));
  CountParams P;
  P.desc = pl.desc;
  P.items = pl.items + item0;
  P.nitems = nitems;
  P.head = scr + SCR_HEAD;
  P.task_count = scr + SCR_TASKS;
  P.vcount = vertex_count;
  P.gid = g->gid;
  P.graph_count = scr + SCR_TASKS + pl.ntasks;
  P.status = reinterpret_cast<int32_t *>(scr + SCR_STATUS);
  P.timeout_ns = (uint64_t)timeout_ms * 1000000ull;
  P.task_cycles = task_cycles;
  P.edge_sup = edge_sup;
  P.task_mask = task_mask;
  const int mode = (vertex_count ? MODE_VERTEX : 0) | (per_graph ? MODE_GRAPH : 0) |
                   (edge_sup ? MODE_EDGE : 0);
  int64_t blocks = (int64_t)num_sms() * pl.blocks_per_sm[mode];
  const int64_t need = (nitems + CT_NT / 32 - 1) / (CT_NT / 32);
  if (blocks > need) blocks = need;
  const size_t smem = count_smem_bytes();
  switch (mode) {
    case 0: k_count<0><<<(unsigned)blocks, CT_NT, smem, s>>>(P); break;
    case 1: k_count<1><<<(unsigned)blocks, CT_NT, smem, s>>>(P); break;
    case 2: k_count<2><<<(unsigned)blocks, CT_NT, smem, s>>>(P); break;
    case 3: k_count<3><<<(unsigned)blocks, CT_NT, smem, s>>>(P); break;
    case 4: k_count<4><<<(unsigned)blocks, CT_NT, smem, s>>>(P); break;
    case 5: k_count<5><<<(unsigned)blocks, CT_NT, smem, s>>>(P); break;
    case 6: k_count<6><<<(unsigned)blocks, CT_NT, smem, s>>>(P); break;
    default: k_count<7><<<(unsigned)blocks, CT_NT, smem, s>>>(P); break;
  }
  BBTC_LAUNCH_CHECK();
  return BBTC_OK;
}

bbtc_status count_status_error(const char *where, int32_t status, uint32_t timeout_ms) {
  if (status == STATUS_TIMEOUT) {
    set_error("%s: the counting kernel passed its %u ms limit", where, timeout_ms);
    return BBTC_ETIMEOUT;
  }
  set_error("%s: a bulk copy into the counting kernel's shared memory did not complete within "
            "its wait limit (status %d)", where, (int)status);
  return BBTC_EINTERNAL;
}

bbtc_status count_finish(const Plan &pl, cudaStream_t s) {
  k_sum_u64<<<grid_for(pl.ntasks, 256, 2), 256, 0, s>>>(pl.scratch + SCR_TASKS, pl.ntasks,
                                                         pl.scratch + SCR_TOTAL);
  BBTC_LAUNCH_CHECK();
  return BBTC_OK;
}

bbtc_status run_count(bbtc_graph *g, const Plan &pl, unsigned long long *vertex_count,
                      bool per_graph, uint32_t timeout_ms, cudaStream_t s,
                      cudaEvent_t ev_begin, cudaEvent_t ev_end,
                      unsigned long long *task_cycles, unsigned *edge_sup,
                      const uint8_t *task_mask) {
  BBTC_TRY(count_reset(g, pl, vertex_count, per_graph, s));
  if (ev_begin) BBTC_CUDA(cudaEventRecord(ev_begin, s));
  BBTC_TRY(count_launch(g, pl, 0, pl.nitems, vertex_count, per_graph, timeout_ms, s,
                        task_cycles, edge_sup, task_mask));
  if (ev_end) BBTC_CUDA(cudaEventRecord(ev_end, s));
  return count_finish(pl, s);
}

// --------------------------------------------- several plans, one launch
//
// A batch of resident handles is counted without copying them into a union:
// each handle keeps its own plan, and one persistent launch drains the work
// items of all of them. The descriptors of the handles' tasks are gathered
// into one array (a task is found through its descriptor alone), and each
// handle's items are copied with their task index moved to the handle's
// first slot in that array.

namespace {

struct PlanRef {
  const TaskDesc *desc;
  const WorkItem *items;
  int64_t ntasks, nitems;
  int64_t task_base, item_base;
};

__global__ void k_gather_plans(const PlanRef *__restrict__ refs, int32_t nref,
                               TaskDesc *__restrict__ desc, WorkItem *__restrict__ items) {
  for (int32_t r = blockIdx.x; r < nref; r += gridDim.x) {
    const PlanRef f = refs[r];
    for (int64_t t = threadIdx.x; t < f.ntasks; t += blockDim.x) desc[f.task_base + t] = f.desc[t];
    for (int64_t x = threadIdx.x; x < f.nitems; x += blockDim.x) {
      WorkItem w = f.items[x];
      w.task += (int32_t)f.task_base;
      items[f.item_base + x] = w;
    }
  }
}

}  // namespace

bbtc_status count_plans(bbtc_graph *const *gs, int32_t ng, uint32_t timeout_ms, cudaStream_t s,
                        uint64_t *counts) {
  // largest item lists first, so that small graphs fill the end of the launch
  std::vector<int32_t> order((size_t)ng);
  for (int32_t i = 0; i < ng; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return gs[a]->plan.nitems > gs[b]->plan.nitems;
  });
  std::vector<PlanRef> refs((size_t)ng);
  std::vector<int64_t> task_base((size_t)ng);
  int64_t ntasks = 0, nitems = 0;
  int blocks_per_sm = 0;
  for (int32_t r = 0; r < ng; ++r) {
    const Plan &pl = gs[order[(size_t)r]]->plan;
    if (pl.streamed || pl.p < 1) {
      set_error("internal: count_plans needs resident plans");
      return BBTC_EINTERNAL;
    }
    refs[(size_t)r] = PlanRef{pl.desc, pl.items, pl.ntasks, pl.nitems, ntasks, nitems};
    task_base[(size_t)order[(size_t)r]] = ntasks;
    ntasks += pl.ntasks;
    nitems += pl.nitems;
    if (pl.blocks_per_sm[0] > blocks_per_sm) blocks_per_sm = pl.blocks_per_sm[0];
  }
  if (ntasks > INT32_MAX) {
    set_error("bbtc_count_batch: %lld tasks in one batch exceed the 32-bit task index",
              (long long)ntasks);
    return BBTC_EINVAL;
  }
  Scratch scratch(s);
  PlanRef *d_refs = nullptr;
  TaskDesc *desc = nullptr;
  WorkItem *items = nullptr;
  unsigned long long *counters = nullptr;  // [0] head, [1] status, [2, 2 + T) per task
  BBTC_TRY(scratch.get(&d_refs, ng));
  BBTC_TRY(scratch.get(&desc, ntasks));
  BBTC_TRY(scratch.get(&items, nitems));
  BBTC_TRY(scratch.get(&counters, 2 + ntasks));
  BBTC_CUDA(cudaMemcpyAsync(d_refs, refs.data(), sizeof(PlanRef) * (size_t)ng,
                            cudaMemcpyHostToDevice, s));
  BBTC_CUDA(cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * (size_t)(2 + ntasks), s));
  k_gather_plans<<<(unsigned)std::min<int64_t>(ng, 4096), 256, 0, s>>>(d_refs, ng, desc, items);
  BBTC_LAUNCH_CHECK();
  if (nitems > 0) {
    CountParams P;
    P.desc = desc;
    P.items = items;
    P.nitems = nitems;
    P.head = counters;
    P.task_count = counters + 2;
    P.vcount = nullptr;
    P.gid = nullptr;
    P.graph_count = nullptr;
    P.task_cycles = nullptr;
    P.edge_sup = nullptr;
    P.task_mask = nullptr;
    P.status = reinterpret_cast<int32_t *>(counters + 1);
    P.timeout_ns = (uint64_t)timeout_ms * 1000000ull;
    if (blocks_per_sm < 1) BBTC_TRY(configure_mode<0>(&blocks_per_sm));
    int64_t blocks = (int64_t)num_sms() * blocks_per_sm;
    const int64_t need = (nitems + CT_NT / 32 - 1) / (CT_NT / 32);
    if (blocks > need) blocks = need;
    k_count<0><<<(unsigned)blocks, CT_NT, count_smem_bytes(), s>>>(P);
    BBTC_LAUNCH_CHECK();
  }
  std::vector<unsigned long long> h((size_t)(2 + ntasks));
  BBTC_CUDA(cudaMemcpyAsync(h.data(), counters, sizeof(unsigned long long) * h.size(),
                            cudaMemcpyDeviceToHost, s));
  BBTC_CUDA(cudaStreamSynchronize(s));
  if ((int32_t)h[1] != 0) return count_status_error("bbtc_count_batch", (int32_t)h[1], timeout_ms);
  for (int32_t i = 0; i < ng; ++i) {
    uint64_t c = 0;
    const int64_t b = task_base[(size_t)i];
    for (int64_t t = 0; t < gs[i]->plan.ntasks; ++t) c += h[(size_t)(2 + b + t)];
    counts[i] = c;
  }
  return BBTC_OK;
}

}  // namespace bbtc

// ------------------------------------------------ allocation-free counting
//
// bbtc_count_noalloc runs the same counting kernel as bbtc_count, but keeps its
// scratch (the work-stealing counter, the status word and the per-task
// accumulators) in the fixed device array below instead of allocating it.
// The array is 8 KiB; every GPU that loads the library holds it until exit.

namespace bbtc {
namespace {

constexpr int NOALLOC_MAX_P = 16;                  // p(p+1)(p+2)/6 = 816 tasks
constexpr int NOALLOC_WORDS = 1024;                // 8 KiB of uint64
constexpr int NOALLOC_HEAD = 0, NOALLOC_STATUS = 1, NOALLOC_TASKS = 2;
static_assert(NOALLOC_TASKS + NOALLOC_MAX_P * (NOALLOC_MAX_P + 1) * (NOALLOC_MAX_P + 2) / 6 <=
                  NOALLOC_WORDS,
              "no-alloc scratch too small for NOALLOC_MAX_P");

static __device__ __align__(256) unsigned long long g_noalloc_scratch[NOALLOC_WORDS];

// Device address of g_noalloc_scratch on each device (the host-side symbol is
// only a stand-in and must never be handed to a kernel). Each device's entry
// is looked up once, under a per-device once-flag, so that host threads making
// their first call at the same time do not race on it.
unsigned long long *g_noalloc_addr[64] = {nullptr};
cudaError_t g_noalloc_err[64] = {cudaSuccess};
std::once_flag g_noalloc_once[64];

bbtc_status noalloc_scratch(unsigned long long **out) {
  int dev = 0;
  BBTC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("bbtc_count_noalloc: device ordinal %d out of range", dev);
    return BBTC_EINVAL;
  }
  std::call_once(g_noalloc_once[dev], [dev] {
    void *ptr = nullptr;
    g_noalloc_err[dev] = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (g_noalloc_err[dev] == cudaSuccess) g_noalloc_addr[dev] = static_cast<unsigned long long *>(ptr);
  });
  if (g_noalloc_err[dev] != cudaSuccess) {
    set_error("bbtc_count_noalloc: cudaGetSymbolAddress failed: %s",
              cudaGetErrorString(g_noalloc_err[dev]));
    return BBTC_ECUDA;
  }
  *out = g_noalloc_addr[dev];
  return BBTC_OK;
}

}  // namespace
}  // namespace bbtc

extern "C" bbtc_status bbtc_count_noalloc(bbtc_graph_t g, int32_t p, uint64_t *count_dev,
                                          uint64_t *per_task_dev, void *stream) {
  using namespace bbtc;
  clear_error();
  if (!g || !count_dev) {
    set_error("bbtc_count_noalloc: NULL handle or count_dev");
    return BBTC_EINVAL;
  }
  if (p < 1 || p > NOALLOC_MAX_P) {
    set_error("bbtc_count_noalloc: p = %d is outside 1..%d (fixed scratch holds %d tasks)", p,
              NOALLOC_MAX_P, NOALLOC_WORDS - NOALLOC_TASKS);
    return BBTC_EINVAL;
  }
  const Plan &pl = g->plan;
  if (pl.p != p || pl.streamed) {
    set_error("bbtc_count_noalloc: no plan for p = %d on this handle; call bbtc_count or "
              "bbtc_graph_get_plan with that p first", p);
    return BBTC_EINVAL;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) == cudaSuccess && prev != g->device) cudaSetDevice(g->device);
  else prev = -1;
  cudaStream_t s = stream ? (cudaStream_t)stream : g->stream;
  bbtc_status st = BBTC_OK;
  do {
    unsigned long long *scratch = nullptr;
    if ((st = noalloc_scratch(&scratch)) != BBTC_OK) break;
    unsigned long long *task_count = scratch + NOALLOC_TASKS;
    const int64_t nt = pl.ntasks;
    // the array keeps the previous call's contents: clear what must start at 0
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (size_t)(NOALLOC_TASKS + nt),
                        s) != cudaSuccess ||
        cudaMemsetAsync(count_dev, 0, sizeof(uint64_t), s) != cudaSuccess) {
      set_error("bbtc_count_noalloc: cudaMemsetAsync failed");
      st = BBTC_ECUDA;
      break;
    }
    if (pl.nitems > 0) {
      CountParams P;
      P.desc = pl.desc;
      P.items = pl.items;
      P.nitems = pl.nitems;
      P.head = scratch + NOALLOC_HEAD;
      P.task_count = task_count;
      P.vcount = nullptr;
      P.gid = nullptr;
      P.graph_count = nullptr;
      P.task_cycles = nullptr;
      P.edge_sup = nullptr;
      P.task_mask = nullptr;
      P.status = reinterpret_cast<int32_t *>(scratch + NOALLOC_STATUS);
      P.timeout_ns = 0;
      const size_t smem = count_smem_bytes();
      int blocks_per_sm = 0;
      if (cudaFuncSetAttribute(k_count<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_count<0>, CT_NT,
                                                        smem) != cudaSuccess) {
        set_error("bbtc_count_noalloc: kernel configuration failed");
        st = BBTC_ECUDA;
        break;
      }
      if (blocks_per_sm < 1) blocks_per_sm = 1;
      int64_t blocks = (int64_t)num_sms() * blocks_per_sm;
      const int64_t need = (pl.nitems + CT_NT / 32 - 1) / (CT_NT / 32);
      if (blocks > need) blocks = need;
      k_count<0><<<(unsigned)blocks, CT_NT, smem, s>>>(P);
      if ((st = launch_status("bbtc_count_noalloc")) != BBTC_OK) break;
    }
    k_sum_u64<<<grid_for(nt, 256, 2), 256, 0, s>>>(
        task_count, nt, reinterpret_cast<unsigned long long *>(count_dev));
    if ((st = launch_status("bbtc_count_noalloc")) != BBTC_OK) break;
    if (per_task_dev &&
        cudaMemcpyAsync(per_task_dev, task_count, sizeof(uint64_t) * (size_t)nt,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      set_error("bbtc_count_noalloc: cudaMemcpyAsync failed");
      st = BBTC_ECUDA;
      break;
    }
  } while (0);
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}
