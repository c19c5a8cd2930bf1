// common.cuh -- shared internals of the bbTC library: error reporting,
// stream-ordered device allocation, and warp/block scan helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bbtc.h"

namespace bbtc {

// Thread-local error message (bbtc_last_error).
void set_error(const char *fmt, ...);
void clear_error();

#define BBTC_CUDA(call)                                                              \
  do {                                                                               \
    cudaError_t _e = (call);                                                         \
    if (_e != cudaSuccess) {                                                         \
      ::bbtc::set_error("%s: %s (%s:%d)", #call, cudaGetErrorString(_e), __FILE__,   \
                        __LINE__);                                                   \
      return _e == cudaErrorMemoryAllocation ? BBTC_ENOMEM : BBTC_ECUDA;             \
    }                                                                                \
  } while (0)

#define BBTC_TRY(expr)                \
  do {                                \
    bbtc_status _s = (expr);          \
    if (_s != BBTC_OK) return _s;     \
  } while (0)

// Every kernel launch is followed by BBTC_LAUNCH_CHECK (or launch_status),
// which also counts it (bbtc_kernel_launches).
void note_launch();
bbtc_status launch_status(const char *where);

#define BBTC_LAUNCH_CHECK()        \
  do {                             \
    ::bbtc::note_launch();         \
    BBTC_CUDA(cudaGetLastError()); \
  } while (0)

// Stream-ordered device allocation from the device's default memory pool.
// Blocks stay cached in the pool between calls (release threshold raised at
// first use), so repeated create/count calls do not pay cudaMalloc.
// Blocks of 64 MB and more are kept when freed and handed out again for a
// request of a similar size (see api.cu); release_cached_blocks returns the
// idle ones of a device to the pool, cached_block_bytes reports their size.
bbtc_status dalloc(void **p, size_t bytes, cudaStream_t s);
void dfree(void *p, cudaStream_t s);
void release_cached_blocks(int dev, cudaStream_t s);
uint64_t cached_block_bytes(int dev);

template <typename T>
inline bbtc_status dalloc_n(T **p, int64_t count, cudaStream_t s) {
  size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
  return dalloc(reinterpret_cast<void **>(p), bytes, s);
}

// Scoped list of stream-ordered temporaries freed together.
struct Scratch {
  static constexpr int kMax = 32;
  void *ptr[kMax];
  int n = 0;
  cudaStream_t s;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() {
    for (int i = n - 1; i >= 0; --i) dfree(ptr[i], s);
  }
  template <typename T>
  bbtc_status get(T **p, int64_t count) {
    if (n >= kMax) {
      set_error("internal: too many scratch buffers");
      return BBTC_EINTERNAL;
    }
    bbtc_status st = dalloc_n(p, count, s);
    if (st == BBTC_OK) ptr[n++] = *p;
    return st;
  }
};

inline int ceil_log2_u64(uint64_t x) {  // smallest b with 2^b >= x (0 for x <= 1)
  int b = 0;
  while (b < 64 && (1ull << b) < x) ++b;
  return b;
}

inline int num_sms() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    if (cached <= 0) cached = 1;
  }
  return cached;
}

inline unsigned grid_for(int64_t work, int threads, int64_t cap_per_sm = 32) {
  int64_t blocks = (work + threads - 1) / threads;
  int64_t cap = (int64_t)num_sms() * cap_per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (unsigned)blocks;
}

// ------------------------------------------------------------ device helpers

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, d);
    if ((int)lane_id() >= d) x += y;
  }
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
  return x;
}

// Exclusive scan across a block of NT threads (NT a multiple of 32, <= 1024).
// `tmp` must hold NT/32 + 1 elements of shared memory. Returns the exclusive
// prefix; *total receives the block-wide sum.
template <typename T, int NT>
__device__ __forceinline__ T block_exclusive_scan(T x, T *tmp, T *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc = warp_inclusive_scan(x);
  if (lane == 31) tmp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < NT / 32 ? tmp[lane] : T(0);
    T winc = warp_inclusive_scan(w);
    if (lane < NT / 32) tmp[lane] = winc - w;
    if (lane == NT / 32 - 1) tmp[NT / 32] = winc;
  }
  __syncthreads();
  T res = inc - x + tmp[warp];
  *total = tmp[NT / 32];
  __syncthreads();
  return res;
}

// First index in [lo, hi) with a[idx] >= x (a sorted ascending).
template <typename T, typename I>
__device__ __forceinline__ I lower_bound_dev(const T *a, I lo, I hi, T x) {
  while (lo < hi) {
    I mid = lo + ((hi - lo) >> 1);
    if (a[mid] < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Part index of position r given cuts[0..p] (c_0 = 0, c_p = n): the i with
// c_i <= r < c_{i+1}; empty parts own nothing.
__device__ __forceinline__ int part_of_dev(const int32_t *cuts, int p, int32_t r) {
  int lo = 0, hi = p;  // find last i in [0,p) with cuts[i] <= r
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (cuts[mid] <= r)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

}  // namespace bbtc
