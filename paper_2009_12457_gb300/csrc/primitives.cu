// primitives.cu -- stable LSD radix sort, exclusive scan, max reduction.
#include "primitives.cuh"

namespace bbtc {

namespace {

constexpr int RS_NT = 256;                 // threads per tile
constexpr int RS_ITEMS = 16;               // keys per thread
constexpr int RS_TILE = RS_NT * RS_ITEMS;  // 4096 keys per tile
constexpr int RS_WARPS = RS_NT / 32;
constexpr int RS_BINS = 256;
constexpr int RS_WARP_SPAN = RS_TILE / RS_WARPS;  // 512 consecutive tile positions per warp

// Per-tile digit counts, digit-major: hist[d * ntiles + tile].
__global__ void __launch_bounds__(RS_NT) k_rs_hist(const uint64_t *__restrict__ keys,
                                                   int64_t count, int shift, uint32_t mask,
                                                   int64_t ntiles, uint64_t *__restrict__ hist) {
  __shared__ uint32_t h[RS_BINS];
  for (int i = threadIdx.x; i < RS_BINS; i += RS_NT) h[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const unsigned lane = threadIdx.x & 31u;
#pragma unroll 4
  for (int i = 0; i < RS_ITEMS; ++i) {
    int64_t idx = base + (int64_t)i * RS_NT + threadIdx.x;
    bool valid = idx < count;
    uint32_t d = valid ? (uint32_t)(keys[idx] >> shift) & mask : RS_BINS;  // RS_BINS = not counted
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (valid && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RS_BINS; d += RS_NT)
    hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// Shared memory layout of the scatter kernel (dynamic).
struct RsSmem {
  uint64_t keys[RS_TILE];
  uint32_t vals[RS_TILE];
  uint32_t whist[RS_WARPS][RS_BINS];  // per-warp digit counts, then per-warp prefixes
  uint32_t bstart[RS_BINS];           // tile-local start of each digit bucket
  uint64_t goff[RS_BINS];             // global start of this tile's part of each bucket
  uint32_t scan_tmp[RS_WARPS + 1];
};

// Stable scatter of one tile. Warp w ranks tile positions [w*512, w*512+512)
// in order, 32 at a time: keys with equal digits in one group of 32 are
// ranked by lane (match_any), groups in order, warps in order -- the tile's
// own order, which is what stability needs.
template <bool HAS_VALS>
__global__ void __launch_bounds__(RS_NT) k_rs_scatter(
    const uint64_t *__restrict__ kin, uint64_t *__restrict__ kout,
    const uint32_t *__restrict__ vin, uint32_t *__restrict__ vout, int64_t count, int shift,
    uint32_t mask, int64_t ntiles, const uint64_t *__restrict__ offsets) {
  extern __shared__ __align__(16) unsigned char rs_smem_raw[];
  RsSmem &sm = *reinterpret_cast<RsSmem *>(rs_smem_raw);
  const int warp = threadIdx.x >> 5;
  const unsigned lane = threadIdx.x & 31u;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_NT) (&sm.whist[0][0])[i] = 0;
  __syncthreads();

  uint64_t k[RS_ITEMS];
  uint32_t v[RS_ITEMS];
  uint32_t rank[RS_ITEMS];
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < RS_ITEMS; ++i) {
    int pos = warp * RS_WARP_SPAN + i * 32 + (int)lane;
    int64_t idx = base + pos;
    bool valid = idx < count;
    // Positions past the end take the largest digit; being last in the tile
    // they rank after every real key, so they never displace one.
    k[i] = valid ? kin[idx] : ~0ull;
    if (HAS_VALS) v[i] = valid ? vin[idx] : 0u;
    uint32_t d = valid ? (uint32_t)(k[i] >> shift) & mask : mask;
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = sm.whist[warp][d];
    __syncwarp();
    if ((peers & lt_mask) == 0) sm.whist[warp][d] = before + (uint32_t)__popc(peers);
    __syncwarp();
    rank[i] = before + (uint32_t)__popc(peers & lt_mask);
  }
  __syncthreads();

  // Per digit: exclusive prefix over warps, and the tile's bucket starts.
  {
    const int d = threadIdx.x;  // RS_NT == RS_BINS
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      uint32_t c = sm.whist[w][d];
      sm.whist[w][d] = run;
      run += c;
    }
    uint32_t total;
    uint32_t start = block_exclusive_scan<uint32_t, RS_NT>(run, sm.scan_tmp, &total);
    sm.bstart[d] = start;
    sm.goff[d] = offsets[(int64_t)d * ntiles + blockIdx.x];
  }
  __syncthreads();

#pragma unroll
  for (int i = 0; i < RS_ITEMS; ++i) {
    uint32_t d = (uint32_t)(k[i] >> shift) & mask;
    uint32_t lpos = sm.bstart[d] + sm.whist[warp][d] + rank[i];
    sm.keys[lpos] = k[i];
    if (HAS_VALS) sm.vals[lpos] = v[i];
  }
  __syncthreads();

  const int64_t nvalid = count - base < RS_TILE ? count - base : RS_TILE;
#pragma unroll 4
  for (int j = 0; j < RS_ITEMS; ++j) {
    int lpos = j * RS_NT + threadIdx.x;
    if (lpos < nvalid) {
      uint64_t key = sm.keys[lpos];
      uint32_t d = (uint32_t)(key >> shift) & mask;
      uint64_t o = sm.goff[d] + (uint64_t)(lpos - (int)sm.bstart[d]);
      kout[o] = key;
      if (HAS_VALS) vout[o] = sm.vals[lpos];
    }
  }
}

constexpr int SC_NT = 512;
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_NT * SC_ITEMS;

__global__ void __launch_bounds__(SC_NT) k_scan_reduce(const uint64_t *__restrict__ in,
                                                       int64_t count,
                                                       uint64_t *__restrict__ partial) {
  __shared__ uint64_t tmp[SC_NT / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * SC_TILE;
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < SC_ITEMS; ++i) {
    int64_t idx = base + (int64_t)i * SC_NT + threadIdx.x;
    if (idx < count) s += in[idx];
  }
  uint64_t total;
  block_exclusive_scan<uint64_t, SC_NT>(s, tmp, &total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SC_NT) k_scan_down(const uint64_t *in, uint64_t *out,
                                                     int64_t count,
                                                     const uint64_t *__restrict__ partial) {
  __shared__ uint64_t tile[SC_TILE];
  __shared__ uint64_t tmp[SC_NT / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * SC_TILE;
#pragma unroll
  for (int i = 0; i < SC_ITEMS; ++i) {
    int64_t idx = base + (int64_t)i * SC_NT + threadIdx.x;
    tile[i * SC_NT + threadIdx.x] = idx < count ? in[idx] : 0;
  }
  __syncthreads();
  uint64_t local[SC_ITEMS];
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < SC_ITEMS; ++i) {
    local[i] = tile[threadIdx.x * SC_ITEMS + i];
    s += local[i];
  }
  uint64_t total;
  uint64_t run = block_exclusive_scan<uint64_t, SC_NT>(s, tmp, &total) +
                 (partial ? partial[blockIdx.x] : 0);
#pragma unroll
  for (int i = 0; i < SC_ITEMS; ++i) {
    tile[threadIdx.x * SC_ITEMS + i] = run;
    run += local[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < SC_ITEMS; ++i) {
    int64_t idx = base + (int64_t)i * SC_NT + threadIdx.x;
    if (idx < count) out[idx] = tile[i * SC_NT + threadIdx.x];
  }
}

template <typename T>
__global__ void k_reduce_max(const T *__restrict__ in, int64_t count,
                             unsigned long long *__restrict__ out) {
  T best = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    best = in[i] > best ? in[i] : best;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    T o = __shfl_xor_sync(0xffffffffu, best, d);
    best = o > best ? o : best;
  }
  if ((threadIdx.x & 31) == 0 && best > 0) atomicMax(out, (unsigned long long)best);
}

bool g_smem_configured[2] = {false, false};

}  // namespace

bbtc_status radix_sort(uint64_t *keys, uint64_t *alt, uint32_t *vals, uint32_t *vals_alt,
                       int64_t count, int bit_lo, int bit_hi, cudaStream_t s, bool *in_alt) {
  *in_alt = false;
  if (count <= 1 || bit_hi <= bit_lo) return BBTC_OK;
  const int64_t ntiles = (count + RS_TILE - 1) / RS_TILE;
  if (ntiles > 0x7fffffffLL) {
    set_error("radix_sort: %lld keys exceed the grid limit", (long long)count);
    return BBTC_EINVAL;
  }
  const bool has_vals = vals != nullptr;
  const size_t smem = sizeof(RsSmem);
  if (!g_smem_configured[has_vals]) {
    if (has_vals)
      BBTC_CUDA(cudaFuncSetAttribute(k_rs_scatter<true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    else
      BBTC_CUDA(cudaFuncSetAttribute(k_rs_scatter<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    g_smem_configured[has_vals] = true;
  }
  Scratch scratch(s);
  uint64_t *hist = nullptr;
  BBTC_TRY(scratch.get(&hist, ntiles * RS_BINS));
  uint64_t *kin = keys, *kout = alt;
  uint32_t *vin = vals, *vout = vals_alt;
  bool flipped = false;
  for (int shift = bit_lo; shift < bit_hi; shift += 8) {
    int bits = bit_hi - shift < 8 ? bit_hi - shift : 8;
    uint32_t mask = (1u << bits) - 1u;
    k_rs_hist<<<(unsigned)ntiles, RS_NT, 0, s>>>(kin, count, shift, mask, ntiles, hist);
    BBTC_LAUNCH_CHECK();
    BBTC_TRY(exclusive_scan_u64(hist, hist, ntiles * RS_BINS, s));
    if (has_vals)
      k_rs_scatter<true><<<(unsigned)ntiles, RS_NT, smem, s>>>(kin, kout, vin, vout, count, shift,
                                                               mask, ntiles, hist);
    else
      k_rs_scatter<false><<<(unsigned)ntiles, RS_NT, smem, s>>>(kin, kout, nullptr, nullptr,
                                                                count, shift, mask, ntiles, hist);
    BBTC_LAUNCH_CHECK();
    uint64_t *tk = kin; kin = kout; kout = tk;
    uint32_t *tv = vin; vin = vout; vout = tv;
    flipped = !flipped;
  }
  *in_alt = flipped;
  return BBTC_OK;
}

bbtc_status exclusive_scan_u64(const uint64_t *in, uint64_t *out, int64_t count,
                               cudaStream_t s) {
  if (count <= 0) return BBTC_OK;
  const int64_t nblocks = (count + SC_TILE - 1) / SC_TILE;
  if (nblocks == 1) {
    k_scan_down<<<1, SC_NT, 0, s>>>(in, out, count, nullptr);
    BBTC_LAUNCH_CHECK();
    return BBTC_OK;
  }
  Scratch scratch(s);
  uint64_t *partial = nullptr;
  BBTC_TRY(scratch.get(&partial, nblocks));
  k_scan_reduce<<<(unsigned)nblocks, SC_NT, 0, s>>>(in, count, partial);
  BBTC_LAUNCH_CHECK();
  BBTC_TRY(exclusive_scan_u64(partial, partial, nblocks, s));
  k_scan_down<<<(unsigned)nblocks, SC_NT, 0, s>>>(in, out, count, partial);
  BBTC_LAUNCH_CHECK();
  return BBTC_OK;
}

bbtc_status reduce_max_i64(const int64_t *in, int64_t count, int64_t *out, cudaStream_t s) {
  BBTC_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
  if (count <= 0) return BBTC_OK;
  k_reduce_max<int64_t><<<grid_for(count, 256, 8), 256, 0, s>>>(
      in, count, reinterpret_cast<unsigned long long *>(out));
  BBTC_LAUNCH_CHECK();
  return BBTC_OK;
}

bbtc_status reduce_max_i32(const int32_t *in, int64_t count, int32_t *out, cudaStream_t s) {
  // accumulate in a 64-bit word; the caller's int32 receives the low half
  unsigned long long *tmp = nullptr;
  Scratch scratch(s);
  BBTC_TRY(scratch.get(&tmp, 1));
  BBTC_CUDA(cudaMemsetAsync(tmp, 0, sizeof(unsigned long long), s));
  if (count > 0) {
    k_reduce_max<int32_t><<<grid_for(count, 256, 8), 256, 0, s>>>(in, count, tmp);
    BBTC_LAUNCH_CHECK();
  }
  BBTC_CUDA(cudaMemcpyAsync(out, tmp, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  return BBTC_OK;
}

}  // namespace bbtc
