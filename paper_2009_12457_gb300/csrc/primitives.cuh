// primitives.cuh -- device-wide building blocks used by the graph preparation
// and planning steps: stable LSD radix sort of 64-bit keys (optionally with a
// 32-bit payload), exclusive scan, and max reduction.
#pragma once

#include "common.cuh"

namespace bbtc {

// Stable sort of `count` keys by bits [bit_lo, bit_hi) (8-bit digits, one pass
// per digit). keys/alt (and vals/vals_alt when vals != nullptr) are ping-pong
// buffers of `count` elements; *in_alt tells which one holds the result.
bbtc_status radix_sort(uint64_t *keys, uint64_t *alt, uint32_t *vals, uint32_t *vals_alt,
                       int64_t count, int bit_lo, int bit_hi, cudaStream_t s, bool *in_alt);

// out[i] = sum_{j<i} in[i] for i in [0, count); out may alias in.
bbtc_status exclusive_scan_u64(const uint64_t *in, uint64_t *out, int64_t count,
                               cudaStream_t s);

// *out (device) = max(in[0..count)) (0 for count == 0).
bbtc_status reduce_max_i64(const int64_t *in, int64_t count, int64_t *out, cudaStream_t s);
bbtc_status reduce_max_i32(const int32_t *in, int64_t count, int32_t *out, cudaStream_t s);

}  // namespace bbtc
