// Shared device helpers of the B300 codec: status handling, Morton bit
// spreading, and the integer primitives of Sec. 3.3 (Eq. 13-14).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lpc.h"

namespace lpc {

constexpr int kMaxDepth = 21;
constexpr int kNsym = 255;      // occupancy classes (codes 1..255)
constexpr int kFreqBits = 16;   // cumulative tables sum to 2^16
constexpr int kFreqTotal = 1 << kFreqBits;

// Frame batches: the frame index sits in the top six key bits, above the
// Morton bits (3 L <= 57 for batched frames), so one sort and one set of
// level arrays hold every frame of a batch, frame-major then Morton order.
constexpr int kFrameShift = 58;
constexpr int kMaxBatch = 64;
constexpr uint64_t kLowMask = (1ull << kFrameShift) - 1;

__host__ __device__ __forceinline__ uint64_t parent_key(uint64_t k) {
  return (k & ~kLowMask) | ((k & kLowMask) >> 3);
}
__host__ __device__ __forceinline__ uint64_t child_key(uint64_t k, uint32_t c) {
  return (k & ~kLowMask) | ((k & kLowMask) << 3) | c;
}

// Device error word values (first error wins).
constexpr int kErrCoord = 1;    // coordinate outside [0, 2^L)
constexpr int kErrHashFull = 2; // hash probe limit reached
constexpr int kErrExpand = 3;   // decoded level is not strictly Morton-ordered
constexpr int kErrCapacity = 4; // decoded level exceeds the level arrays
constexpr int kErrStream = 5;   // range-coded substream is corrupt
constexpr int kErrTimeout = 6;  // a bounded wait on the device gave up

__device__ __forceinline__ void set_error(int* err, int code) { atomicCAS(err, 0, code); }

// Spread the low 21 bits of v to every third bit (bit i -> bit 3i).
__host__ __device__ __forceinline__ uint64_t spread3(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

// Inverse of spread3: gather every third bit.
__host__ __device__ __forceinline__ uint32_t compact3(uint64_t v) {
  v &= 0x1249249249249249ull;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
  v = (v ^ (v >> 32)) & 0x1fffffull;
  return (uint32_t)v;
}

// Morton key: x is the most significant bit of every 3-bit group, so the low
// three bits of a key are the child index 4*xbit + 2*ybit + zbit.
__host__ __device__ __forceinline__ uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  return (spread3(x) << 2) | (spread3(y) << 1) | spread3(z);
}

// Eq. 14: clip(round_half_up(acc * m / 2^r) + z, -128, 127), int64 product,
// arithmetic (floor) shift.
__device__ __forceinline__ int requant(int32_t acc, int32_t m, int r, int z) {
  long long p = (long long)acc * (long long)m;
  long long q = ((p + (1ll << (r - 1))) >> r) + z;
  q = q < -128 ? -128 : q;
  q = q > 127 ? 127 : q;
  return (int)q;
}

// The same in the high-word form: with ms = m 2^(32 - r) (exact when r <= 32
// and ms < 2^31), floor((acc m + 2^(r-1)) / 2^r) = floor((acc ms + 2^31) /
// 2^32), so one wide multiply-add with K = 2^31 + z 2^32 and the high word
// give the rounded, offset value (|acc ms| < 2^62: the high word fits int32).
__device__ __forceinline__ int requant_hi(int32_t acc, int32_t ms, int z) {
  const long long p = (long long)acc * ms + ((long long)z * 4294967296ll + 2147483648ll);
  const int q = (int)(p >> 32);
  return min(max(q, -128), 127);
}

// Whether a multiplier m with shift r admits requant_hi, and the scaled form.
__host__ __device__ __forceinline__ bool hi_ok(int32_t m, int r) {
  return r >= 1 && r <= 32 && m >= 0 && ((long long)m << (32 - r)) <= 0x7FFFFFFFll;
}
__host__ __device__ __forceinline__ int32_t hi_scale(int32_t m, int r) {
  return (int32_t)((long long)m << (32 - r));
}

// PReLU on the INT32 accumulator with a Q15 slope, round half up.
__device__ __forceinline__ int32_t prelu(int32_t acc, int a) {
  if (acc >= 0) return acc;
  return (int32_t)(((long long)acc * a + (1 << 14)) >> 15);
}

}  // namespace lpc
