// Decoding of the coarse levels (depths below b) on the device.  Each level
// is coded in chunks of a few hundred nodes, each chunk a range-coded
// substream with its own adaptive symbol-frequency model (the supplement's
// coarse-level coding by symbol frequencies): 255 counts that start at 1,
// the coded symbol's count grows by 32, every count is halved (rounding up)
// once the total exceeds 2^16.  Chunks are independent, so one warp decodes
// one chunk and every chunk of every frame runs in one launch.
//
// A warp holds the model in registers, lane l the counts of symbols
// 8l .. 8l + 7 and the cumulative counts before them (symbol 255 of lane 31
// is not a symbol and keeps count 0).  Symbol search without the division
// of the target: C <= floor(code / r) exactly when r C <= code (r C < 2^32,
// since C <= total and r total <= range); the symbol is the count of
// cumulative values with r C <= code, less one, its interval the largest
// such value and the smallest other one (or the total), as in the table
// decoder.  Every lane keeps the same decoder state.  The stream framing is
// stream version 3's: the decoder starts from the first four bytes, and up to
// four bytes past the substream's end read as zero.
#include "common.cuh"
#include "kernels.h"

namespace lpc {
namespace {

constexpr int kCdWarps = 4;
constexpr uint32_t kAmInc = 32;
constexpr uint32_t kAmLimit = 1u << 16;
constexpr int64_t kPadBytes = 4;

__global__ void __launch_bounds__(kCdWarps * 32)
k_coarse_decode(const CoarseChunk* __restrict__ ck, int n, const uint8_t* __restrict__ in,
                int* err) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * kCdWarps + (threadIdx.x >> 5);
  if (w >= n) return;
  const CoarseChunk c = ck[w];
  uint8_t* dst = c.out;
  if (c.fill) {  // a frame's carried root: n copies of the code `fill`
    for (int i = lane; i < c.n; i += 32) dst[i] = (uint8_t)c.fill;
    return;
  }
  const bool pad = lane == 31;  // lane 31's entry 7 is symbol 255: no symbol
  uint32_t f[8], cum[8];
#pragma unroll
  for (int m = 0; m < 8; m++) {
    f[m] = (pad && m == 7) ? 0u : 1u;
    cum[m] = 8 * lane + m;  // every count 1: C_s = s
  }
  uint32_t total = 255;
  const uint8_t* p = in + c.in_off;
  const int64_t len = c.in_len;
  auto byte = [&](int64_t i) -> uint32_t { return i < len ? (uint32_t)__ldg(p + i) : 0u; };
  uint32_t code = (byte(0) << 24) | (byte(1) << 16) | (byte(2) << 8) | byte(3);
  uint32_t range = 0xFFFFFFFFu;
  int64_t pos = 4;
  bool bad = false;
  for (int i = 0; i < c.n; i++) {
    const uint32_t b0 = byte(pos), b1 = byte(pos + 1), b2 = byte(pos + 2);
    const uint32_t r = range / total;
    uint32_t cnt = 0, lo = 0, hi = total;
#pragma unroll
    for (int m = 0; m < 8; m++) {
      const bool real = m < 7 || !pad;
      const bool le = real && r * cum[m] <= code;
      cnt += le;
      lo = le ? cum[m] : lo;  // cumulative counts ascend: the last one is the largest
      hi = (real && !le) ? min(hi, cum[m]) : hi;
    }
    const uint32_t s = __reduce_add_sync(0xffffffffu, cnt) - 1;
    lo = __reduce_max_sync(0xffffffffu, lo);
    hi = __reduce_min_sync(0xffffffffu, hi);
    code -= r * lo;
    range = r * (hi - lo);
    if (code >= range) bad = true;
    // renormalise: range >= r >= 255 here, so at most three bytes
    const int nb = (range < (1u << 24)) + (range < (1u << 16)) + (range < (1u << 8));
    const uint64_t wide = ((uint64_t)code << 24) | (b0 << 16) | (b1 << 8) | b2;
    code = (uint32_t)(wide >> (24 - 8 * nb));
    range <<= 8 * nb;
    pos += nb;
    if (lane == 0) dst[i] = (uint8_t)(s + 1);  // symbol s codes occupancy s + 1
    // the model after symbol s
#pragma unroll
    for (int m = 0; m < 8; m++) {
      const uint32_t sym = 8 * lane + m;
      if (sym == s) f[m] += kAmInc;
      if (sym > s) cum[m] += kAmInc;
    }
    total += kAmInc;
    if (total > kAmLimit) {
      uint32_t run = 0;
#pragma unroll
      for (int m = 0; m < 8; m++) {
        f[m] = (f[m] + 1) >> 1;
        cum[m] = run;
        run += f[m];
      }
      uint32_t x = run;  // inclusive scan of the lane sums
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
      }
      const uint32_t before = x - run;
#pragma unroll
      for (int m = 0; m < 8; m++) cum[m] += before;
      total = __shfl_sync(0xffffffffu, x, 31);
    }
  }
  if (pos > len + kPadBytes) bad = true;  // read past the zero bytes a flush may leave out
  if (bad && lane == 0) set_error(err, kErrStream);
}

// Occupancy codes of a coarse level against the next level's size: the
// popcounts of level d's codes add up to N_{d+1} (the header's size).
__global__ void __launch_bounds__(256)
k_coarse_check(const CoarseCheck* __restrict__ ck, int n, int* err) {
  __shared__ uint32_t part[8];
  if (blockIdx.x >= n) return;
  const CoarseCheck c = ck[blockIdx.x];
  uint32_t s = 0;
  for (int64_t i = threadIdx.x; i < c.n; i += blockDim.x) s += __popc((uint32_t)c.codes[i]);
  s = __reduce_add_sync(0xffffffffu, s);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += part[i];
    if ((int64_t)t != c.expect) set_error(err, kErrStream);
  }
}

}  // namespace

void launch_coarse_decode(const CoarseChunk* ck, int n, const uint8_t* in, int* err,
                          cudaStream_t st) {
  if (n <= 0) return;
  k_coarse_decode<<<(n + kCdWarps - 1) / kCdWarps, kCdWarps * 32, 0, st>>>(ck, n, in, err);
  count_launches(1);
}

void launch_coarse_check(const CoarseCheck* ck, int n, int* err, cudaStream_t st) {
  if (n <= 0) return;
  k_coarse_check<<<n, 256, 0, st>>>(ck, n, err);
  count_launches(1);
}

}  // namespace lpc
