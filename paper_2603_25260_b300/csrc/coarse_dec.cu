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
// decoder; the one division a symbol, floor(range / total), is a high
// multiply by a reciprocal formed a symbol ahead.  Every lane keeps the same
// decoder state.  The stream framing is
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
  // cum[m]: the cumulative count before symbol 8 lane + m (lane 31's entry 7
  // stays the total); the counts themselves are only needed when the model
  // halves, and are the differences of neighbouring entries then
  uint32_t cum[8];
#pragma unroll
  for (int m = 0; m < 8; m++) cum[m] = 8 * lane + m;  // every count 1: C_s = s
  uint32_t total = 255;
  // r = floor(range / total) from inv = floor((2^32 - 1) / total): inv >=
  // (2^32 - total) / total, so range inv / 2^32 > range / total - 1 and the
  // high word of range inv is the quotient or one less (one correction).
  // total grows by kAmInc whatever the symbol, so the next reciprocal is
  // formed beside the search instead of a division on the serial chain.
  uint32_t inv = 0xFFFFFFFFu / total;
  const uint8_t* p = in + c.in_off;
  const int64_t len = c.in_len;
  auto byte = [&](int64_t i) -> uint32_t { return i < len ? (uint32_t)__ldg(p + i) : 0u; };
  uint32_t code = (byte(0) << 24) | (byte(1) << 16) | (byte(2) << 8) | byte(3);
  uint32_t range = 0xFFFFFFFFu;
  int64_t pos = 4;
  bool bad = false;
  for (int i = 0; i < c.n; i++) {
    const uint32_t inv_next = 0xFFFFFFFFu / (total + kAmInc);
    const uint32_t b0 = byte(pos), b1 = byte(pos + 1), b2 = byte(pos + 2);
    uint32_t r = __umulhi(range, inv);
    if (range - r * total >= total) r++;
    // cumulative counts increase with the symbol (every count >= 1): one
    // max reduction of the qualifying keys C << 8 | symbol gives the symbol
    // and its interval's start together, a min reduction of the others (or
    // the total) its end
    uint32_t kv[8], hv[8];
#pragma unroll
    for (int m = 0; m < 8; m++) {
      const bool real = m < 7 || !pad;
      const bool le = real && r * cum[m] <= code;
      kv[m] = le ? (cum[m] << 8) | (uint32_t)(8 * lane + m) : 0u;
      hv[m] = (real && !le) ? cum[m] : total;
    }
    const uint32_t kmax = max(max(max(kv[0], kv[1]), max(kv[2], kv[3])), max(max(kv[4], kv[5]), max(kv[6], kv[7])));
    const uint32_t hmin = min(min(min(hv[0], hv[1]), min(hv[2], hv[3])), min(min(hv[4], hv[5]), min(hv[6], hv[7])));
    const uint32_t key = __reduce_max_sync(0xffffffffu, kmax);
    const uint32_t hi = __reduce_min_sync(0xffffffffu, hmin);
    const uint32_t lo = key >> 8, s = key & 0xFFu;
    code -= r * lo;
    range = r * (hi - lo);
    if (code >= range) bad = true;
    // renormalise: range >= r >= 255 here, so at most three bytes
    const int nb = (range < (1u << 24)) + (range < (1u << 16)) + (range < (1u << 8));
    // the top 32 bits of code:b0:b1:b2 shifted left by 8 nb (one funnel shift)
    code = __funnelshift_l((b0 << 24) | (b1 << 16) | (b2 << 8), code, 8 * nb);
    range <<= 8 * nb;
    pos += nb;
    if (lane == 0) dst[i] = (uint8_t)(s + 1);  // symbol s codes occupancy s + 1
    // the model after symbol s: every cumulative count past s grows
    const int ds = (int)s - 8 * lane;
#pragma unroll
    for (int m = 0; m < 8; m++) cum[m] += m > ds ? kAmInc : 0u;
    total += kAmInc;
    inv = inv_next;
    if (total > kAmLimit) {
      // counts from the differences (lane 31's entry 7 has none), halved
      // rounding up, and the cumulative counts again
      const uint32_t nxt = __shfl_down_sync(0xffffffffu, cum[0], 1);
      uint32_t f[8];
#pragma unroll
      for (int m = 0; m < 8; m++)
        f[m] = m < 7 ? cum[m + 1] - cum[m] : (pad ? 0u : nxt - cum[7]);
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
      inv = 0xFFFFFFFFu / total;
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
