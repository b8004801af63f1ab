// Range coding of the network levels on the device, byte-identical to the
// host coder (coder.h): 32-bit range, low kept to 33 bits, a settled byte
// held back with a count of pending 0xFF bytes until the carry is known;
// stream version 3 substreams (the cache's initial byte is not written, the
// flush codes the value with the most trailing zero bits in the final
// interval and leaves out up to four trailing zero bytes, which the decoder
// reads as zero); intervals of a total 2^16 from the integer softmax tables.
//
// Substreams are independent, so every chunk is coded in parallel:
//  - encode: one warp per chunk (its lane 0) walks the packed (lo, f)
//    intervals, or one lane per chunk when chunks are many;
//  - decode: one warp per chunk.  Table rows are staged in shared memory by
//    bulk copies well ahead of use; the 256 entries of a row are spread over
//    the warp, 8 a lane.  The target floor(code / r) is never formed:
//    C <= floor(code / r) holds exactly when r C <= code (r C < 2^32), and
//    the clamp of the target to 2^16 - 1 changes nothing since every C is
//    below 2^16.  The symbol s is the count of entries with r C <= code, the
//    interval [C_s, C_{s+1}) the largest such entry and the smallest other
//    one: a max reduction of keys C << 8 | count (which increase with the
//    entry) and a min reduction, independent of each other.  The two stream bytes a
//    renormalisation can take (range >= 2^8 after every update) are loaded
//    before they are needed.  Every lane keeps the same copy of the decoder
//    state, so no broadcasts are needed.  The symbol loop is a serial chain
//    of dependent instructions in one warp (about 170 ns a symbol on a B300),
//    so a level takes chunk x that: the chunk length sets the latency.
#include "common.cuh"
#include "kernels.h"
#include "tc_util.cuh"

namespace lpc {
namespace {

using tc::fence_async_smem;
using tc::fence_mbar_init;
using tc::mbar_init;
using tc::mbar_wait;
using tc::smem_u32;

constexpr int kEncWarps = 4;
// bytes a substream may be short of at its end (read as zero)
constexpr int kRcPad = 4;
constexpr int kEncAhead = 4;
// With at least this many chunks every lane codes a chunk of its own (the
// warps would otherwise issue one lane's instructions each and the launch
// becomes issue-bound); with fewer, one chunk a warp.
constexpr int kEncLaneChunks = 148 * 32;

// Range-encoder state of one chunk, kept by one thread: put() codes one
// packed interval lo | f << 16, finish() flushes and returns the length.
// low stays below 2^32 + range <= 2^33, so it is kept as its low word l and
// one carry bit c; lengths fit 32 bits (a chunk's capacity does).
struct RcEnc {
  uint8_t* o;
  uint32_t cap;
  uint32_t len = 0;      // counts the leading cache byte too; byte i is o[i - 1]
  uint32_t pending = 1;  // the cache byte and the 0xFF bytes held back with it
  uint32_t l = 0, c = 0;
  uint32_t range = 0xFFFFFFFFu;
  uint32_t cache = 0;

  __device__ __forceinline__ void emit(uint32_t b) {
    if (len - 1 < cap) o[len - 1] = (uint8_t)b;  // 0 < len <= cap
    len++;
  }
  __device__ __forceinline__ void shift_low() {
    if (l < 0xFF000000u || c != 0) {
      emit(cache + c);
      for (; pending > 1; pending--) emit(0xFFu + c);
      pending = 0;
      cache = l >> 24;
    }
    pending++;
    l <<= 8;  // (low mod 2^24) << 8: the top byte leaves, the carry was spent
    c = 0;
  }
  __device__ __forceinline__ void put(uint32_t x) {
    const uint32_t r = range >> 16;
    const uint32_t a = r * (x & 0xFFFFu);  // below 2^32
    l += a;
    c += l < a;
    range = r * (x >> 16);
    while (range < (1u << 24)) {
      range <<= 8;
      shift_low();
    }
  }
  // flush: the multiple of 2^k in [low, low + range) with k largest; up to
  // kRcPad trailing zero bytes are left out
  __device__ uint32_t finish(int* err) {
    const uint64_t low = ((uint64_t)c << 32) | l;
    const uint64_t end = low + range;
    for (int k = 32; k > 0; k--) {
      const uint64_t v = ((low + ((1ull << k) - 1)) >> k) << k;
      if (v < end) {
        l = (uint32_t)v;
        c = (uint32_t)(v >> 32);
        break;
      }
    }
    for (int i = 0; i < 5; i++) shift_low();
    uint32_t n = len - 1;  // the leading cache byte is not part of the stream
    if (n > cap) {
      set_error(err, kErrCapacity);
    } else {
      for (int i = 0; i < kRcPad && n > 0 && o[n - 1] == 0; i++) n--;
    }
    return n;
  }
};

// 4-byte asynchronous copy global -> shared (both 4-byte aligned).
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}

// One chunk per warp, coded by its lane 0 (few chunks: lanes of other chunks
// in the same warp would only lengthen each chain by divergence).  The whole
// warp copies the chunk's intervals into shared memory a piece of
// kEncPiece ahead, so the serial chain reads them at shared-memory latency.
constexpr int kEncPiece = 256;

__global__ void __launch_bounds__(kEncWarps * 32)
k_rc_encode(const RcChunk* __restrict__ ck, int n, const uint32_t* __restrict__ lofreq,
            uint8_t* __restrict__ out, uint32_t* __restrict__ lens, int* err) {
  __shared__ __align__(16) uint32_t stage[kEncWarps][2][kEncPiece];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int t = blockIdx.x * kEncWarps + wi;
  if (t >= n) return;  // t is the same for the whole warp
  const RcChunk c = ck[t];
  const uint32_t* src = lofreq + c.row;
  const int64_t npc = (c.rows + kEncPiece - 1) / kEncPiece;
  auto load = [&](int64_t p) {  // every lane: its entries of piece p, into buffer p & 1
    uint32_t* b = stage[wi][p & 1];
    const int64_t i0 = p * kEncPiece;
    for (int k = lane; k < kEncPiece && i0 + k < c.rows; k += 32)
      cp_async4(smem_u32(b + k), src + i0 + k);
    tc::cp_async_commit();
  };
  RcEnc e;
  e.o = out + c.byte_off;
  e.cap = (uint32_t)min(c.byte_len, (int64_t)0x7fffffff);
  if (npc > 0) load(0);
  for (int64_t p = 0; p < npc; p++) {
    if (p + 1 < npc) {
      load(p + 1);  // in flight while piece p is coded
      tc::cp_async_wait<1>();
    } else {
      tc::cp_async_wait<0>();
    }
    __syncwarp();  // every lane's copies of piece p are visible to lane 0
    if (lane == 0) {
      const uint32_t* b = stage[wi][p & 1];
      const int m = (int)(c.rows - p * kEncPiece < kEncPiece ? c.rows - p * kEncPiece : kEncPiece);
#pragma unroll 8
      for (int k = 0; k < m; k++) e.put(b[k]);
    }
    __syncwarp();  // buffer p & 1 is free for piece p + 2
  }
  if (lane == 0) lens[t] = e.finish(err);
}

// One chunk per lane (many chunks: the lanes' chains hide each other's
// latency); intervals loaded kEncAhead ahead into registers.
__global__ void __launch_bounds__(128)
k_rc_encode_lanes(const RcChunk* __restrict__ ck, int n, const uint32_t* __restrict__ lofreq,
                  uint8_t* __restrict__ out, uint32_t* __restrict__ lens, int* err) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const RcChunk c = ck[t];
  RcEnc e;
  e.o = out + c.byte_off;
  e.cap = (uint32_t)min(c.byte_len, (int64_t)0x7fffffff);
  const uint32_t* src = lofreq + c.row;
  uint32_t nx[kEncAhead];
#pragma unroll
  for (int k = 0; k < kEncAhead; k++) nx[k] = k < c.rows ? __ldg(src + k) : 0u;
  for (int64_t i0 = 0; i0 < c.rows; i0 += kEncAhead) {
#pragma unroll
    for (int k = 0; k < kEncAhead; k++) {
      if (i0 + k < c.rows) {
        const uint32_t x = nx[k];
        if (i0 + k + kEncAhead < c.rows) nx[k] = __ldg(src + i0 + k + kEncAhead);
        e.put(x);
      }
    }
  }
  lens[t] = e.finish(err);
}

// Table rows reach shared memory by bulk copies (TMA, one per stage of
// kStageRows rows, completion counted on the stage's mbarrier) STAGES stages
// ahead of use: rows do not depend on earlier symbols.  A deep ring (8
// stages, 32 KB) hides the copies of a launch with few substreams, where
// each SM holds a few of them; a launch with many substreams (a frame
// batch) takes the 2-stage ring (8 KB), so that about 24 instead of 7 of
// its one-warp blocks fit on a SM and the warps hide each other's waits.
constexpr int kStageRows = 8;
constexpr int kRowBytes = 512;
constexpr int kDeepStages = 8, kShallowStages = 2;
constexpr int kDeepBlocksPerSm = 7;  // 32 KB blocks in 228 KB
template <int STAGES>
constexpr size_t dec_smem() { return (size_t)STAGES * kStageRows * kRowBytes + 8 * STAGES; }

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%2], [%3], %1, [%0];"
      ::"r"(smem_u32(bar)), "r"(bytes), "r"(dst), "l"(src)
      : "memory");
}

template <int STAGES>
__global__ void __launch_bounds__(32)
k_rc_decode(const RcChunk* __restrict__ ck, int n, const int64_t* d_n,
            const uint16_t* __restrict__ cdf, const uint8_t* __restrict__ in,
            uint8_t* __restrict__ codes, int* err) {
  extern __shared__ __align__(128) uint8_t sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + (size_t)STAGES * kStageRows * kRowBytes);
  const int lane = threadIdx.x;
  const int w = blockIdx.x;
  if (d_n) n = (int)min(*d_n, (int64_t)n);
  if (w >= n) return;
  const RcChunk c = ck[w];
  const int64_t nst = (c.rows + kStageRows - 1) / kStageRows;
  const uint8_t* src = reinterpret_cast<const uint8_t*>(cdf + c.row * 256);
  auto issue = [&](int64_t st) {  // lane 0: rows of stage st into its slot
    const int slot = (int)(st % STAGES);
    const int64_t r0 = st * kStageRows;
    const int64_t nr = c.rows - r0 < kStageRows ? c.rows - r0 : kStageRows;
    const uint32_t bytes = (uint32_t)(nr * kRowBytes);
    bulk_g2s(smem_u32(sm + (size_t)slot * kStageRows * kRowBytes), src + r0 * kRowBytes, bytes,
             bar + slot);
  };
  if (lane == 0) {
    for (int s = 0; s < STAGES; s++) mbar_init(bar + s, 1);
    fence_mbar_init();
    for (int64_t st = 0; st < STAGES && st < nst; st++) issue(st);
  }
  __syncwarp();
  const uint8_t* p = in + c.byte_off;
  const uint8_t* const end = p + c.byte_len;
  bool bad = false, lost = false;
  uint32_t range = 0xFFFFFFFFu, code = 0;
  for (int i = 0; i < 4; i++) {
    code = (code << 8) | (p < end ? __ldg(p) : 0u);
    p++;
  }
  // lane l holds entries 8l .. 8l+7 of a row; only entries 0..253 are
  // cumulative values (254, 255 are padding, in lane 31)
  const bool pad = lane == 31;
  uint8_t* dst = codes + c.row;
  int64_t st = 0;
  for (; st < nst; st++) {
    const int slot = (int)(st % STAGES);
    const bool ok = mbar_wait(bar + slot, (uint32_t)((st / STAGES) & 1));
    if (!__all_sync(0xFFFFFFFFu, ok)) {  // leave together
      lost = true;
      break;
    }
    const uint8_t* stage = sm + (size_t)slot * kStageRows * kRowBytes;
    const int64_t r0 = st * kStageRows;
    const int nr = (int)(c.rows - r0 < kStageRows ? c.rows - r0 : kStageRows);
    // the next row's entries are read a symbol ahead.  Entry i of a row is
    // C_{i+1} (C_0 = 0 is implicit), so the symbol is the number of
    // qualifying entries; the keys C_{i+1} << 8 | (i + 1) increase with i
    // (every f >= 1), and one max reduction of the qualifying keys (0 when
    // none qualifies: s = 0, C_0 = 0) gives s and C_s together, beside one
    // min reduction for C_{s+1} (max / min reductions take about half the
    // time of an add reduction)
    uint4 qn = *reinterpret_cast<const uint4*>(stage + 16 * lane);
#pragma unroll
    for (int k = 0; k < kStageRows; k++) {
      const uint4 q = qn;
      if (k + 1 < kStageRows)
        qn = *reinterpret_cast<const uint4*>(stage + (k + 1) * kRowBytes + 16 * lane);
      if (k < nr) {
        const uint32_t b0 = p < end ? __ldg(p) : 0u;
        const uint32_t b1 = p + 1 < end ? __ldg(p + 1) : 0u;
        const uint32_t e[8] = {q.x & 0xFFFFu, q.x >> 16, q.y & 0xFFFFu, q.y >> 16,
                               q.z & 0xFFFFu, q.z >> 16, q.w & 0xFFFFu, q.w >> 16};
        const uint32_t r = range >> 16;
        uint32_t kv[8], hv[8];
#pragma unroll
        for (int m = 0; m < 8; m++) {
          const bool real = m < 6 || !pad;
          const bool le = real && r * e[m] <= code;
          kv[m] = le ? (e[m] << 8) | (uint32_t)(8 * lane + m + 1) : 0u;
          hv[m] = real && !le ? e[m] : 65536u;
        }
        const uint32_t kmax = max(max(max(kv[0], kv[1]), max(kv[2], kv[3])),
                                  max(max(kv[4], kv[5]), max(kv[6], kv[7])));
        const uint32_t hmin = min(min(min(hv[0], hv[1]), min(hv[2], hv[3])),
                                  min(min(hv[4], hv[5]), min(hv[6], hv[7])));
        const uint32_t key = __reduce_max_sync(0xFFFFFFFFu, kmax);
        const uint32_t hi = __reduce_min_sync(0xFFFFFFFFu, hmin);
        const uint32_t lo = key >> 8, s = key & 0xFFu;
        code -= r * lo;
        range = r * (hi - lo);
        if (code >= range) bad = true;
        // renormalise: range >= 2^8 here, so at most two bytes
        const int nb = (range < (1u << 24)) + (range < (1u << 16));
        code = __funnelshift_l((b0 << 24) | (b1 << 16), code, 8 * nb);  // code:b0:b1 << 8 nb
        range <<= 8 * nb;
        p += nb;
        if (lane == 0) dst[r0 + k] = (uint8_t)(s + 1);
      }
    }
    __syncwarp();
    if (lane == 0 && st + STAGES < nst) {
      fence_async_smem();  // this stage's reads come before the copy that reuses it
      issue(st + STAGES);
    }
  }
  if (lost) {
    // a copy never completed: report it and give the copies still counted
    // on the other stages a bounded chance to land before the block exits
    if (lane == 0) set_error(err, kErrTimeout);
    for (int64_t q = st + 1; q < nst && q < st + STAGES; q++)
      mbar_wait(bar + (int)(q % STAGES), (uint32_t)((q / STAGES) & 1));
    return;
  }
  if (p > end + kRcPad) bad = true;  // read past the zero bytes a flush may leave out
  if (bad && lane == 0) set_error(err, kErrStream);
}

}  // namespace

void launch_rc_encode(const RcChunk* ck, int n, const uint32_t* lofreq, uint8_t* out,
                      uint32_t* lens, int* err, cudaStream_t st) {
  if (n <= 0) return;
  if (n >= kEncLaneChunks)
    k_rc_encode_lanes<<<(n + 127) / 128, 128, 0, st>>>(ck, n, lofreq, out, lens, err);
  else
    k_rc_encode<<<(n + kEncWarps - 1) / kEncWarps, kEncWarps * 32, 0, st>>>(ck, n, lofreq, out,
                                                                            lens, err);
  count_launches(1);
}

namespace {
// the deep ring unless the launch has more than two waves of its blocks
bool shallow_ring(int64_t nsub) { return nsub > 2 * 148 * kDeepBlocksPerSm; }
}  // namespace

void launch_rc_decode(const RcChunk* ck, int n, const uint16_t* cdf, const uint8_t* in,
                      uint8_t* codes, int* err, cudaStream_t st) {
  if (n <= 0) return;
  if (shallow_ring(n))
    k_rc_decode<kShallowStages><<<n, 32, dec_smem<kShallowStages>(), st>>>(ck, n, nullptr, cdf,
                                                                           in, codes, err);
  else
    k_rc_decode<kDeepStages><<<n, 32, dec_smem<kDeepStages>(), st>>>(ck, n, nullptr, cdf, in,
                                                                     codes, err);
  count_launches(1);
}

void launch_rc_decode_dev(const RcChunk* ck, const int64_t* d_n, int64_t cap, const uint16_t* cdf,
                          const uint8_t* in, uint8_t* codes, int* err, cudaStream_t st) {
  if (cap <= 0) return;
  if (shallow_ring(cap))
    k_rc_decode<kShallowStages><<<(unsigned)cap, 32, dec_smem<kShallowStages>(), st>>>(
        ck, (int)cap, d_n, cdf, in, codes, err);
  else
    k_rc_decode<kDeepStages><<<(unsigned)cap, 32, dec_smem<kDeepStages>(), st>>>(
        ck, (int)cap, d_n, cdf, in, codes, err);
  count_launches(1);
}

// One block: per frame its chunk count (thread f), the frames' chunk bases
// (a serial prefix over at most 64 frames), then each frame's chunks written
// by the whole block.
__global__ void __launch_bounds__(1024)
k_rc_chunks(const int64_t* __restrict__ foff, int nf, DevSubFrame* fr,
            const int64_t* __restrict__ subs, RcChunk* out, int64_t cap, int64_t maxp,
            int64_t* d_nck, int* err) {
  __shared__ int64_t base[kMaxBatch + 1], nch[kMaxBatch];
  const int t = threadIdx.x;
  if (t < nf) {
    int64_t cnt = foff[t + 1] - foff[t];
    if (cnt > maxp) {
      set_error(err, kErrCapacity);
      cnt = 0;
    }
    nch[t] = (cnt + fr[t].chunk - 1) / fr[t].chunk;
  }
  __syncthreads();
  if (t == 0) {
    int64_t b = 0;
    for (int f = 0; f < nf; f++) {
      base[f] = b;
      if (b + nch[f] > cap) {
        set_error(err, kErrCapacity);
        nch[f] = b < cap ? cap - b : 0;
      }
      b += nch[f];
    }
    base[nf] = b;
    *d_nck = b;
  }
  __syncthreads();
  for (int f = 0; f < nf; f++) {
    const DevSubFrame F = fr[f];
    const int64_t r0 = foff[f], cnt = foff[f + 1] - foff[f];
    for (int64_t c = t; c < nch[f]; c += blockDim.x) {
      const int64_t s = F.next + c;
      RcChunk k{r0 + c * F.chunk, min(F.chunk, cnt - c * F.chunk), 0, 0};
      if (s < F.nsub) {
        k.byte_off = F.in_base + subs[2 * (F.sub0 + s)];
        k.byte_len = subs[2 * (F.sub0 + s) + 1];
      } else {
        set_error(err, kErrStream);  // a frame with too few substreams
      }
      out[base[f] + c] = k;
    }
  }
  __syncthreads();
  if (t < nf) fr[t].next += nch[t];
}

void launch_rc_chunks(const int64_t* foff, int nf, DevSubFrame* fr, const int64_t* subs,
                      RcChunk* out, int64_t cap, int64_t maxp, int64_t* d_nck, int* err,
                      cudaStream_t st) {
  if (nf <= 0) return;
  k_rc_chunks<<<1, 1024, 0, st>>>(foff, nf, fr, subs, out, cap, maxp, d_nck, err);
  count_launches(1);
}

}  // namespace lpc
