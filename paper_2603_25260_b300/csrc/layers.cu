// Integer layers of the network (Sec. 3.1-3.3): occupancy-code embedding,
// Upsampling + Pruning (Eq. 6, 9, 11), the stride-2 sparse conv of
// Downsampling (Eq. 4), and the Predictor (Eq. 7) fused with the integer
// softmax and the cumulative frequency table (Eq. 15).  The 3x3x3 sparse conv
// of the ResBlock runs on the tensor cores (conv_tc.cu).
//
// Layout: one warp per output row, lane = output channel (C = 32).  Input
// rows are int8, read as 16-byte vectors (every lane reads the same row, a
// broadcast); weights sit in shared memory as int8x4 words [slice][cin/4][32]
// so that lane co reads consecutive words (no bank conflicts).  INT8 x INT8
// products accumulate exactly in INT32 with dp4a: sum (x - z) w is computed as
// sum x w - z * sum w, which is the same integer.
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "softmax.cuh"
#include "tc_util.cuh"

namespace lpc {

constexpr int kWarps = 8;  // warps per block of the row kernels
constexpr int kBlocksRow = 148 * 4;

__device__ __forceinline__ int64_t warp_id_global() {
  return (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
}
__device__ __forceinline__ int64_t warps_total() { return (int64_t)gridDim.x * kWarps; }

template <int CIN>
__device__ __forceinline__ void load_row(const int8_t* p, int32_t (&w)[CIN / 4]) {
  const int4* v = reinterpret_cast<const int4*>(p);
#pragma unroll
  for (int i = 0; i < CIN / 16; i++) {
    int4 t = __ldg(v + i);
    w[4 * i] = t.x;
    w[4 * i + 1] = t.y;
    w[4 * i + 2] = t.z;
    w[4 * i + 3] = t.w;
  }
}

// Shared-memory image of one layer: W words, wsum, bias, mult, slope (int32).
// W is kept four words a lane: int4 (slice c, words 4q .. 4q + 3, lane) at
// index (c (cin / 16) + q) 32 + lane, so that a lane reads its weights of
// four dp4a's in one 16-byte load (a warp's load: 512 contiguous bytes).
struct SmemLayer {
  int32_t* W;
  int32_t* wsum;
  int32_t* bias;
  int32_t* mult;
  int32_t* slope;
};

// hi: stage the high-word multipliers (DLayer::mult_hi, which must be set)
__device__ __forceinline__ SmemLayer stage_layer(const DLayer& L, int32_t* sm, bool hi) {
  const int nw = L.S * (L.cin / 4) * 32;
  const int P = L.per_slice ? L.S : 1;
  SmemLayer s;
  s.W = sm;
  s.wsum = s.W + nw;
  s.bias = s.wsum + L.S * 32;
  s.mult = s.bias + P * 32;
  s.slope = s.mult + P * 32;
  // packed word (4 g + e) 32 + lane goes to int4 g 32 + lane, component e;
  // four int4's a thread per pass, their 16 loads in flight together
  const int nq = nw / 4;
  int4* Wq = reinterpret_cast<int4*>(s.W);
  for (int d0 = threadIdx.x; d0 < nq; d0 += 4 * blockDim.x) {
    int32_t v[4][4];
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int d = d0 + e * (int)blockDim.x;
      const int g = (d < nq ? d : 0) >> 5, ln = d & 31;
#pragma unroll
      for (int q = 0; q < 4; q++) v[e][q] = __ldg(L.Wp + (4 * g + q) * 32 + ln);
    }
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int d = d0 + e * (int)blockDim.x;
      if (d < nq) Wq[d] = make_int4(v[e][0], v[e][1], v[e][2], v[e][3]);
    }
  }
  for (int i = threadIdx.x; i < L.S * 32; i += blockDim.x) s.wsum[i] = L.wsum[i];
  const int32_t* mult = hi ? L.mult_hi : L.mult;
  for (int i = threadIdx.x; i < P * 32; i += blockDim.x) {
    s.bias[i] = L.bias[i];
    s.mult[i] = mult[i];
    s.slope[i] = L.slope[i];
  }
  return s;
}

__host__ __device__ __forceinline__ size_t smem_layer_bytes_dev(const DLayer& L) {
  const int P = L.per_slice ? L.S : 1;
  // rounded up to 16 bytes: staging buffers follow the layer image
  return (sizeof(int32_t) * ((size_t)L.S * (L.cin / 4) * 32 + (size_t)L.S * 32 + 3 * (size_t)P * 32) +
          15) & ~(size_t)15;
}
static size_t smem_layer_bytes(const DLayer& L) { return smem_layer_bytes_dev(L); }

template <int CIN>
__device__ __forceinline__ int32_t dot_slice(const int32_t (&x)[CIN / 4], const int32_t* W,
                                             int slice, int lane, int32_t acc) {
  const int4* w = reinterpret_cast<const int4*>(W) + slice * (CIN / 16) * 32 + lane;
#pragma unroll
  for (int q = 0; q < CIN / 16; q++) {
    const int4 t = w[q * 32];
    acc = __dp4a(x[4 * q], t.x, acc);
    acc = __dp4a(x[4 * q + 1], t.y, acc);
    acc = __dp4a(x[4 * q + 2], t.z, acc);
    acc = __dp4a(x[4 * q + 3], t.w, acc);
  }
  return acc;
}

// ------------------------------------------------------------- embedding --
__global__ void k_embed(const int8_t* __restrict__ table, const uint8_t* __restrict__ codes,
                        const int64_t* d_n, int8_t* out, int stride, int col) {
  const int64_t n = *d_n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 2 * n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t >> 1;
    const int h = (int)(t & 1);
    const int4 v = __ldg(reinterpret_cast<const int4*>(table + codes[r] * 32) + h);
    *reinterpret_cast<int4*>(out + r * stride + col + 16 * h) = v;
  }
}

void launch_embed(const DEmb& E, const uint8_t* codes, const int64_t* d_n, int64_t n_host,
                  int8_t* out, int stride, int col, cudaStream_t st) {
  if (n_host <= 0) return;
  int blocks = (int)std::min<int64_t>((2 * n_host + 255) / 256, 148 * 8);
  k_embed<<<blocks, 256, 0, st>>>(E.table, codes, d_n, out, stride, col);
  count_launches(1);
}

// ------------------------------------------------------------- up-prune --
// A warp takes 32 consecutive children at a time: lane i reads child i's
// parent row and slot (coalesced) and copies the parent's input row into the
// warp's shared staging buffer with cp.async, so 32 rows are in flight per
// warp instead of one dependent chain per child; the next 32 rows are copied
// while the current ones are computed (two buffers).  Then the warp walks
// the 32 children, lane = output channel, reading each row as a broadcast.
constexpr int kUpGroup = 32;
constexpr int kUpIlp = 4;  // children computed side by side

// (the 64-bit requantisation: the high-word form's extra registers spill at
// 64 input channels and measured no faster here)
template <int CIN>
__global__ void __launch_bounds__(kWarps * 32)
k_up_prune(DLayer L, const uint64_t* __restrict__ ckey, const uint32_t* __restrict__ cpar,
           const int64_t* d_nc, const int8_t* __restrict__ x, int x_stride, int8_t* out,
           int out_stride, int out_col, EmbSrc oe, int oe_col) {
  extern __shared__ int32_t sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int8_t* stage = reinterpret_cast<int8_t*>(sm + smem_layer_bytes_dev(L) / 4) +
                  (size_t)w * 2 * kUpGroup * CIN;
  const int64_t n = *d_nc;
  const int64_t step = warps_total() * kUpGroup;
  // lane's child of group g0: slot (with oe, its code << 8 beside it), and
  // its parent row copied into buffer b
  auto issue = [&](int64_t g0, int b) -> int {
    const int64_t r = g0 + lane;
    int c = 0;
    const int8_t* src = x;
    if (r < n) {
      c = (int)(__ldg(ckey + r) & 7);
      if (oe.table) c |= (int)__ldg(oe.code + r) << 8;
      src = x + (int64_t)__ldg(cpar + r) * x_stride;
    }
    const uint32_t dst = tc::smem_u32(stage + (b * kUpGroup + lane) * CIN);
#pragma unroll
    for (int k = 0; k < CIN / 16; k++) tc::cp_async16(dst + 16 * k, src + 16 * k, r < n);
    tc::cp_async_commit();
    return c;
  };
  int64_t g0 = warp_id_global() * kUpGroup;
  int b = 0;
  int c_cur = g0 < n ? issue(g0, 0) : 0;  // in flight while the layer is staged
  const SmemLayer s = stage_layer(L, sm, false);
  // embedding rows move as 16-byte pieces when every row start is aligned
  const bool emb16 = ((reinterpret_cast<uintptr_t>(out) | (uintptr_t)out_stride |
                       (uintptr_t)oe_col) & 15) == 0;
  __syncthreads();
  for (; g0 < n; g0 += step, b ^= 1) {
    const int c_next = g0 + step < n ? issue(g0 + step, b ^ 1) : 0;
    if (g0 + step < n)
      tc::cp_async_wait<1>();  // this group's copies have landed
    else
      tc::cp_async_wait<0>();
    __syncwarp();
    const int m = (int)(n - g0 < kUpGroup ? n - g0 : kUpGroup);
    // the next step's Concat(., E[Y]) half: lane j copies child j's row
    if (oe.table && lane < m) {
      const int8_t* es = oe.table + (c_cur >> 8) * 32;
      int8_t* ed = out + (g0 + lane) * out_stride + oe_col;
      if (emb16) {
        const uint4* e4 = reinterpret_cast<const uint4*>(es);
        uint4* d4 = reinterpret_cast<uint4*>(ed);
        d4[0] = __ldg(e4);
        d4[1] = __ldg(e4 + 1);
      } else {
        for (int i = 0; i < 32; i++) ed[i] = __ldg(es + i);
      }
    }
    // the group's children slot by slot: a slot's weight row and constants
    // are loaded once into registers for all its children (lane = output
    // channel), up to kUpIlp children side by side
    const int myslot = lane < m ? (c_cur & 7) : 8;
#pragma unroll 1
    for (int c = 0; c < 8; c++) {
      uint32_t mc = __ballot_sync(0xffffffffu, myslot == c);
      if (!mc) continue;
      const int32_t a0 = s.bias[c * 32 + lane] - L.z_in * s.wsum[c * 32 + lane];
      const int32_t mlt = s.mult[c * 32 + lane], slp = s.slope[c * 32 + lane];
      int4 wr[CIN / 16];
      const int4* Wq = reinterpret_cast<const int4*>(s.W) + c * (CIN / 16) * 32 + lane;
#pragma unroll
      for (int q = 0; q < CIN / 16; q++) wr[q] = Wq[q * 32];
      while (mc) {
        int jj[kUpIlp];  // the next children of slot c (warp-uniform; -1: none)
#pragma unroll
        for (int u = 0; u < kUpIlp; u++) {
          jj[u] = mc ? __ffs(mc) - 1 : -1;
          mc &= mc - 1;
        }
        int32_t acc[kUpIlp];
#pragma unroll
        for (int u = 0; u < kUpIlp; u++) acc[u] = a0;
#pragma unroll
        for (int q = 0; q < CIN / 16; q++)
#pragma unroll
          for (int u = 0; u < kUpIlp; u++) {
            if (jj[u] < 0) continue;
            const int4 x = reinterpret_cast<const int4*>(stage + (b * kUpGroup + jj[u]) * CIN)[q];
            acc[u] = __dp4a(x.x, wr[q].x, acc[u]);
            acc[u] = __dp4a(x.y, wr[q].y, acc[u]);
            acc[u] = __dp4a(x.z, wr[q].z, acc[u]);
            acc[u] = __dp4a(x.w, wr[q].w, acc[u]);
          }
#pragma unroll
        for (int u = 0; u < kUpIlp; u++) {
          if (jj[u] < 0) continue;
          int32_t v = acc[u];
          if (L.prelu) v = prelu(v, slp);
          out[(g0 + jj[u]) * out_stride + out_col + lane] =
              (int8_t)requant(v, mlt, L.shift, L.z_out);
        }
      }
    }
    __syncwarp();  // buffer b is free for the group after next
    c_cur = c_next;
  }
  tc::cp_async_wait<0>();
}

void launch_up_prune(const DLayer& W, const uint64_t* ckey, const uint32_t* cpar,
                     const int64_t* d_nc, int64_t nc_host, const int8_t* x, int x_stride,
                     int8_t* out, int out_stride, int out_col, cudaStream_t st, EmbSrc oe,
                     int oe_col) {
  if (nc_host <= 0) return;
  const size_t smem = smem_layer_bytes(W) + (size_t)kWarps * 2 * kUpGroup * W.cin;
  const int blocks = (int)std::min<int64_t>((nc_host + kWarps * kUpGroup - 1) / (kWarps * kUpGroup),
                                            kBlocksRow);
  auto go = [&](auto k) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<blocks, kWarps * 32, smem, st>>>(W, ckey, cpar, d_nc, x, x_stride, out, out_stride,
                                         out_col, oe, oe_col);
  };
  if (W.cin == 32) go(k_up_prune<32>);
  else go(k_up_prune<64>);
  count_launches(1);
}

// ------------------------------------------------------------ down (s2) --
// A warp takes 16 consecutive parents at a time.  Their children are the
// consecutive rows poff[p0] .. poff[p0 + 16] - 1 (at most 128): the warp
// copies those input rows into its staging buffer with cp.async and their
// slots (key & 7) beside them, the next 16 parents' rows while the current
// ones are computed (two buffers); then it walks the parents, lane = output
// channel, summing the children's slices.
constexpr int kDownGroup = 16;
constexpr int kDownRows = 8 * kDownGroup;

// HI: the layer's multipliers in the high-word form (DLayer::mult_hi)
template <int CIN, bool HI>
__global__ void __launch_bounds__(kWarps * 32)
k_down(DLayer L, const uint64_t* __restrict__ ckey, const uint32_t* __restrict__ poff,
       const int64_t* d_np, const int8_t* __restrict__ x, int x_stride, int8_t* out,
       int out_stride, int out_col) {
  extern __shared__ int32_t sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int kBuf = kDownRows * CIN + kDownRows;  // rows, then slots
  int8_t* stage = reinterpret_cast<int8_t*>(sm + smem_layer_bytes_dev(L) / 4) + (size_t)w * 2 * kBuf;
  const int64_t n = *d_np;
  const int64_t step = warps_total() * kDownGroup;
  // lane j <= 16 holds poff[p0 + j] (clamped at the last parent)
  auto issue = [&](int64_t p0, int b) -> uint32_t {
    const int64_t pj = p0 + (lane <= kDownGroup ? lane : kDownGroup);
    const uint32_t o = __ldg(poff + (pj < n ? pj : n));
    const uint32_t o0 = __shfl_sync(0xffffffffu, o, 0), o1 = __shfl_sync(0xffffffffu, o, kDownGroup);
    const int rows = min((int)(o1 - o0), kDownRows);  // 8 children a parent at most
    int8_t* buf = stage + b * kBuf;
    const uint32_t dst = tc::smem_u32(buf);
    for (int k = lane; k < rows * (CIN / 16); k += 32) {
      const int r = k / (CIN / 16), part = k % (CIN / 16);
      tc::cp_async16(dst + r * CIN + 16 * part, x + (int64_t)(o0 + r) * x_stride + 16 * part, true);
    }
    tc::cp_async_commit();
    for (int r = lane; r < rows; r += 32) buf[kDownRows * CIN + r] = (int8_t)(__ldg(ckey + o0 + r) & 7);
    return o;
  };
  int64_t p0 = warp_id_global() * kDownGroup;
  int b = 0;
  uint32_t o_cur = p0 < n ? issue(p0, 0) : 0;  // in flight while the layer is staged
  const SmemLayer s = stage_layer(L, sm, HI);
  __syncthreads();
  for (; p0 < n; p0 += step, b ^= 1) {
    const uint32_t o_next = p0 + step < n ? issue(p0 + step, b ^ 1) : 0;
    if (p0 + step < n)
      tc::cp_async_wait<1>();
    else
      tc::cp_async_wait<0>();
    __syncwarp();
    const int8_t* buf = stage + b * kBuf;
    const uint32_t o0 = __shfl_sync(0xffffffffu, o_cur, 0);
    const int m = (int)(n - p0 < kDownGroup ? n - p0 : kDownGroup);
    // four parents at a time: their children's dp4a chains are independent;
    // a parent with fewer children repeats its last row and drops the sum.
    // A parent without children (a corrupt code 0, or the capacity clamp)
    // reads row ra, which this group may not have copied: its slot is masked
    // so that a stale byte still indexes the weights in range.
    int j = 0;
    for (; j + kUpIlp <= m; j += kUpIlp) {
      int ra[kUpIlp], len[kUpIlp], maxlen = 0;
      int32_t acc[kUpIlp];
#pragma unroll
      for (int u = 0; u < kUpIlp; u++) {
        ra[u] = min((int)(__shfl_sync(0xffffffffu, o_cur, j + u) - o0), kDownRows);
        const int rb = min((int)(__shfl_sync(0xffffffffu, o_cur, j + u + 1) - o0), kDownRows);
        len[u] = rb - ra[u];
        maxlen = max(maxlen, len[u]);
        acc[u] = s.bias[lane];
      }
      for (int k = 0; k < maxlen; k++) {
        int c[kUpIlp];
        int32_t xv[kUpIlp][CIN / 4], part[kUpIlp];
#pragma unroll
        for (int u = 0; u < kUpIlp; u++) {
          const int r = ra[u] + max(0, min(k, len[u] - 1));
          c[u] = buf[kDownRows * CIN + r] & 7;
          const int4* row = reinterpret_cast<const int4*>(buf + r * CIN);
#pragma unroll
          for (int i = 0; i < CIN / 16; i++) {
            const int4 t = row[i];
            xv[u][4 * i] = t.x, xv[u][4 * i + 1] = t.y, xv[u][4 * i + 2] = t.z,
            xv[u][4 * i + 3] = t.w;
          }
          part[u] = -L.z_in * s.wsum[c[u] * 32 + lane];
        }
        const int4* Wq = reinterpret_cast<const int4*>(s.W) + lane;
#pragma unroll
        for (int q = 0; q < CIN / 16; q++)
#pragma unroll
          for (int u = 0; u < kUpIlp; u++) {
            const int4 t = Wq[(c[u] * (CIN / 16) + q) * 32];
            part[u] = __dp4a(xv[u][4 * q], t.x, part[u]);
            part[u] = __dp4a(xv[u][4 * q + 1], t.y, part[u]);
            part[u] = __dp4a(xv[u][4 * q + 2], t.z, part[u]);
            part[u] = __dp4a(xv[u][4 * q + 3], t.w, part[u]);
          }
#pragma unroll
        for (int u = 0; u < kUpIlp; u++) acc[u] += k < len[u] ? part[u] : 0;
      }
#pragma unroll
      for (int u = 0; u < kUpIlp; u++) {
        int32_t a = acc[u];
        if (L.prelu) a = prelu(a, s.slope[lane]);
        out[(p0 + j + u) * out_stride + out_col + lane] =
            (int8_t)(HI ? requant_hi(a, s.mult[lane], L.z_out)
                    : requant(a, s.mult[lane], L.shift, L.z_out));
      }
    }
    for (; j < m; j++) {
      const int r0 = min((int)(__shfl_sync(0xffffffffu, o_cur, j) - o0), kDownRows);
      const int r1 = min((int)(__shfl_sync(0xffffffffu, o_cur, j + 1) - o0), kDownRows);
      int32_t acc = s.bias[lane];
      for (int r = r0; r < r1; r++) {
        const int c = buf[kDownRows * CIN + r];
        int32_t xv[CIN / 4];
        const int4* row = reinterpret_cast<const int4*>(buf + r * CIN);
#pragma unroll
        for (int i = 0; i < CIN / 16; i++) {
          const int4 t = row[i];
          xv[4 * i] = t.x, xv[4 * i + 1] = t.y, xv[4 * i + 2] = t.z, xv[4 * i + 3] = t.w;
        }
        acc -= L.z_in * s.wsum[c * 32 + lane];
        acc = dot_slice<CIN>(xv, s.W, c, lane, acc);
      }
      if (L.prelu) acc = prelu(acc, s.slope[lane]);
      out[(p0 + j) * out_stride + out_col + lane] =
          (int8_t)(HI ? requant_hi(acc, s.mult[lane], L.z_out)
               : requant(acc, s.mult[lane], L.shift, L.z_out));
    }
    __syncwarp();  // buffer b is free for the group after next
    o_cur = o_next;
  }
  tc::cp_async_wait<0>();
}

void launch_down(const DLayer& W, const uint64_t* ckey, const uint32_t* poff, const int64_t* d_np,
                 int64_t np_host, const int8_t* x, int x_stride, int8_t* out, int out_stride,
                 int out_col, cudaStream_t st) {
  if (np_host <= 0) return;
  const size_t smem =
      smem_layer_bytes(W) + (size_t)kWarps * 2 * ((size_t)kDownRows * W.cin + kDownRows);
  const int64_t want = (np_host + kWarps * kDownGroup - 1) / (kWarps * kDownGroup);
  auto go = [&](auto k) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // at most one wave of resident blocks (the warps stride over the
    // parents): a second, partial wave cost nearly a whole one's latency
    static int per_sm = 0;
    if (!per_sm && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWarps * 32, smem) !=
                        cudaSuccess ||
                    per_sm < 1)) {
      cudaGetLastError();
      per_sm = kBlocksRow / 148;
    }
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, 148 * per_sm));
    k<<<blocks, kWarps * 32, smem, st>>>(W, ckey, poff, d_np, x, x_stride, out, out_stride,
                                         out_col);
  };
  const bool hi = W.mult_hi != nullptr;
  if (W.cin == 32) go(hi ? k_down<32, true> : k_down<32, false>);
  else go(hi ? k_down<64, true> : k_down<64, false>);
  count_launches(1);
}

// Eq. 14 in a cheaper exact form when the shift r <= 32 and the multiplier
// scaled by 2^(32 - r) stays below 2^31: floor((a m + 2^(r-1)) / 2^r) is the
// high word of a (m 2^(32-r)) + 2^31; the zero point joins the high word.
__global__ void __launch_bounds__(kWarps * 32)
k_softmax_cdf(const int8_t* __restrict__ logits, int64_t n, const uint32_t* __restrict__ lut,
              uint16_t* cdf) {
  __shared__ uint32_t slut[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) slut[i] = lut[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  int ck[8];
  tie_keys(lane, ck);
  for (int64_t r = warp_id_global(); r < n; r += warps_total()) {
    int l[8];
#pragma unroll
    for (int i = 0; i < 8; i++) l[i] = lane * 8 + i < kNsym ? logits[r * kNsym + lane * 8 + i] : 0;
    SoftRow o;
    softmax_row(l, ck, lane == 31, slut, o);
    store_cdf_row(o, lane, cdf + r * 256);
  }
}

void launch_softmax_cdf(const int8_t* logits, int64_t n, const uint32_t* lut, uint16_t* cdf,
                        cudaStream_t st) {
  if (n <= 0) return;
  const int blocks = (int)std::min<int64_t>((n + kWarps - 1) / kWarps, kBlocksRow);
  k_softmax_cdf<<<blocks, kWarps * 32, 0, st>>>(logits, n, lut, cdf);
  count_launches(1);
}

// ----------------------------------- predictor, CUDA-core (dp4a) variant --
// h = requant(prelu(W1 (F - z1) + b1)) (C -> C), logits = requant(W2 (h - z2)
// + b2) (C -> 255), then the integer softmax.  Modes: full CDF row, the
// (C_s, f_s) pair of the true symbol (encoder), or the logits (debug).
__global__ void __launch_bounds__(kWarps * 32)
k_predictor_dp4a(DLayer P1, DPred2 P2, const uint32_t* __restrict__ lut,
            const int8_t* __restrict__ F, int f_stride, const int64_t* d_n, int mode,
            const uint8_t* __restrict__ codes, uint16_t* cdf, uint32_t* enc, int8_t* logits) {
  __shared__ int32_t sW1[8 * 32], sW1s[32], sB1[32], sM1[32], sS1[32];
  __shared__ int32_t sW2[8 * 8 * 32];
  __shared__ int32_t sW2s[256], sB2[256], sM2[256];
  __shared__ uint32_t slut[256];
  __shared__ int32_t hbuf[kWarps][8];
  for (int i = threadIdx.x; i < 8 * 32; i += blockDim.x) sW1[i] = P1.Wp[i];
  for (int i = threadIdx.x; i < 8 * 8 * 32; i += blockDim.x) sW2[i] = P2.Wp[i];
  bool ok = true;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    sW2s[i] = P2.wsum[i];
    sB2[i] = P2.bias[i];
    slut[i] = lut[i];
    ok = ok && hi_ok(P2.mult[i], P2.shift);
  }
  // the logits' requantisation takes the high-word form when every
  // multiplier admits it
  const bool fast2 = __syncthreads_and(ok);
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    sM2[i] = fast2 ? hi_scale(P2.mult[i], P2.shift) : P2.mult[i];
  for (int i = threadIdx.x; i < 32; i += blockDim.x) {
    sW1s[i] = P1.wsum[i];
    sB1[i] = P1.bias[i];
    sM1[i] = P1.mult[i];
    sS1[i] = P1.slope[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int ck[8];
  tie_keys(lane, ck);
  const int64_t n = *d_n;
  for (int64_t r = warp_id_global(); r < n; r += warps_total()) {
    int32_t xv[8];
    load_row<32>(F + r * f_stride, xv);
    int32_t a = sB1[lane] - P1.z_in * sW1s[lane];
#pragma unroll
    for (int k = 0; k < 8; k++) a = __dp4a(xv[k], sW1[k * 32 + lane], a);
    if (P1.prelu) a = prelu(a, sS1[lane]);
    const int h = requant(a, sM1[lane], P1.shift, P1.z_out);
    reinterpret_cast<int8_t*>(hbuf[w])[lane] = (int8_t)h;
    __syncwarp();
    int32_t hv[8];
#pragma unroll
    for (int k = 0; k < 8; k++) hv[k] = hbuf[w][k];
    __syncwarp();
    int l[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
      const int sidx = lane * 8 + i;
      int32_t acc = sB2[sidx] - P2.z_in * sW2s[sidx];
#pragma unroll
      for (int k = 0; k < 8; k++) acc = __dp4a(hv[k], sW2[(i * 8 + k) * 32 + lane], acc);
      l[i] = fast2 ? requant_hi(acc, sM2[sidx], P2.z_out)
                   : requant(acc, sM2[sidx], P2.shift, P2.z_out);
    }
    if (mode == kPredLogits) {
#pragma unroll
      for (int i = 0; i < 8; i++)
        if (lane * 8 + i < kNsym) logits[r * kNsym + lane * 8 + i] = (int8_t)l[i];
      continue;
    }
    SoftRow o;
    softmax_row(l, ck, lane == 31, slut, o);
    if (mode == kPredCdf) {
      store_cdf_row(o, lane, cdf + r * 256);
    } else {
      const int s = (int)codes[r] - 1;
      const uint32_t pair = enc_pair(o, lane, s);
      if ((s >> 3) == lane) enc[r] = pair;
    }
  }
}

// ------------------------------------------- predictor + softmax + CDF --
// h = requant(prelu(W1 (F - z1) + b1)) (C -> C), logits = requant(W2 (h - z2)
// + b2) (C -> 255) on the tcgen05 tensor cores, then the integer softmax.
// Modes: full CDF row, the (C_s, f_s) pair of the true symbol (encoder), or
// the logits (debug).
//
// One persistent CTA of 16 warps per SM, as two independent groups of 8
// warps that take alternate tiles of 128 rows (own shared-memory tiles, own
// half of TMEM, own mbarrier, own named barrier), so that one group's MMA
// waits and loads overlap the other group's arithmetic.  Per tile: the rows
// (F - z1) go to shared memory as bf16 (exact: |F - z1| <= 255), an M=128
// N=32 K=32 MMA gives layer 1 in TMEM (every fp32 partial sum is an integer
// below 2^22: 32 products of at most 255 * 127), the warps write (h - z2)
// back as bf16 (warp: TMEM lane quadrant and half of the columns), an M=128
// N=256 K=32 MMA gives the 255 logits.  The softmax then runs one thread per
// half row, on the half row the thread reads from TMEM (row = its TMEM lane,
// half = its warp's column half), in four passes over its 128 symbols with
// the two halves of a row exchanging one word through shared memory after
// each of the first three: (1) requantise into 16-bit keys kept in the
// shared tile, smallest key; (2) S from the bank-replicated exp table;
// (3) the quotients by one exact 40-bit reciprocal of S, f = 1 + q stored in
// place of the keys; (4) the cumulative row two entries per multiply-add,
// in place, copied out coalesced.  Per-row work that a warp-per-row softmax
// spends on reductions and scans is here a handful of scalar instructions
// per thread.
namespace {

constexpr int kPTile = 128;
constexpr int kPThreads = 512;
constexpr int kPGroup = 256;     // threads of one group
constexpr int kLogStride = 528;  // key row stride in shared memory (16 B x odd: conflict-free)
constexpr int kPredB1 = 0, kPredB2 = 2048;  // weight images
constexpr int kPredA = 18432;               // per group: A1 (8 KB), A2 (8 KB)
constexpr int kPredLg = kPredA + 2 * 16384; // per group: key tile (128 rows of 256 u16)
constexpr int kPredTab = kPredLg + 2 * kPTile * kLogStride;  // exp table, one copy per bank
constexpr int kPredSmem = 1024 + kPredTab + 256 * 32 * 4;

__device__ int g_pred_error = 0;

// Named barrier of one group (ids 1 and 2; 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(kPGroup) : "memory");
}
__device__ __forceinline__ bool group_sync_or(int g, bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, %2, %3, p;\n"
      "selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(1 + g), "n"(kPGroup)
      : "memory");
  return r != 0;
}

// fp32 x holding an integer |x| < 2^22: x + 1.5 2^23 has unit spacing, so
// its bits are kMagicBits + x exactly; (bits - (kMagicBits - b)) = x + b.
constexpr float kMagic = 12582912.0f;
constexpr uint32_t kMagicBits = 0x4B400000u;
__device__ __forceinline__ int32_t acc_plus(float x, int32_t off) {
  return (int32_t)(__float_as_uint(x + kMagic) - (uint32_t)off);
}

// 8 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8f(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}

// 8 values (v - z) as bf16: chunk c of row `row` of a 64-byte-row,
// 64-byte-swizzled tile at smem address base.
__device__ __forceinline__ void bf16_chunk8(const int32_t (&v)[8], int z, uint32_t base, int row,
                                            int c) {
  uint32_t w[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const __nv_bfloat162 p =
        __halves2bfloat162(__int2bfloat16_rn(v[2 * k] - z), __int2bfloat16_rn(v[2 * k + 1] - z));
    w[k] = *reinterpret_cast<const uint32_t*>(&p);
  }
  const uint32_t a = base + tc::swz<64>(row * 64 + c * 16);
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(w[0]), "r"(w[1]),
               "r"(w[2]), "r"(w[3])
               : "memory");
}

__global__ void __launch_bounds__(kPThreads, 1)
k_predictor_tc(DLayer P1, DPred2 P2, const uint32_t* __restrict__ lut,
               const int8_t* __restrict__ F, int f_stride, const int64_t* d_n, int mode,
               const uint8_t* __restrict__ codes, uint16_t* cdf, uint32_t* enc, int8_t* logits) {
  extern __shared__ unsigned char smraw[];
  // aligned to 1024 by offsetting smraw itself, so that accesses through sm
  // stay shared-memory accesses (an integer round trip would make them generic)
  unsigned char* sm = smraw + ((1024u - (tc::smem_u32(smraw) & 1023u)) & 1023u);
  __shared__ int32_t sB1[32], sM1[32], sS1[32];
  __shared__ __align__(16) int32_t sB2[256], sM2[256];
  __shared__ __align__(16) long long sK2[256];
  __shared__ uint64_t mbars[2];
  __shared__ uint32_t tslot;
  // per group, half and row: the two halves of a row exchange their smallest
  // key, then their S, then their sum of q (two arrays used alternately)
  __shared__ uint32_t sXa[2][2][kPTile], sXb[2][2][kPTile];
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (w == 0) tc::tmem_alloc(&tslot, 512);
  if (t == 0) {
    tc::mbar_init(&mbars[0], 1);
    tc::mbar_init(&mbars[1], 1);
    tc::fence_mbar_init();
  }
  // requantisation in the high-word form when every multiplier of a layer
  // admits it; accumulators leave TMEM as fp32 holding integers below 2^22
  // in magnitude (32 products of at most 255 x 127), converted exactly by
  // adding 1.5 2^23 and reading the bits, the bias folded into the offset
  const bool fast2 = __syncthreads_and(t >= 256 || hi_ok(P2.mult[t], P2.shift));
  const bool fast1 = __syncthreads_and(t >= 32 || hi_ok(P1.mult[t], P1.shift));
  if (t < 256) {
    const uint32_t off = kMagicBits - (uint32_t)P2.bias[t];
    sB2[t] = (int32_t)off;
    sM2[t] = P2.mult[t];
    sK2[t] = 0;
    if (fast2) {
      // the key's 127 - l in the high-word form: with the accumulator's bits
      // v = off + a, a ms + 2^31 + z 2^32 = v ms + K, K = 2^31 + z 2^32 -
      // off ms, and 127 - floor(y / 2^32) = floor((128 2^32 - 1 - y) / 2^32),
      // so 127 - l = high word of v (-ms) + (128 2^32 - 1 - K) before the
      // clamp (one wide multiply-add); the padding column gives 255
      const long long ms = hi_scale(P2.mult[t], P2.shift);
      const long long K = 2147483648ll + (long long)P2.z_out * 4294967296ll - (long long)off * ms;
      sM2[t] = t < kNsym ? (int32_t)-ms : 0;
      sK2[t] = t < kNsym ? 128ll * 4294967296ll - 1 - K : 255ll * 4294967296ll;
    }
  }
  {  // the exp table, word 32 d + j = lut[d] for every bank j: the 256
     // entries read from global memory once (one load a thread instead of
     // sixteen), then replicated from shared memory
    uint32_t* tab = reinterpret_cast<uint32_t*>(sm + kPredTab);
    __shared__ uint32_t slut0[256];
    if (t < 256) slut0[t] = __ldg(lut + t);
    __syncthreads();
    for (int i = t; i < 256 * 32; i += kPThreads) tab[i] = slut0[i >> 5];
  }
  if (t < 32) {
    sB1[t] = (int32_t)(kMagicBits - (uint32_t)P1.bias[t]);
    sM1[t] = fast1 ? hi_scale(P1.mult[t], P1.shift) : P1.mult[t];
    sS1[t] = P1.prelu ? P1.slope[t] : 0;
  }
  {  // the weight images: layer 1 (2 KB) and layer 2 (16 KB)
    const uint4* s1 = reinterpret_cast<const uint4*>(P1.Wtc);
    const uint4* s2 = reinterpret_cast<const uint4*>(P2.Wtc);
    uint4* d1 = reinterpret_cast<uint4*>(sm + kPredB1);
    uint4* d2 = reinterpret_cast<uint4*>(sm + kPredB2);
    if (t < 128) d1[t] = __ldg(s1 + t);
    for (int i = t; i < 1024; i += kPThreads) d2[i] = __ldg(s2 + i);
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const int g = w >> 3, wl = w & 7, tl = t & (kPGroup - 1);  // group, warp and thread in it
  const uint32_t tbase = tslot + 256 * g;
  uint64_t* mbar = &mbars[g];
  const uint32_t tab_lane = tc::smem_u32(sm + kPredTab) + 4u * (uint32_t)lane;
  const int quad = wl & 3, cg = wl >> 2;  // TMEM lane quadrant, column half
  const int erow = quad * 32 + lane;      // tile row this thread handles in the epilogues
  const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
  const uint32_t sA1 = tc::smem_u32(sm + kPredA + g * 16384), sA2 = sA1 + 8192;
  const uint32_t sB1w = tc::smem_u32(sm + kPredB1), sB2w = tc::smem_u32(sm + kPredB2);
  unsigned char* sLg = sm + kPredLg + g * (kPTile * kLogStride);
  const int64_t n = *d_n;
  const int64_t ntiles = (n + kPTile - 1) / kPTile;
  uint32_t phase = 0;
  bool ok = true;
  // this thread's 16 input bytes of a tile (row, 16-column half), loaded a
  // tile ahead so that the load's latency overlaps the previous tile
  const int in_row = tl >> 1, in_c2 = tl & 1;
  auto load_in = [&](int64_t tile) {
    const int64_t r = tile * kPTile + in_row;
    return tile < ntiles && r < n
               ? __ldg(reinterpret_cast<const uint4*>(F + r * f_stride) + in_c2)
               : make_uint4(0, 0, 0, 0);
  };
  uint4 q_next = load_in(2 * (int64_t)blockIdx.x + g);
  for (int64_t tile = 2 * (int64_t)blockIdx.x + g; tile < ntiles; tile += 2 * (int64_t)gridDim.x) {
    const int64_t r0 = tile * kPTile;
    // ---- layer-1 input: (F - z1) as bf16, thread = (row, 16-column half)
    {
      const int row = in_row, c2 = in_c2;
      const uint4 q = q_next;
      q_next = load_in(tile + 2 * (int64_t)gridDim.x);
      int32_t v[2][8];
      if (r0 + row < n) {
        const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 16; k++) v[k >> 3][k & 7] = (int)(wd[k >> 2] << (24 - 8 * (k & 3))) >> 24;
      } else {
#pragma unroll
        for (int k = 0; k < 16; k++) v[k >> 3][k & 7] = P1.z_in;
      }
      bf16_chunk8(v[0], P1.z_in, sA1, row, 2 * c2);
      bf16_chunk8(v[1], P1.z_in, sA1, row, 2 * c2 + 1);
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    group_sync(g);
    if (tl == 0) {
      tc::tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < 2; ks++)
        tc::mma_bf16(tbase, tc::smem_desc<64>(sA1 + ks * 32, 512),
                     tc::smem_desc<64>(sB1w + ks * 32, 512), tc::idesc_bf16(kPTile, 32),
                     ks ? 1u : 0u);
      tc::mma_commit(mbar);
    }
    ok = tc::mbar_wait(mbar, phase);
    phase ^= 1;
    if (group_sync_or(g, !ok)) {
      ok = false;
      break;
    }
    tc::tc_fence_after();
    // ---- layer-1 epilogue: 16 columns a warp; (h - z2) as bf16
#pragma unroll
    for (int hh = 0; hh < 2; hh++) {
      const int cb = 16 * cg + 8 * hh;
      float fv[8];
      int32_t v[8];
      tmem_ld8f(tbase + lane_off + cb, fv);
#pragma unroll
      for (int i = 0; i < 8; i++) {
        const int c = cb + i;
        int32_t a = acc_plus(fv[i], sB1[c]);
        if (P1.prelu) a = prelu(a, sS1[c]);
        v[i] = fast1 ? requant_hi(a, sM1[c], P1.z_out) : requant(a, sM1[c], P1.shift, P1.z_out);
      }
      bf16_chunk8(v, P2.z_in, sA2, erow, 2 * cg + hh);
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    group_sync(g);
    if (tl == 0) {
      tc::tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < 2; ks++)
        tc::mma_bf16(tbase, tc::smem_desc<64>(sA2 + ks * 32, 512),
                     tc::smem_desc<64>(sB2w + ks * 32, 512), tc::idesc_bf16(kPTile, 256),
                     ks ? 1u : 0u);
      tc::mma_commit(mbar);
    }
    ok = tc::mbar_wait(mbar, phase);
    phase ^= 1;
    if (group_sync_or(g, !ok)) {
      ok = false;
      break;
    }
    tc::tc_fence_after();
    // ---- pass 1: this thread's half row (row erow, symbols 128 cg ..
    // 128 cg + 127) of logits from TMEM, requantised into the keys
    // (127 - l) 128 + (s & 127) (saturating packs clamp 127 - l to 0..255);
    // their smallest key, and their table offsets (127 - l) 128 stored in
    // the shared tile; the accumulator columns come in pairs of 16-column
    // loads per wait
    const int64_t r = r0 + erow;
    unsigned char* rowp = sLg + erow * kLogStride + 256 * cg;
    uint4* row4 = reinterpret_cast<uint4*>(rowp);
    uint16_t* row16 = reinterpret_cast<uint16_t*>(rowp);
    uint32_t mn = 0xFFFFFFFFu;
    uint32_t fr[2][16];
#pragma unroll
    for (int gi = 0; gi < 8; gi++) {
      const int c0 = 128 * cg + 16 * gi;
      if ((gi & 1) == 0) {
        tc::tmem_ld16_issue(tbase + lane_off + c0, fr[0]);
        tc::tmem_ld16_issue(tbase + lane_off + c0 + 16, fr[1]);
        tc::tmem_wait_ld();
        tc::tmem_regs_ready(fr[0]);
        tc::tmem_regs_ready(fr[1]);
      }
      int32_t u[16];
      if (fast2) {
        int32_t ms[16];
        long long kk[16];
#pragma unroll
        for (int i = 0; i < 16; i += 4) {
          const int4 m4 = *reinterpret_cast<const int4*>(sM2 + c0 + i);
          ms[i] = m4.x, ms[i + 1] = m4.y, ms[i + 2] = m4.z, ms[i + 3] = m4.w;
        }
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
          const longlong2 k2 = *reinterpret_cast<const longlong2*>(sK2 + c0 + i);
          kk[i] = k2.x, kk[i + 1] = k2.y;
        }
#pragma unroll
        for (int i = 0; i < 16; i++) {
          const int32_t v = (int32_t)__float_as_uint(__uint_as_float(fr[gi & 1][i]) + kMagic);
          u[i] = (int)(((long long)v * ms[i] + kk[i]) >> 32);
        }
      } else {
#pragma unroll
        for (int i = 0; i < 16; i++) {
          const int c = c0 + i;
          const int32_t a = acc_plus(__uint_as_float(fr[gi & 1][i]), sB2[c]);
          u[i] = c >= kNsym ? 255 : 127 - requant(a, sM2[c], P2.shift, P2.z_out);
        }
      }
      if (mode == kPredLogits && r < n) {
#pragma unroll
        for (int i = 0; i < 16; i++)
          if (c0 + i < kNsym) logits[r * kNsym + c0 + i] = (int8_t)(127 - min(max(u[i], 0), 255));
      }
      uint32_t kw[8];
#pragma unroll
      for (int j = 0; j < 4; j++) {
        uint32_t p2, p4;  // saturated bytes u[4j .. 4j + 3]
        asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, 0;" : "=r"(p2) : "r"(u[4 * j + 3]), "r"(u[4 * j + 2]));
        asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, %3;"
            : "=r"(p4)
            : "r"(u[4 * j + 1]), "r"(u[4 * j]), "r"(p2));
        const uint32_t s4 = (uint32_t)(16 * gi + 4 * j);  // s & 127 of u[4j]
        kw[2 * j] = __byte_perm(p4, 0, 0x4140) * 128u + (s4 | ((s4 + 1) << 16));
        kw[2 * j + 1] = __byte_perm(p4, 0, 0x4342) * 128u + ((s4 + 2) | ((s4 + 3) << 16));
        mn = min_u16x2(mn, min_u16x2(kw[2 * j], kw[2 * j + 1]));
      }
      // the tile keeps the table offsets (127 - l) 128 only
      row4[2 * gi] = make_uint4(kw[0] & kKeyOff2, kw[1] & kKeyOff2, kw[2] & kKeyOff2, kw[3] & kKeyOff2);
      row4[2 * gi + 1] =
          make_uint4(kw[4] & kKeyOff2, kw[5] & kKeyOff2, kw[6] & kKeyOff2, kw[7] & kKeyOff2);
    }
    // the row's key (127 - l) 256 + s of its largest logit at its lowest index
    mn = min(mn & 0xFFFFu, mn >> 16);
    const uint32_t hkey = ((mn & kKeyOff) << 1) | (uint32_t)(128 * cg) | (mn & 127u);
    sXa[g][cg][erow] = hkey;
    tc::tc_fence_before();
    group_sync(g);
    if (mode == kPredLogits) continue;
    // ---- pass 2: S = sum of e_s = lut[(127 - l_s) - u0] over the row, the
    // table read from the copy in this thread's bank
    const uint32_t key = min(hkey, sXa[g][cg ^ 1][erow]);
    const int first = (int)(key & 255u);
    const uint32_t tb = tab_lane - (key >> 8) * 128u;
    uint32_t S = 0;
#pragma unroll 4
    for (int c = 0; c < 16; c++) {
      const uint4 k4 = row4[c];
      const uint32_t kv[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const uint32_t e0 = lds_u32(tb + (kv[j] & 0xFFFFu));
        uint32_t e1 = lds_u32(tb + (kv[j] >> 16));
        if (c == 15 && j == 3) e1 = cg ? 0u : e1;  // the padding entry takes no frequency
        S += e0 + e1;
      }
    }
    sXb[g][cg][erow] = S;
    group_sync(g);
    S += sXb[g][cg ^ 1][erow];
    // ---- pass 3: q_s = floor(e_s (2^16 - 255) / S) = floor(e_s A / 2^40)
    // with A = ceil((2^16 - 255) 2^40 / S): exact for every e_s <= 2^16 as
    // e_s S < 2^40 (the rounding up of A moves e_s A / 2^40 by less than
    // 1 / S, less than the distance of a non-integer e_s K / S to the next
    // integer); f_s = 1 + q_s stored in place of the keys, two to a word
    const unsigned long long A =
        (((unsigned long long)kQScale << 40) + S - 1) / (unsigned long long)S;
    const uint32_t ahi = (uint32_t)(A >> 32), alo = (uint32_t)A;
    uint32_t tot = 0;
#pragma unroll 4
    for (int c = 0; c < 16; c++) {
      const uint4 k4 = row4[c];
      const uint32_t kv[4] = {k4.x, k4.y, k4.z, k4.w};
      uint32_t fw[4];
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const uint32_t e0 = lds_u32(tb + (kv[j] & 0xFFFFu));
        uint32_t e1 = lds_u32(tb + (kv[j] >> 16));
        if (c == 15 && j == 3) e1 = cg ? 0u : e1;
        const uint32_t q0 = (e0 * ahi + __umulhi(e0, alo)) >> 8;
        const uint32_t q1 = (e1 * ahi + __umulhi(e1, alo)) >> 8;
        tot += q0 + q1;
        fw[j] = (q0 | (q1 << 16)) + 0x00010001u;
      }
      row4[c] = make_uint4(fw[0], fw[1], fw[2], fw[3]);
    }
    sXa[g][cg][erow] = tot;
    group_sync(g);
    const uint32_t tot_o = sXa[g][cg ^ 1][erow];
    const uint32_t R = kQScale - (tot + tot_o);  // the remainder, taken by the first maximum
    {
      const int fl = first - 128 * cg;
      if (fl >= 0 && fl < 128) {
        row16[fl] = (uint16_t)(row16[fl] + R);
      }
    }
    // 1 + q summed over half 0 (and R once the first maximum lies there)
    const uint32_t base = cg ? 128u + tot_o + (first < 128 ? R : 0u) : 0u;
    if (mode == kPredCdf) {
      // ---- pass 4: C_{s+1} = base + f_0 + ... + f_s two at a time, in
      // place: with w = f_s | f_{s+1} << 16 and run in both halves,
      // w 65537 + run = C_{s+1} | C_{s+2} << 16 (no carry leaves the low half
      // below 2^16); entries 254 and 255 hold 0xFFFF
      uint32_t runp = base * 0x10001u;
#pragma unroll 4
      for (int c = 0; c < 16; c++) {
        const uint4 f4 = row4[c];
        const uint32_t fv[4] = {f4.x, f4.y, f4.z, f4.w};
        uint32_t cw[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
          cw[j] = fv[j] * 0x10001u + runp;
          runp = __byte_perm(cw[j], 0, 0x3232);
        }
        if (c == 15 && cg) cw[3] = 0xFFFFFFFFu;
        row4[c] = make_uint4(cw[0], cw[1], cw[2], cw[3]);
      }
      group_sync(g);
      // the tile's rows leave coalesced: a warp copies 16 rows, 512 B each
#pragma unroll 4
      for (int k = 0; k < kPTile / 8; k++) {
        const int tr = wl * (kPTile / 8) + k;
        if (r0 + tr < n)
          reinterpret_cast<uint4*>(cdf + (r0 + tr) * 256)[lane] =
              *reinterpret_cast<const uint4*>(sLg + tr * kLogStride + 16 * lane);
      }
    } else if (r < n) {
      // the encoder's (C_s, f_s): C_s = base + the f of this half before s;
      // any 254 or fewer f sum below 2^16, so words add with their halves
      // apart
      const int sl = (int)codes[r] - 1 - 128 * cg;
      if (sl >= 0 && sl < 128) {
        uint32_t acc = 0;
        for (int c = 0; c < (sl >> 3); c++) {
          const uint4 f4 = row4[c];
          acc += f4.x + f4.y + f4.z + f4.w;
        }
        uint32_t cs = base + (acc & 0xFFFFu) + (acc >> 16);
        for (int k = sl & ~7; k < sl; k++) cs += row16[k];
        const uint32_t fs = row16[sl];
        enc[r] = cs | (fs << 16);
      }
    }
  }
  if (!ok) {
    if (tl == 0) atomicExch(&g_pred_error, 1);
    tc::mbar_wait(mbar, phase ^ 1);  // an MMA still in flight lands first
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (w == 0) tc::tmem_dealloc(tslot, 512);
}

}  // namespace

void pack_pred_tc_weights(const int8_t* W, int rows, int rows_total, uint16_t* img) {
  unsigned char* p = reinterpret_cast<unsigned char*>(img);
  for (int i = 0; i < rows_total * 64; i++) p[i] = 0;
  for (int r = 0; r < rows; r++)
    for (int k = 0; k < 32; k++) {
      const __nv_bfloat16 b = __float2bfloat16_rn((float)W[(size_t)r * 32 + k]);
      uint32_t off = (uint32_t)(r * 64 + k * 2);
      off ^= ((off >> 7) & 3) << 4;
      memcpy(p + off, &b, 2);
    }
}

int pred_tc_error(bool reset) {
  int e = 0;
  cudaMemcpyFromSymbol(&e, g_pred_error, sizeof(int));
  if (reset && e) {
    const int z = 0;
    cudaMemcpyToSymbol(g_pred_error, &z, sizeof(int));
  }
  return e;
}

void launch_predictor(const DLayer& P1, const DPred2& P2, const uint32_t* lut, const int8_t* F,
                      int f_stride, const int64_t* d_n, int64_t n_host, int mode,
                      const uint8_t* codes, uint16_t* cdf, uint32_t* enc, int8_t* logits,
                      cudaStream_t st, int variant) {
  if (n_host <= 0) return;
  if (variant == 1 && P1.Wtc && P2.Wtc) {
    const int64_t ntiles = (n_host + kPTile - 1) / kPTile;
    const int blocks = (int)std::min<int64_t>((ntiles + 1) / 2, 148);  // two groups a CTA
    cudaFuncSetAttribute(k_predictor_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kPredSmem);
    k_predictor_tc<<<blocks, kPThreads, kPredSmem, st>>>(P1, P2, lut, F, f_stride, d_n, mode,
                                                           codes, cdf, enc, logits);
  } else {
    const int blocks = (int)std::min<int64_t>((n_host + kWarps - 1) / kWarps, kBlocksRow);
    k_predictor_dp4a<<<blocks, kWarps * 32, 0, st>>>(P1, P2, lut, F, f_stride, d_n, mode, codes,
                                                     cdf, enc, logits);
  }
  count_launches(1);
}

}  // namespace lpc
