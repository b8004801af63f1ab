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
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

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
struct SmemLayer {
  int32_t* W;
  int32_t* wsum;
  int32_t* bias;
  int32_t* mult;
  int32_t* slope;
};

__device__ __forceinline__ SmemLayer stage_layer(const DLayer& L, int32_t* sm) {
  const int nw = L.S * (L.cin / 4) * 32;
  const int P = L.per_slice ? L.S : 1;
  SmemLayer s;
  s.W = sm;
  s.wsum = s.W + nw;
  s.bias = s.wsum + L.S * 32;
  s.mult = s.bias + P * 32;
  s.slope = s.mult + P * 32;
  for (int i = threadIdx.x; i < nw; i += blockDim.x) s.W[i] = L.Wp[i];
  for (int i = threadIdx.x; i < L.S * 32; i += blockDim.x) s.wsum[i] = L.wsum[i];
  for (int i = threadIdx.x; i < P * 32; i += blockDim.x) {
    s.bias[i] = L.bias[i];
    s.mult[i] = L.mult[i];
    s.slope[i] = L.slope[i];
  }
  return s;
}

static size_t smem_layer_bytes(const DLayer& L) {
  const int P = L.per_slice ? L.S : 1;
  return sizeof(int32_t) * ((size_t)L.S * (L.cin / 4) * 32 + (size_t)L.S * 32 + 3 * (size_t)P * 32);
}

template <int CIN>
__device__ __forceinline__ int32_t dot_slice(const int32_t (&x)[CIN / 4], const int32_t* W,
                                             int slice, int lane, int32_t acc) {
  const int32_t* w = W + slice * (CIN / 4) * 32 + lane;
#pragma unroll
  for (int k = 0; k < CIN / 4; k++) acc = __dp4a(x[k], w[k * 32], acc);
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
template <int CIN>
__global__ void __launch_bounds__(kWarps * 32)
k_up_prune(DLayer L, const uint64_t* __restrict__ ckey, const uint32_t* __restrict__ cpar,
           const int64_t* d_nc, const int8_t* __restrict__ x, int x_stride, int8_t* out,
           int out_stride, int out_col) {
  extern __shared__ int32_t sm[];
  const SmemLayer s = stage_layer(L, sm);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t n = *d_nc;
  for (int64_t r = warp_id_global(); r < n; r += warps_total()) {
    const uint32_t p = cpar[r];
    const int c = (int)(ckey[r] & 7);
    int32_t xv[CIN / 4];
    load_row<CIN>(x + (int64_t)p * x_stride, xv);
    int32_t acc = s.bias[c * 32 + lane] - L.z_in * s.wsum[c * 32 + lane];
    acc = dot_slice<CIN>(xv, s.W, c, lane, acc);
    if (L.prelu) acc = prelu(acc, s.slope[c * 32 + lane]);
    out[r * out_stride + out_col + lane] = (int8_t)requant(acc, s.mult[c * 32 + lane], L.shift,
                                                           L.z_out);
  }
}

void launch_up_prune(const DLayer& W, const uint64_t* ckey, const uint32_t* cpar,
                     const int64_t* d_nc, int64_t nc_host, const int8_t* x, int x_stride,
                     int8_t* out, int out_stride, int out_col, cudaStream_t st) {
  if (nc_host <= 0) return;
  const size_t smem = smem_layer_bytes(W);
  const int blocks = (int)std::min<int64_t>((nc_host + kWarps - 1) / kWarps, kBlocksRow);
  if (W.cin == 32)
    k_up_prune<32><<<blocks, kWarps * 32, smem, st>>>(W, ckey, cpar, d_nc, x, x_stride, out,
                                                      out_stride, out_col);
  else
    k_up_prune<64><<<blocks, kWarps * 32, smem, st>>>(W, ckey, cpar, d_nc, x, x_stride, out,
                                                      out_stride, out_col);
  count_launches(1);
}

// ------------------------------------------------------------ down (s2) --
template <int CIN>
__global__ void __launch_bounds__(kWarps * 32)
k_down(DLayer L, const uint64_t* __restrict__ ckey, const uint32_t* __restrict__ poff,
       const int64_t* d_np, const int8_t* __restrict__ x, int x_stride, int8_t* out,
       int out_stride, int out_col) {
  extern __shared__ int32_t sm[];
  const SmemLayer s = stage_layer(L, sm);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t n = *d_np;
  for (int64_t p = warp_id_global(); p < n; p += warps_total()) {
    int32_t acc = s.bias[lane];
    const uint32_t r0 = poff[p], r1 = poff[p + 1];
    for (uint32_t r = r0; r < r1; r++) {
      const int c = (int)(ckey[r] & 7);
      int32_t xv[CIN / 4];
      load_row<CIN>(x + (int64_t)r * x_stride, xv);
      acc -= L.z_in * s.wsum[c * 32 + lane];
      acc = dot_slice<CIN>(xv, s.W, c, lane, acc);
    }
    if (L.prelu) acc = prelu(acc, s.slope[lane]);
    out[p * out_stride + out_col + lane] = (int8_t)requant(acc, s.mult[lane], L.shift, L.z_out);
  }
}

void launch_down(const DLayer& W, const uint64_t* ckey, const uint32_t* poff, const int64_t* d_np,
                 int64_t np_host, const int8_t* x, int x_stride, int8_t* out, int out_stride,
                 int out_col, cudaStream_t st) {
  if (np_host <= 0) return;
  const size_t smem = smem_layer_bytes(W);
  const int blocks = (int)std::min<int64_t>((np_host + kWarps - 1) / kWarps, kBlocksRow);
  if (W.cin == 32)
    k_down<32><<<blocks, kWarps * 32, smem, st>>>(W, ckey, poff, d_np, x, x_stride, out,
                                                  out_stride, out_col);
  else
    k_down<64><<<blocks, kWarps * 32, smem, st>>>(W, ckey, poff, d_np, x, x_stride, out,
                                                  out_stride, out_col);
  count_launches(1);
}

// ------------------------------------------- integer softmax -> CDF row --
// Lane l holds symbols s = 8l + i, i = 0..7; symbol 255 (lane 31, i = 7) is
// not a class and takes no frequency.
//   M = max l_s; e_s = lut[M - l_s]; S = sum e_s (< 2^24);
//   f_s = 1 + floor(e_s (2^16 - 255) / S)  (the product fits in 32 bits);
//   the remainder 2^16 - sum f_s goes to the lowest s with l_s = M.
// The 255 divisions by the row's S share one reciprocal: with
// inv = floor((2^32 - 1) / S), q = umulhi(x, inv) is floor(x / S) or at most
// two less (x < 2^32), and two conditional corrections make it exact.
__device__ __forceinline__ uint32_t div_by(uint32_t x, uint32_t S, uint32_t inv) {
  uint32_t q = __umulhi(x, inv);
  uint32_t r = x - q * S;
  if (r >= S) {
    q++;
    r -= S;
  }
  if (r >= S) q++;
  return q;
}

__device__ __forceinline__ void softmax_freq(const int (&l)[8], const uint32_t* slut, int lane,
                                             uint32_t (&f)[8]) {
  int mx = -1000;
#pragma unroll
  for (int i = 0; i < 8; i++)
    if (lane * 8 + i < kNsym) mx = max(mx, l[i]);
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  uint32_t e[8];
  uint32_t S = 0;
  int first = 1 << 20;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const bool v = lane * 8 + i < kNsym;
    e[i] = v ? slut[mx - l[i]] : 0u;
    S += e[i];
    if (v && l[i] == mx && first == (1 << 20)) first = lane * 8 + i;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    S += __shfl_xor_sync(0xffffffffu, S, o);
    first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
  }
  uint32_t tot = 0;
  const uint32_t inv = 0xFFFFFFFFu / S;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    f[i] = lane * 8 + i < kNsym ? 1u + div_by(e[i] * (uint32_t)(kFreqTotal - kNsym), S, inv) : 0u;
    tot += f[i];
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
  if ((first >> 3) == lane) {
#pragma unroll
    for (int i = 0; i < 8; i++)
      if (lane * 8 + i == first) f[i] += (uint32_t)kFreqTotal - tot;
  }
}

// Inclusive cumulative values c[i] = C_{s+1} for s = 8 lane + i.
__device__ __forceinline__ void cumulate(const uint32_t (&f)[8], int lane, uint32_t (&c)[8]) {
  uint32_t run = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    run += f[i];
    c[i] = run;
  }
  uint32_t x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  const uint32_t ex = x - run;
#pragma unroll
  for (int i = 0; i < 8; i++) c[i] += ex;
}

__device__ __forceinline__ void store_cdf_row(const uint32_t (&c)[8], int lane, uint16_t* row) {
  uint32_t h[8];
#pragma unroll
  for (int i = 0; i < 8; i++) h[i] = (lane * 8 + i <= 253) ? c[i] : 0xFFFFu;
  uint4 v;
  v.x = h[0] | (h[1] << 16);
  v.y = h[2] | (h[3] << 16);
  v.z = h[4] | (h[5] << 16);
  v.w = h[6] | (h[7] << 16);
  reinterpret_cast<uint4*>(row)[lane] = v;
}

__global__ void __launch_bounds__(kWarps * 32)
k_softmax_cdf(const int8_t* __restrict__ logits, int64_t n, const uint32_t* __restrict__ lut,
              uint16_t* cdf) {
  __shared__ uint32_t slut[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) slut[i] = lut[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int64_t r = warp_id_global(); r < n; r += warps_total()) {
    int l[8];
#pragma unroll
    for (int i = 0; i < 8; i++) l[i] = lane * 8 + i < kNsym ? logits[r * kNsym + lane * 8 + i] : 0;
    uint32_t f[8], c[8];
    softmax_freq(l, slut, lane, f);
    cumulate(f, lane, c);
    store_cdf_row(c, lane, cdf + r * 256);
  }
}

void launch_softmax_cdf(const int8_t* logits, int64_t n, const uint32_t* lut, uint16_t* cdf,
                        cudaStream_t st) {
  if (n <= 0) return;
  const int blocks = (int)std::min<int64_t>((n + kWarps - 1) / kWarps, kBlocksRow);
  k_softmax_cdf<<<blocks, kWarps * 32, 0, st>>>(logits, n, lut, cdf);
  count_launches(1);
}

// ------------------------------------------- predictor + softmax + CDF --
// h = requant(prelu(W1 (F - z1) + b1)) (C -> C), logits = requant(W2 (h - z2)
// + b2) (C -> 255), then the integer softmax.  Modes: full CDF row, the
// (C_s, f_s) pair of the true symbol (encoder), or the logits (debug).
__global__ void __launch_bounds__(kWarps * 32)
k_predictor(DLayer P1, DPred2 P2, const uint32_t* __restrict__ lut,
            const int8_t* __restrict__ F, int f_stride, const int64_t* d_n, int mode,
            const uint8_t* __restrict__ codes, uint16_t* cdf, uint32_t* enc, int8_t* logits) {
  __shared__ int32_t sW1[8 * 32], sW1s[32], sB1[32], sM1[32], sS1[32];
  __shared__ int32_t sW2[8 * 8 * 32];
  __shared__ int32_t sW2s[256], sB2[256], sM2[256];
  __shared__ uint32_t slut[256];
  __shared__ int32_t hbuf[kWarps][8];
  for (int i = threadIdx.x; i < 8 * 32; i += blockDim.x) sW1[i] = P1.Wp[i];
  for (int i = threadIdx.x; i < 8 * 8 * 32; i += blockDim.x) sW2[i] = P2.Wp[i];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    sW2s[i] = P2.wsum[i];
    sB2[i] = P2.bias[i];
    sM2[i] = P2.mult[i];
    slut[i] = lut[i];
  }
  for (int i = threadIdx.x; i < 32; i += blockDim.x) {
    sW1s[i] = P1.wsum[i];
    sB1[i] = P1.bias[i];
    sM1[i] = P1.mult[i];
    sS1[i] = P1.slope[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
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
      l[i] = requant(acc, sM2[sidx], P2.shift, P2.z_out);
    }
    if (mode == kPredLogits) {
#pragma unroll
      for (int i = 0; i < 8; i++)
        if (lane * 8 + i < kNsym) logits[r * kNsym + lane * 8 + i] = (int8_t)l[i];
      continue;
    }
    uint32_t f[8], c[8];
    softmax_freq(l, slut, lane, f);
    cumulate(f, lane, c);
    if (mode == kPredCdf) {
      store_cdf_row(c, lane, cdf + r * 256);
    } else {
      const int s = (int)codes[r] - 1;
      if ((s >> 3) == lane) {
        const int i = s & 7;
        uint32_t fs = 0, cs = 0;
#pragma unroll
        for (int k = 0; k < 8; k++)
          if (k == i) {
            fs = f[k];
            cs = c[k] - f[k];
          }
        enc[r] = cs | (fs << 16);
      }
    }
  }
}

void launch_predictor(const DLayer& P1, const DPred2& P2, const uint32_t* lut, const int8_t* F,
                      int f_stride, const int64_t* d_n, int64_t n_host, int mode,
                      const uint8_t* codes, uint16_t* cdf, uint32_t* enc, int8_t* logits,
                      cudaStream_t st) {
  if (n_host <= 0) return;
  const int blocks = (int)std::min<int64_t>((n_host + kWarps - 1) / kWarps, kBlocksRow);
  k_predictor<<<blocks, kWarps * 32, 0, st>>>(P1, P2, lut, F, f_stride, d_n, mode, codes, cdf,
                                              enc, logits);
  count_launches(1);
}

}  // namespace lpc
