// Predictor and rate loss of the differentiable twin, fused: the two linear
// layers of the predictor (Eq. 7: C -> C with PReLU, then C -> 255 logits),
// the fake quantisers of its two inputs (Eq. 12, straight-through), the
// log-softmax over the 255 occupancy symbols and the cross-entropy of the
// true symbol in bits (supplement, Training, Eq. 16), in one kernel; the
// backward recomputes the forward row by row and produces every gradient
// (input features, both weights, biases and the PReLU slope) without writing
// the [N x 255] logits or their gradients to memory.
//
// Layout: one warp takes R rows at a time.  Lane j holds channel j of a row
// (features, hidden units) and the logits j, j + 32, ..., j + 224 of every
// row (entry 255 is padding).  Weights live in shared memory with a row
// stride of 33 floats, so that both the forward (lanes over outputs) and
// the backward (lanes over inputs) read them without bank conflicts.  The
// backward stages the logit gradients and the layer inputs of the block's
// rows in shared memory, and each thread accumulates a tile of the weight
// gradients in registers (dW2 row o = thread o, dW1 four entries a thread);
// the block adds its partial sums to the caller's gradients once at the end.
// bf16 = 1 rounds both operands of every product to bf16 (the gradient of a
// product's output is not rounded, as in a linear layer's backward on
// rounded operands); accumulation is float32.
#include <cuda_bf16.h>

#include <algorithm>

#include "../../include/lpc.h"
#include "../../include/lpc_train.h"
#include "common.cuh"
#include "kernels.h"

namespace lpc {
namespace {

constexpr int kC = 32;        // channels
constexpr int kNS = 255;      // occupancy symbols
constexpr int kOut = 8;       // logits per lane (256 / 32)
constexpr int kR = 4;         // rows per warp per round
constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kLd = kC + 1;   // shared-memory row stride of the weights
constexpr float kInvLn2 = 1.4426950408889634f;
constexpr float kActScale = 1.0f / 32.0f;  // fake-quantiser scale, zero point 0

struct PredArgs {
  const float* F;
  int64_t N;
  const float *W1, *b1, *a1, *W2, *b2;
  const uint8_t* codes;
  int qat, bf16;
  float* logits;
  double* bits;
  const float* dbits;
  float *dF, *dW1, *db1, *da1, *dW2, *db2;
};

__device__ __forceinline__ float rnd(float v, int bf16) {
  return bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
}

// fake quantisation at scale 1/32, zero point 0 (the same rounding as the
// stand-alone quantiser); *pass = the clip is inactive (straight-through)
__device__ __forceinline__ float fq(float x, bool* pass) {
  const float r = rintf(x / kActScale);
  const float c = fminf(fmaxf(r, -128.f), 127.f);
  *pass = r >= -128.f && r <= 127.f;
  return c * kActScale;
}

struct Smem {
  float W2[256 * kLd];  // [o][k], row 255 zero
  float W1[kC * kLd];   // [j][k]
  float b2[256];
  float b1[kC], a1[kC];
  // backward staging, per warp and row
  float dl[kWarps][kR][256];
  float hq[kWarps][kR][kC];
  float xq[kWarps][kR][kC];
  float dz[kWarps][kR][kC];
  double red[kWarps];
};

template <bool BWD>
__global__ void __launch_bounds__(kThreads)
k_pred(PredArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Smem& s = *reinterpret_cast<Smem*>(smraw);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 256 * kC; i += kThreads) {
    const int o = i / kC, k = i % kC;
    s.W2[o * kLd + k] = o < kNS ? rnd(a.W2[o * kC + k], a.bf16) : 0.f;
  }
  for (int i = tid; i < kC * kC; i += kThreads)
    s.W1[(i / kC) * kLd + i % kC] = rnd(a.W1[i], a.bf16);
  for (int i = tid; i < 256; i += kThreads) s.b2[i] = i < kNS ? a.b2[i] : 0.f;
  if (tid < kC) {
    s.b1[tid] = a.b1[tid];
    s.a1[tid] = a.a1[tid];
  }
  __syncthreads();
  const float gs = BWD ? a.dbits[0] * kInvLn2 : 0.f;
  // backward partial sums: thread o's row of dW2 and db2, four entries of
  // dW1, lane j's db1 and da1
  float gW2[kC], gb2 = 0.f, gW1[4] = {0.f, 0.f, 0.f, 0.f}, gb1 = 0.f, ga1 = 0.f;
#pragma unroll
  for (int k = 0; k < kC; k++) gW2[k] = 0.f;
  double loss = 0.0;

  const int64_t per_round = (int64_t)gridDim.x * kWarps * kR;
  const int64_t rounds = (a.N + per_round - 1) / per_round;
  for (int64_t rd = 0; rd < rounds; rd++) {
    const int64_t row0 = rd * per_round + ((int64_t)blockIdx.x * kWarps + w) * kR;
    // ---- forward, kR rows: lane k holds input channel k
    float x[kR], z1[kR], hq[kR];
    bool xpass[kR], hpass[kR];
    int y[kR];
#pragma unroll
    for (int r = 0; r < kR; r++) {
      const int64_t row = row0 + r;
      const bool ok = row < a.N;
      const float f = ok ? a.F[row * kC + lane] : 0.f;
      x[r] = a.qat ? fq(f, &xpass[r]) : f;
      if (!a.qat) xpass[r] = true;
      x[r] = rnd(x[r], a.bf16);
      y[r] = ok ? (int)a.codes[row] - 1 : -1;
    }
    // hidden layer: lane j = output j
#pragma unroll
    for (int r = 0; r < kR; r++) z1[r] = s.b1[lane];
#pragma unroll 8
    for (int k = 0; k < kC; k++) {
      const float wjk = s.W1[lane * kLd + k];
#pragma unroll
      for (int r = 0; r < kR; r++) z1[r] = fmaf(wjk, __shfl_sync(0xffffffffu, x[r], k), z1[r]);
    }
#pragma unroll
    for (int r = 0; r < kR; r++) {
      const float h = z1[r] >= 0.f ? z1[r] : s.a1[lane] * z1[r];
      hq[r] = a.qat ? fq(h, &hpass[r]) : h;
      if (!a.qat) hpass[r] = true;
      hq[r] = rnd(hq[r], a.bf16);
    }
    // logits: lane j = outputs j + 32 m
    float lg[kR][kOut];
#pragma unroll
    for (int m = 0; m < kOut; m++)
#pragma unroll
      for (int r = 0; r < kR; r++) lg[r][m] = s.b2[lane + 32 * m];
#pragma unroll 4
    for (int k = 0; k < kC; k++) {
      float hk[kR];
#pragma unroll
      for (int r = 0; r < kR; r++) hk[r] = __shfl_sync(0xffffffffu, hq[r], k);
#pragma unroll
      for (int m = 0; m < kOut; m++) {
        const float wok = s.W2[(lane + 32 * m) * kLd + k];
#pragma unroll
        for (int r = 0; r < kR; r++) lg[r][m] = fmaf(wok, hk[r], lg[r][m]);
      }
    }
    // log-softmax over the 255 real entries and the true symbol's term
    float lse[kR];
#pragma unroll
    for (int r = 0; r < kR; r++) {
      float mx = -INFINITY;
#pragma unroll
      for (int m = 0; m < kOut; m++)
        if (lane + 32 * m < kNS) mx = fmaxf(mx, lg[r][m]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      float se = 0.f;
#pragma unroll
      for (int m = 0; m < kOut; m++)
        if (lane + 32 * m < kNS) se += __expf(lg[r][m] - mx);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
      lse[r] = mx + __logf(se);
      const int yr = y[r] < 0 ? 0 : y[r];
      float ly = 0.f;
#pragma unroll
      for (int m = 0; m < kOut; m++)
        if (m == (yr >> 5)) ly = lg[r][m];
      ly = __shfl_sync(0xffffffffu, ly, yr & 31);
      if (!BWD && lane == 0 && y[r] >= 0) loss += (double)(lse[r] - ly);
      if (!BWD && a.logits && y[r] >= 0) {
        float* dst = a.logits + (row0 + r) * kNS;
#pragma unroll
        for (int m = 0; m < kOut; m++)
          if (lane + 32 * m < kNS) dst[lane + 32 * m] = lg[r][m];
      }
    }
    if (!BWD) continue;

    // ---- backward: dlogits = (softmax - onehot) * dbits / ln 2
#pragma unroll
    for (int r = 0; r < kR; r++) {
#pragma unroll
      for (int m = 0; m < kOut; m++) {
        const int o = lane + 32 * m;
        float d = 0.f;
        if (o < kNS && y[r] >= 0) d = gs * (__expf(lg[r][m] - lse[r]) - (o == y[r] ? 1.f : 0.f));
        s.dl[w][r][o] = d;
      }
      s.hq[w][r][lane] = y[r] >= 0 ? hq[r] : 0.f;
      s.xq[w][r][lane] = y[r] >= 0 ? x[r] : 0.f;
    }
    __syncwarp();
    // dhq = W2^T dl: lane k over the 255 outputs
    float dh[kR];
#pragma unroll
    for (int r = 0; r < kR; r++) dh[r] = 0.f;
#pragma unroll 2
    for (int o = 0; o < 256; o += 4) {
      const float w0 = s.W2[(o + 0) * kLd + lane], w1 = s.W2[(o + 1) * kLd + lane];
      const float w2 = s.W2[(o + 2) * kLd + lane], w3 = s.W2[(o + 3) * kLd + lane];
#pragma unroll
      for (int r = 0; r < kR; r++) {
        const float4 d = *reinterpret_cast<const float4*>(&s.dl[w][r][o]);
        dh[r] = fmaf(w0, d.x, fmaf(w1, d.y, fmaf(w2, d.z, fmaf(w3, d.w, dh[r]))));
      }
    }
    // through the quantiser (straight-through) and the PReLU: lane j
    float dz[kR];
#pragma unroll
    for (int r = 0; r < kR; r++) {
      const float g = hpass[r] ? dh[r] : 0.f;
      const bool neg = z1[r] < 0.f;
      dz[r] = neg ? s.a1[lane] * g : g;
      if (y[r] >= 0) {
        if (neg) ga1 = fmaf(g, z1[r], ga1);
        gb1 += dz[r];
      } else {
        dz[r] = 0.f;
      }
      s.dz[w][r][lane] = dz[r];
    }
    // dx = W1^T dz: lane k over the 32 hidden units
    float dx[kR];
#pragma unroll
    for (int r = 0; r < kR; r++) dx[r] = 0.f;
#pragma unroll 8
    for (int j = 0; j < kC; j++) {
      const float wjk = s.W1[j * kLd + lane];
#pragma unroll
      for (int r = 0; r < kR; r++) dx[r] = fmaf(wjk, __shfl_sync(0xffffffffu, dz[r], j), dx[r]);
    }
#pragma unroll
    for (int r = 0; r < kR; r++) {
      const int64_t row = row0 + r;
      if (row < a.N && a.dF) a.dF[row * kC + lane] = xpass[r] ? dx[r] : 0.f;
    }
    __syncthreads();
    // weight gradients over the block's rows: thread o, dW2[o][:] and db2[o]
    {
      const int o = tid;
#pragma unroll 1
      for (int ww = 0; ww < kWarps; ww++)
#pragma unroll
        for (int r = 0; r < kR; r++) {
          const float d = s.dl[ww][r][o];
          gb2 += d;
#pragma unroll
          for (int k = 0; k < kC; k += 4) {
            const float4 h4 = *reinterpret_cast<const float4*>(&s.hq[ww][r][k]);
            gW2[k] = fmaf(d, h4.x, gW2[k]);
            gW2[k + 1] = fmaf(d, h4.y, gW2[k + 1]);
            gW2[k + 2] = fmaf(d, h4.z, gW2[k + 2]);
            gW2[k + 3] = fmaf(d, h4.w, gW2[k + 3]);
          }
        }
      // dW1[j][k0..k0+3], j = tid / 8, k0 = 4 (tid % 8)
      const int j = tid >> 3, k0 = (tid & 7) * 4;
#pragma unroll 1
      for (int ww = 0; ww < kWarps; ww++)
#pragma unroll
        for (int r = 0; r < kR; r++) {
          const float d = s.dz[ww][r][j];
          const float4 x4 = *reinterpret_cast<const float4*>(&s.xq[ww][r][k0]);
          gW1[0] = fmaf(d, x4.x, gW1[0]);
          gW1[1] = fmaf(d, x4.y, gW1[1]);
          gW1[2] = fmaf(d, x4.z, gW1[2]);
          gW1[3] = fmaf(d, x4.w, gW1[3]);
        }
    }
    __syncthreads();
  }

  if (!BWD) {
    if (lane == 0) s.red[w] = loss;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < kWarps; i++) t += s.red[i];
      atomicAdd(a.bits, t * (double)kInvLn2);
    }
    return;
  }
  // the block's partial gradients into the caller's
  if (tid < kNS) {
#pragma unroll
    for (int k = 0; k < kC; k++) atomicAdd(a.dW2 + tid * kC + k, gW2[k]);
    atomicAdd(a.db2 + tid, gb2);
  }
  {
    const int j = tid >> 3, k0 = (tid & 7) * 4;
#pragma unroll
    for (int i = 0; i < 4; i++) atomicAdd(a.dW1 + j * kC + k0 + i, gW1[i]);
  }
  // db1, da1: lane j of every warp
  __shared__ float sb1[kWarps][kC], sa1[kWarps][kC];
  sb1[w][lane] = gb1;
  sa1[w][lane] = ga1;
  __syncthreads();
  if (tid < kC) {
    float b = 0.f, c = 0.f;
    for (int i = 0; i < kWarps; i++) {
      b += sb1[i][tid];
      c += sa1[i][tid];
    }
    atomicAdd(a.db1 + tid, b);
    atomicAdd(a.da1 + tid, c);
  }
}

int pred_grid(int64_t N) {
  const int64_t need = (N + kWarps * kR - 1) / (kWarps * kR);
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, 148 * 2));
}

int launch_pred(bool bwd, const PredArgs& a, cudaStream_t st) {
  const size_t smem = sizeof(Smem);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_pred<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_pred<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  if (bwd)
    k_pred<true><<<pred_grid(a.N), kThreads, smem, st>>>(a);
  else
    k_pred<false><<<pred_grid(a.N), kThreads, smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? LPC_OK : LPC_CUDA_ERROR;
}

}  // namespace
}  // namespace lpc

using namespace lpc;

extern "C" {

int lpc_t_pred_fwd(const float* F, int64_t N, const float* W1, const float* b1, const float* a1,
                   const float* W2, const float* b2, const uint8_t* codes, int qat, int bf16,
                   float* logits, double* bits, uint64_t stream) {
  if (N < 0 || !bits || (N > 0 && (!F || !W1 || !b1 || !a1 || !W2 || !b2 || !codes)))
    return LPC_INVALID_ARG;
  if (N == 0) return LPC_OK;
  PredArgs a{F, N, W1, b1, a1, W2, b2, codes, qat, bf16, logits, bits, nullptr,
             nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  return launch_pred(false, a, reinterpret_cast<cudaStream_t>(stream));
}

int lpc_t_pred_bwd(const float* F, int64_t N, const float* W1, const float* b1, const float* a1,
                   const float* W2, const float* b2, const uint8_t* codes, int qat, int bf16,
                   const float* dbits, float* dF, float* dW1, float* db1, float* da1, float* dW2,
                   float* db2, uint64_t stream) {
  if (N < 0 || !dbits || !dW1 || !db1 || !da1 || !dW2 || !db2 ||
      (N > 0 && (!F || !W1 || !b1 || !a1 || !W2 || !b2 || !codes)))
    return LPC_INVALID_ARG;
  if (N == 0) return LPC_OK;
  PredArgs a{F, N, W1, b1, a1, W2, b2, codes, qat, bf16, nullptr, nullptr, dbits,
             dF, dW1, db1, da1, dW2, db2};
  return launch_pred(true, a, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
