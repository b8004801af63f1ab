// Differentiable (quantisation-aware) twin of the network ops, forward and
// hand-written backward, float32 with an optional bf16 rounding of every
// product operand (fp32 accumulation).  Two generic kernels cover the sparse
// ops:
//  - k_gmv: out[row] = (bias) + sum over the row's items (slice s, source
//    row r) of Wsl[s] in[r], one warp per output row, the weight tensor in
//    shared memory laid out [slice][k][j] so that lane j reads consecutive
//    words.  Forward of conv / up / down and their input gradients (through
//    the mirrored index structure) are instances.
//  - k_outer: dW[s] += sum over rows of dy[a(row)] x[b(row)]^T for the rows
//    whose item belongs to slice s: the weight gradients.
#include <cuda_bf16.h>

#include <algorithm>

#include "../../include/lpc.h"
#include "../../include/lpc_train.h"
#include "common.cuh"
#include "kernels.h"

namespace lpc {
namespace {

__device__ __forceinline__ float rnd(float v, int bf16) {
  return bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
}

constexpr int kWarpsT = 8;

// ---- index structures as item visitors --------------------------------------
// conv forward: row i, items (o, nbr[i][o]); backward dx: (o, nbr[i][26 - o])
struct ConvItems {
  const int32_t* nbr;
  int mirror;
  template <class F>
  __device__ void visit(int64_t i, F f) const {
    for (int o = 0; o < 27; o++) {
      const int32_t r = nbr[i * 27 + (mirror ? 26 - o : o)];
      if (r >= 0) f(o, (int64_t)r);
    }
  }
};
// up forward: child row r, one item (c_r, par[r])
struct UpFwdItems {
  const uint32_t* par;
  const uint64_t* ckey;
  template <class F>
  __device__ void visit(int64_t r, F f) const {
    f((int)(ckey[r] & 7), (int64_t)par[r]);
  }
};
// up backward dx / down forward: parent row p, items (c_r, r) over children
struct ChildItems {
  const uint32_t* off;
  const uint64_t* ckey;
  template <class F>
  __device__ void visit(int64_t p, F f) const {
    for (uint32_t r = off[p]; r < off[p + 1]; r++) f((int)(ckey[r] & 7), (int64_t)r);
  }
};

template <int OUT, int IN, class Items>
__global__ void __launch_bounds__(kWarpsT * 32)
k_gmv(Items items, const float* __restrict__ W, int S, int transpose,
      const float* __restrict__ bias, int bias_mode, const float* __restrict__ in, int64_t rows,
      float* __restrict__ out, int bf16) {
  extern __shared__ float sW[];  // [S][IN][OUT]
  const int n = S * IN * OUT;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int s = idx / (IN * OUT), rem = idx % (IN * OUT), k = rem / OUT, j = rem % OUT;
    // W is [S][cout][cin]; forward: k = cin, j = cout; transpose: k = cout, j = cin
    const float w = transpose ? W[((size_t)s * IN + k) * OUT + j] : W[((size_t)s * OUT + j) * IN + k];
    sW[idx] = rnd(w, bf16);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * kWarpsT;
  for (int64_t row = (int64_t)blockIdx.x * kWarpsT + (threadIdx.x >> 5); row < rows;
       row += warps) {
    float acc[OUT / 32];
#pragma unroll
    for (int q = 0; q < OUT / 32; q++) acc[q] = bias_mode == 1 ? bias[lane + 32 * q] : 0.f;
    items.visit(row, [&](int s, int64_t src) {
      const float* w = sW + (size_t)s * IN * OUT + lane;
      const float* x = in + src * IN;
      if (bias_mode == 2) {
#pragma unroll
        for (int q = 0; q < OUT / 32; q++) acc[q] += bias[s * OUT + lane + 32 * q];
      }
      for (int k = 0; k < IN; k++) {
        const float v = rnd(__ldg(x + k), bf16);
#pragma unroll
        for (int q = 0; q < OUT / 32; q++) acc[q] += w[k * OUT + 32 * q] * v;
      }
    });
#pragma unroll
    for (int q = 0; q < OUT / 32; q++) out[row * OUT + lane + 32 * q] = acc[q];
  }
}

// ---- weight gradients ---------------------------------------------------------
// pair(s, row) -> (a, b): dW[s][i][j] += dy[a][i] * x[b][j]; a < 0 skips.
struct ConvPairs {
  const int32_t* nbr;
  __device__ void pair(int s, int64_t row, int64_t& a, int64_t& b) const {
    const int32_t r = nbr[row * 27 + s];
    a = r >= 0 ? row : -1;
    b = r;
  }
};
struct UpPairs {  // rows = children; dy row = child, x row = parent
  const uint32_t* par;
  const uint64_t* ckey;
  __device__ void pair(int s, int64_t row, int64_t& a, int64_t& b) const {
    a = (int)(ckey[row] & 7) == s ? row : -1;
    b = par[row];
  }
};
struct DownPairs {  // rows = children; dy row = parent, x row = child
  const uint32_t* par;
  const uint64_t* ckey;
  __device__ void pair(int s, int64_t row, int64_t& a, int64_t& b) const {
    a = (int)(ckey[row] & 7) == s ? (int64_t)par[row] : -1;
    b = row;
  }
};

constexpr int kOuterRows = 512;  // rows per block
constexpr int kStage = 32;       // rows staged in shared memory at a time

template <int A, int B, class Pairs>
__global__ void __launch_bounds__(256)
k_outer(Pairs pairs, const float* __restrict__ dy, const float* __restrict__ x, int64_t rows,
        float* dW, int bf16) {
  __shared__ float sy[kStage][A];
  __shared__ float sx[kStage][B];
  // every thread a register tile of outputs i = ti + 16 a, j = tj + 16 b,
  // so each staged value it loads feeds several products
  constexpr int NA = A / 16, NB = B / 16;
  const int s = blockIdx.y;
  const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
  float acc[NA][NB];
#pragma unroll
  for (int u = 0; u < NA; u++)
#pragma unroll
    for (int v = 0; v < NB; v++) acc[u][v] = 0.f;
  // the block's rows that contribute to slice s, as (dy row, x row) pairs
  // (absent neighbours and children of other slices take no work)
  __shared__ int64_t pa[kOuterRows], pb[kOuterRows];
  __shared__ int np;
  if (threadIdx.x == 0) np = 0;
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.x * kOuterRows;
  const int64_t r1 = std::min<int64_t>(rows, r0 + kOuterRows);
  for (int64_t row = r0 + threadIdx.x; row < r1; row += 256) {
    int64_t a = -1, b = -1;
    pairs.pair(s, row, a, b);
    if (a >= 0) {
      const int k = atomicAdd(&np, 1);
      pa[k] = a;
      pb[k] = b;
    }
  }
  __syncthreads();
  const int n = np;
  if (n == 0) return;  // nothing of this slice in the block's rows
  for (int base = 0; base < n; base += kStage) {
    for (int idx = threadIdx.x; idx < kStage * (A + B); idx += 256) {
      const int r = idx / (A + B), c = idx % (A + B);
      float v = 0.f;
      if (base + r < n) v = c < A ? dy[pa[base + r] * A + c] : x[pb[base + r] * B + (c - A)];
      if (c < A) sy[r][c] = rnd(v, bf16);
      else sx[r][c - A] = rnd(v, bf16);
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < kStage; r++) {
      float ya[NA], xb[NB];
#pragma unroll
      for (int u = 0; u < NA; u++) ya[u] = sy[r][ti + 16 * u];
#pragma unroll
      for (int v = 0; v < NB; v++) xb[v] = sx[r][tj + 16 * v];
#pragma unroll
      for (int u = 0; u < NA; u++)
#pragma unroll
        for (int v = 0; v < NB; v++) acc[u][v] += ya[u] * xb[v];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < NA; u++)
#pragma unroll
    for (int v = 0; v < NB; v++)
      atomicAdd(dW + (size_t)s * A * B + (size_t)(ti + 16 * u) * B + tj + 16 * v, acc[u][v]);
}

// ---- embedding, PReLU, fake quantisation, bias gradients --------------------
// Row kernels: one warp per row of C channels (lane l holds channels l,
// l + 32, ..., at most kCh of them), kRowIlp rows in flight per warp.  No
// per-element division; PReLU slopes and the per-channel gradient sums stay
// in registers until one shared-memory reduction per block.
constexpr int kCh = 8, kRowIlp = 4, kRowThreads = 256;

struct RowWalk {  // the warp's rows r0, r0 + 1, ... r0 + kRowIlp - 1 per step
  int64_t first, step;
  __device__ RowWalk()
      : first(((blockIdx.x * (int64_t)kRowThreads + threadIdx.x) >> 5) * kRowIlp),
        step((((int64_t)gridDim.x * kRowThreads) >> 5) * kRowIlp) {}
};

__global__ void __launch_bounds__(kRowThreads)
    k_embed_f(const uint8_t* __restrict__ codes, int64_t N, const float* __restrict__ E, int C,
              float* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const RowWalk w;
  for (int64_t r0 = w.first; r0 < N; r0 += w.step) {
    int code[kRowIlp];
#pragma unroll
    for (int u = 0; u < kRowIlp; u++) code[u] = r0 + u < N ? codes[r0 + u] : 0;
#pragma unroll
    for (int u = 0; u < kRowIlp; u++) {
      if (r0 + u >= N) break;
      for (int j = lane; j < C; j += 32) y[(r0 + u) * C + j] = __ldg(E + code[u] * C + j);
    }
  }
}

// dE[code] += dy[row]: with acc_smem, into a block-private [256][C] table in
// shared memory first (the codes of a level are few and skewed: global
// atomics on them serialise), flushed once per block where non-zero.
__global__ void __launch_bounds__(kRowThreads)
    k_embed_b(const uint8_t* __restrict__ codes, int64_t N, const float* __restrict__ dy, int C,
              float* dE, int acc_smem) {
  extern __shared__ float tab[];
  float* acc = acc_smem ? tab : dE;
  if (acc_smem) {
    for (int i = threadIdx.x; i < 256 * C; i += kRowThreads) tab[i] = 0.f;
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const RowWalk w;
  for (int64_t r0 = w.first; r0 < N; r0 += w.step) {
    int code[kRowIlp];
#pragma unroll
    for (int u = 0; u < kRowIlp; u++) code[u] = r0 + u < N ? codes[r0 + u] : 0;
    for (int j = lane; j < C; j += 32) {
      float g[kRowIlp];
#pragma unroll
      for (int u = 0; u < kRowIlp; u++) g[u] = r0 + u < N ? __ldg(dy + (r0 + u) * C + j) : 0.f;
#pragma unroll
      for (int u = 0; u < kRowIlp; u++)
        if (r0 + u < N) atomicAdd(acc + code[u] * C + j, g[u]);
    }
  }
  if (acc_smem) {
    __syncthreads();
    for (int i = threadIdx.x; i < 256 * C; i += kRowThreads)
      if (tab[i] != 0.f) atomicAdd(dE + i, tab[i]);
  }
}

__global__ void __launch_bounds__(kRowThreads)
    k_prelu_f(const float* __restrict__ x, int64_t N, int C, const float* __restrict__ a,
              float* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  float al[kCh];
#pragma unroll
  for (int k = 0; k < kCh; k++) al[k] = lane + 32 * k < C ? a[lane + 32 * k] : 0.f;
  const RowWalk w;
  for (int64_t r0 = w.first; r0 < N; r0 += w.step)
#pragma unroll
    for (int k = 0; k < kCh; k++) {
      const int j = lane + 32 * k;
      if (j >= C) break;
      float v[kRowIlp];
#pragma unroll
      for (int u = 0; u < kRowIlp; u++) v[u] = r0 + u < N ? __ldg(x + (r0 + u) * C + j) : 0.f;
#pragma unroll
      for (int u = 0; u < kRowIlp; u++)
        if (r0 + u < N) y[(r0 + u) * C + j] = v[u] >= 0.f ? v[u] : al[k] * v[u];
    }
}

__global__ void __launch_bounds__(kRowThreads)
    k_prelu_b(const float* __restrict__ x, const float* __restrict__ dy, int64_t N, int C,
              const float* __restrict__ a, float* __restrict__ dx, float* da) {
  __shared__ float part[32 * kCh];
  for (int i = threadIdx.x; i < C; i += kRowThreads) part[i] = 0.f;
  const int lane = threadIdx.x & 31;
  float al[kCh], acc[kCh];
#pragma unroll
  for (int k = 0; k < kCh; k++) {
    al[k] = lane + 32 * k < C ? a[lane + 32 * k] : 0.f;
    acc[k] = 0.f;
  }
  const RowWalk w;
  for (int64_t r0 = w.first; r0 < N; r0 += w.step)
#pragma unroll
    for (int k = 0; k < kCh; k++) {
      const int j = lane + 32 * k;
      if (j >= C) break;
      float v[kRowIlp], g[kRowIlp];
#pragma unroll
      for (int u = 0; u < kRowIlp; u++) {
        v[u] = r0 + u < N ? __ldg(x + (r0 + u) * C + j) : 0.f;
        g[u] = r0 + u < N ? __ldg(dy + (r0 + u) * C + j) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kRowIlp; u++) {
        if (r0 + u >= N) break;
        if (dx) dx[(r0 + u) * C + j] = v[u] >= 0.f ? g[u] : al[k] * g[u];
        if (v[u] < 0.f) acc[k] += g[u] * v[u];
      }
    }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kCh; k++)
    if (lane + 32 * k < C && acc[k] != 0.f) atomicAdd(&part[lane + 32 * k], acc[k]);
  __syncthreads();
  for (int i = threadIdx.x; i < C; i += kRowThreads)
    if (part[i] != 0.f) atomicAdd(da + i, part[i]);
}

// db[slice(row)][j] += dy[row][j]; slice_key = nullptr: one slice (sums kept
// in registers), else the child slot of the row's key (shared-memory sums:
// one row per warp at a time, so the lanes' addresses differ).
__global__ void __launch_bounds__(kRowThreads)
    k_bias_grad(const float* __restrict__ dy, int64_t rows, int C,
                const uint64_t* __restrict__ slice_key, float* db) {
  __shared__ float part[8 * 32 * kCh];
  const int ns = slice_key ? 8 : 1;
  for (int i = threadIdx.x; i < ns * C; i += kRowThreads) part[i] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  float acc[kCh];
#pragma unroll
  for (int k = 0; k < kCh; k++) acc[k] = 0.f;
  const RowWalk w;
  for (int64_t r0 = w.first; r0 < rows; r0 += w.step) {
    int s[kRowIlp];
#pragma unroll
    for (int u = 0; u < kRowIlp; u++)
      s[u] = slice_key && r0 + u < rows ? (int)(slice_key[r0 + u] & 7) : 0;
#pragma unroll
    for (int k = 0; k < kCh; k++) {
      const int j = lane + 32 * k;
      if (j >= C) break;
      float g[kRowIlp];
#pragma unroll
      for (int u = 0; u < kRowIlp; u++) g[u] = r0 + u < rows ? __ldg(dy + (r0 + u) * C + j) : 0.f;
#pragma unroll
      for (int u = 0; u < kRowIlp; u++) {
        if (slice_key) atomicAdd(&part[s[u] * C + j], g[u]);
        else acc[k] += g[u];
      }
    }
  }
  if (!slice_key) {
#pragma unroll
    for (int k = 0; k < kCh; k++)
      if (lane + 32 * k < C && acc[k] != 0.f) atomicAdd(&part[lane + 32 * k], acc[k]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ns * C; i += kRowThreads)
    if (part[i] != 0.f) atomicAdd(db + i, part[i]);
}

// Elementwise kernels: four elements a thread (one 16-byte access) when
// every pointer allows it, the tail and unaligned tensors one at a time.
__device__ __forceinline__ float fq1(float v, float s, int z, uint8_t& m) {
  const float r = rintf(v / s) + (float)z;
  const float c = fminf(fmaxf(r, -128.f), 127.f);
  m = r >= -128.f && r <= 127.f;
  return (c - (float)z) * s;
}

__global__ void k_fq_f(const float* __restrict__ x, int64_t n, float s, int z,
                       float* __restrict__ y, uint8_t* __restrict__ mask, int vec) {
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                nt = (int64_t)gridDim.x * blockDim.x;
  const int64_t n4 = vec ? n / 4 : 0;
  for (int64_t q = t0; q < n4; q += nt) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(x) + q);
    uchar4 m;
    float4 o;
    o.x = fq1(v.x, s, z, m.x);
    o.y = fq1(v.y, s, z, m.y);
    o.z = fq1(v.z, s, z, m.z);
    o.w = fq1(v.w, s, z, m.w);
    reinterpret_cast<float4*>(y)[q] = o;
    reinterpret_cast<uchar4*>(mask)[q] = m;
  }
  for (int64_t q = 4 * n4 + t0; q < n; q += nt) y[q] = fq1(x[q], s, z, mask[q]);
}

// Weights: the symmetric per-tensor scale max|w| / 127 (at least 1e-12 / 127)
// found on the device by one block, then the same rounding as k_fq_f with
// z = 0; the scale is formed in double and rounded to float like a host-side
// max(...) / 127.0 passed as a float.
__global__ void __launch_bounds__(1024) k_fq_w(const float* w, int64_t n, float* y,
                                               uint8_t* mask) {
  __shared__ float red[32];
  float m = 0.f;
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) m = fmaxf(m, fabsf(w[q]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) red[0] = m;
  }
  __syncthreads();
  const float s = (float)((double)fmaxf(red[0], 1e-12f) / 127.0);
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) y[q] = fq1(w[q], s, 0, mask[q]);
}

__global__ void k_fq_b(const float* __restrict__ dy, const uint8_t* __restrict__ mask, int64_t n,
                       float* __restrict__ dx, int vec) {
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                nt = (int64_t)gridDim.x * blockDim.x;
  const int64_t n4 = vec ? n / 4 : 0;
  for (int64_t q = t0; q < n4; q += nt) {
    const float4 g = __ldg(reinterpret_cast<const float4*>(dy) + q);
    const uchar4 m = __ldg(reinterpret_cast<const uchar4*>(mask) + q);
    reinterpret_cast<float4*>(dx)[q] =
        make_float4(m.x ? g.x : 0.f, m.y ? g.y : 0.f, m.z ? g.z : 0.f, m.w ? g.w : 0.f);
  }
  for (int64_t q = 4 * n4 + t0; q < n; q += nt) dx[q] = mask[q] ? dy[q] : 0.f;
}

bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// blocks for the row kernels: kRowIlp rows a warp, at most 8 blocks an SM
int rows_grid(int64_t rows, int max_blocks = 148 * 8) {
  const int64_t warps = (rows + kRowIlp - 1) / kRowIlp;
  return (int)std::max<int64_t>(
      1, std::min<int64_t>((warps * 32 + kRowThreads - 1) / kRowThreads, max_blocks));
}

int grid_for(int64_t work, int threads = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, 148 * 8));
}

template <class Items>
int gmv(Items it, const float* W, int S, int out, int in, int transpose, const float* bias,
        int bias_mode, const float* x, int64_t rows, float* y, int bf16, cudaStream_t st) {
  if (rows <= 0) return LPC_OK;
  const size_t smem = sizeof(float) * (size_t)S * in * out;
  const int blocks = (int)std::min<int64_t>((rows + kWarpsT - 1) / kWarpsT, 148 * 2);
#define LPC_GMV(O, I)                                                                       \
  do {                                                                                      \
    cudaFuncSetAttribute(k_gmv<O, I, Items>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                         (int)smem);                                                        \
    k_gmv<O, I, Items><<<blocks, kWarpsT * 32, smem, st>>>(it, W, S, transpose, bias,       \
                                                           bias_mode, x, rows, y, bf16);    \
  } while (0)
  if (out == 32 && in == 32) LPC_GMV(32, 32);
  else if (out == 32 && in == 64) LPC_GMV(32, 64);
  else if (out == 64 && in == 32) LPC_GMV(64, 32);
  else return LPC_INVALID_ARG;
#undef LPC_GMV
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? LPC_OK : LPC_CUDA_ERROR;
}

template <class Pairs>
int outer(Pairs p, int S, int A, int B, const float* dy, const float* x, int64_t rows,
          float* dW, int bf16, cudaStream_t st) {
  if (rows <= 0 || !dW) return LPC_OK;
  dim3 grid((unsigned)((rows + kOuterRows - 1) / kOuterRows), (unsigned)S);
  if (A == 32 && B == 32) k_outer<32, 32, Pairs><<<grid, 256, 0, st>>>(p, dy, x, rows, dW, bf16);
  else if (A == 32 && B == 64) k_outer<32, 64, Pairs><<<grid, 256, 0, st>>>(p, dy, x, rows, dW, bf16);
  else return LPC_INVALID_ARG;
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? LPC_OK : LPC_CUDA_ERROR;
}

int bias_grad(const float* dy, int64_t rows, int C, const uint64_t* slice_key, float* db,
              cudaStream_t st) {
  if (rows <= 0 || !db) return LPC_OK;
  if (C > 32 * kCh) return LPC_INVALID_ARG;
  k_bias_grad<<<rows_grid(rows), kRowThreads, 0, st>>>(dy, rows, C, slice_key, db);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? LPC_OK : LPC_CUDA_ERROR;
}

bool ok_dims(int cin, int cout) { return cout == 32 && (cin == 32 || cin == 64); }

}  // namespace
}  // namespace lpc

using namespace lpc;

extern "C" {

int lpc_t_conv_fwd(const float* x, int64_t N, int cin, const int32_t* nbr, const float* W,
                   const float* b, int cout, float* y, int bf16, uint64_t stream) {
  if (N < 0 || !ok_dims(cin, cout)) return LPC_INVALID_ARG;
  // bf16 operands: the gather-GEMM on the tensor cores
  if (bf16) return tconv_tc(x, N, cin, nbr, W, b, y, 0, reinterpret_cast<cudaStream_t>(stream));
  return gmv(ConvItems{nbr, 0}, W, 27, cout, cin, 0, b, b ? 1 : 0, x, N, y, bf16,
             reinterpret_cast<cudaStream_t>(stream));
}

int lpc_t_conv_bwd(const float* x, const float* dy, int64_t N, int cin, const int32_t* nbr,
                   const float* W, int cout, float* dx, float* dW, float* db, int bf16,
                   uint64_t stream) {
  if (N < 0 || !ok_dims(cin, cout)) return LPC_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int s = LPC_OK;
  if (bf16 && dW) {  // dW and dx from one gather of dy on the tensor cores
    s = tconv_bwd_tc(x, dy, N, cin, nbr, W, dx, dW, st);
    if (!s) s = bias_grad(dy, N, cout, nullptr, db, st);
    return s;
  }
  if (dx && bf16) s = tconv_tc(dy, N, cin, nbr, W, nullptr, dx, 1, st);
  else if (dx) s = gmv(ConvItems{nbr, 1}, W, 27, cin, cout, 1, nullptr, 0, dy, N, dx, bf16, st);
  if (!s) s = outer(ConvPairs{nbr}, 27, cout, cin, dy, x, N, dW, bf16, st);
  if (!s) s = bias_grad(dy, N, cout, nullptr, db, st);
  return s;
}

int lpc_t_up_fwd(const float* x, int64_t Np, int cin, const uint32_t* off, const uint32_t* par,
                 const uint64_t* ckey, int64_t Nc, const float* W, const float* b, int cout,
                 float* y, int bf16, uint64_t stream) {
  if (Nc < 0 || Np < 0 || !ok_dims(cin, cout)) return LPC_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // bf16 operands: every parent against all eight slots on the tensor cores
  if (bf16 && cout == 32 && off) return texpand_tc(x, Np, off, ckey, W, cout, cin, b, y, 0, st);
  return gmv(UpFwdItems{par, ckey}, W, 8, cout, cin, 0, b, b ? 2 : 0, x, Nc, y, bf16, st);
}

int lpc_t_up_bwd(const float* x, const float* dy, int64_t Np, int cin, const uint32_t* off,
                 const uint32_t* par, const uint64_t* ckey, int64_t Nc, const float* W, int cout,
                 float* dx, float* dW, float* db, int bf16, uint64_t stream) {
  if (Nc < 0 || Np < 0 || !ok_dims(cin, cout)) return LPC_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int s = LPC_OK;
  if (bf16 && cout == 32 && dW && off) {  // dW and dx from one gather of the children's dy
    s = tup_bwd_tc(x, dy, Np, Nc, cin, off, ckey, W, dx, dW, st);
    if (!s) s = bias_grad(dy, Nc, cout, ckey, db, st);
    return s;
  }
  if (dx && bf16 && cout == 32)  // the parents' eight child slots on the tensor cores
    s = tslot_tc(dy, Np, Nc, off, ckey, W, cout, cin, nullptr, dx, 1, st);
  else if (dx)
    s = gmv(ChildItems{off, ckey}, W, 8, cin, cout, 1, nullptr, 0, dy, Np, dx, bf16, st);
  if (!s) s = outer(UpPairs{par, ckey}, 8, cout, cin, dy, x, Nc, dW, bf16, st);
  if (!s) s = bias_grad(dy, Nc, cout, ckey, db, st);
  return s;
}

int lpc_t_down_fwd(const float* x, int64_t Nc, int cin, const uint32_t* off, const uint64_t* ckey,
                   int64_t Np, const float* W, const float* b, int cout, float* y, int bf16,
                   uint64_t stream) {
  if (Np < 0 || Nc < 0 || !ok_dims(cin, cout)) return LPC_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // bf16 operands: the parents' eight child slots gathered on the tensor cores
  if (bf16 && cin == 32 && (cout == 32 || cout == 64))
    return tslot_tc(x, Np, Nc, off, ckey, W, cout, cin, b, y, 0, st);
  return gmv(ChildItems{off, ckey}, W, 8, cout, cin, 0, b, b ? 1 : 0, x, Np, y, bf16, st);
}

int lpc_t_down_bwd(const float* x, const float* dy, int64_t Nc, int cin, const uint32_t* off,
                   const uint32_t* par, const uint64_t* ckey, int64_t Np, const float* W,
                   int cout, float* dx, float* dW, float* db, int bf16, uint64_t stream) {
  if (Nc < 0 || Np < 0 || !ok_dims(cin, cout)) return LPC_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int s = LPC_OK;
  if (dx && bf16 && cin == 32 && off)  // every parent's dy against all slots on the tensor cores
    s = texpand_tc(dy, Np, off, ckey, W, cout, cin, nullptr, dx, 1, st);
  else if (dx)
    s = gmv(UpFwdItems{par, ckey}, W, 8, cin, cout, 1, nullptr, 0, dy, Nc, dx, bf16, st);
  if (!s && bf16 && cin == 32 && off && dW)  // the children's x by slot against the parents' dy
    s = tdown_dw_tc(x, dy, Np, Nc, cout, off, ckey, dW, st);
  else if (!s) s = outer(DownPairs{par, ckey}, 8, cout, cin, dy, x, Nc, dW, bf16, st);
  if (!s) s = bias_grad(dy, Np, cout, nullptr, db, st);
  return s;
}

int lpc_t_embed_fwd(const uint8_t* codes, int64_t N, const float* E, int C, float* y,
                    uint64_t stream) {
  if (N < 0 || C < 1) return LPC_INVALID_ARG;
  if (N == 0) return LPC_OK;
  k_embed_f<<<rows_grid(N), kRowThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(codes, N,
                                                                                      E, C, y);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? LPC_OK : LPC_CUDA_ERROR;
}

int lpc_t_embed_bwd(const uint8_t* codes, int64_t N, const float* dy, int C, float* dE,
                    uint64_t stream) {
  if (N < 0 || C < 1) return LPC_INVALID_ARG;
  if (N == 0) return LPC_OK;
  // block-private tables in shared memory up to 64 channels (64 KB a block)
  const int acc_smem = C <= 64;
  const size_t smem = acc_smem ? sizeof(float) * 256 * C : 0;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_embed_b, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(float) * 256 * 64));
    attr = true;
  }
  k_embed_b<<<rows_grid(N, 148 * 2), kRowThreads, smem, reinterpret_cast<cudaStream_t>(stream)>>>(
      codes, N, dy, C, dE, acc_smem);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? LPC_OK : LPC_CUDA_ERROR;
}

int lpc_t_prelu_fwd(const float* x, int64_t N, int C, const float* a, float* y, uint64_t stream) {
  if (N < 0 || C < 1 || C > 256) return LPC_INVALID_ARG;
  if (N == 0) return LPC_OK;
  k_prelu_f<<<rows_grid(N), kRowThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(x, N, C, a,
                                                                                      y);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? LPC_OK : LPC_CUDA_ERROR;
}

int lpc_t_prelu_bwd(const float* x, const float* dy, int64_t N, int C, const float* a, float* dx,
                    float* da, uint64_t stream) {
  if (N < 0 || C < 1 || C > 256 || !da) return LPC_INVALID_ARG;
  if (N == 0) return LPC_OK;
  k_prelu_b<<<rows_grid(N), kRowThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(x, dy, N, C,
                                                                                      a, dx, da);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? LPC_OK : LPC_CUDA_ERROR;
}

int lpc_t_fq_fwd(const float* x, int64_t n, float s, int z, float* y, uint8_t* mask,
                 uint64_t stream) {
  if (n < 0 || !(s > 0.f) || z < -128 || z > 127) return LPC_INVALID_ARG;
  if (n == 0) return LPC_OK;
  const int vec = al16(x) && al16(y) && (reinterpret_cast<uintptr_t>(mask) & 3) == 0;
  k_fq_f<<<grid_for(vec ? (n + 3) / 4 : n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      x, n, s, z, y, mask, vec);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? LPC_OK : LPC_CUDA_ERROR;
}

int lpc_t_fq_w(const float* w, int64_t n, float* y, uint8_t* mask, uint64_t stream) {
  if (n < 0) return LPC_INVALID_ARG;
  if (n == 0) return LPC_OK;
  k_fq_w<<<1, 1024, 0, reinterpret_cast<cudaStream_t>(stream)>>>(w, n, y, mask);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? LPC_OK : LPC_CUDA_ERROR;
}

int lpc_t_fq_bwd(const float* dy, const uint8_t* mask, int64_t n, float* dx, uint64_t stream) {
  if (n < 0) return LPC_INVALID_ARG;
  if (n == 0) return LPC_OK;
  const int vec = al16(dy) && al16(dx) && (reinterpret_cast<uintptr_t>(mask) & 3) == 0;
  k_fq_b<<<grid_for(vec ? (n + 3) / 4 : n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      dy, mask, n, dx, vec);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? LPC_OK : LPC_CUDA_ERROR;
}

}  // extern "C"
