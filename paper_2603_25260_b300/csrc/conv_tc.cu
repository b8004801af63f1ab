// 3x3x3 sparse convolution of the ResBlock (Eq. 5, 8, 10) on the tcgen05
// tensor cores, exact in integer arithmetic.
//
// sm_103a has no INT8 tcgen05 path, so the contraction runs on the bf16 pipe:
// every input value is the integer (q - z) in [-255, 255] and every weight an
// integer in [-127, 127]; both are exact in bf16 and every product (|p| <=
// 32,385) is exact in fp32.  Each fp32 accumulator in tensor memory sums at
// most 256 products (|partial sum| <= 256 * 32,640 < 2^23), so every partial
// sum is an integer below 2^23 whatever the order of accumulation: the fp32
// result is exact.  The 27 x Cin reduction is split into ceil(27 Cin / 256)
// such accumulators (separate TMEM column blocks) which the epilogue adds in
// INT32.
//
// One CTA (256 threads) owns a tile of 128 output nodes (Morton order) at a
// time, persistent over tiles.  The weights of all 27 offsets stay in shared
// memory (bf16, 128-byte swizzled K-major).  For every offset that at least
// one node of the tile has, the threads gather the 128 neighbour rows
// (pre-subtracted bf16 rows, 16-byte cp.async copies, zero-filled when the
// neighbour is absent, which is the exact zero padding of the sparse conv)
// into a swizzled stage; one thread issues the M=128, N=32, K=16 MMAs into
// the offset's accumulator.  Gathers run several offsets ahead of the MMAs.
// The epilogue reads the accumulators from TMEM, adds the bias, applies the
// PReLU and the fixed-point requantisation (Eq. 14), the fused residual
// merge of the ResBlock, and writes int8 (and optionally the next conv's
// bf16 input).
#include <cuda_bf16.h>

#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc_util.cuh"

namespace lpc {

namespace {

constexpr int kTileM = 128;
constexpr int kThreads = 256;
constexpr int kDepth = 3;  // offsets gathered ahead of the MMA issue

template <int CIN>
struct ConvCfg {
  static constexpr int RB = CIN * 2;                 // bf16 row bytes
  static constexpr int SW = CIN == 64 ? 128 : 64;    // swizzle of the A stage
  static constexpr int kStages = CIN == 64 ? 6 : 8;
  static constexpr int kStageBytes = kTileM * RB;
  static constexpr int kPerGroup = 256 / CIN;        // offsets per fp32 accumulator
  static constexpr int kBBlocks = (27 * CIN + 63) / 64;
  static constexpr int kBBytes = kBBlocks * 4096;
  static constexpr int kChunks = RB / 16;            // 16-byte chunks per row
  static constexpr int kNbrBytes = kTileM * 27 * 4;  // the tile's neighbour rows
  static constexpr size_t kSmem =
      1024 + kBBytes + (size_t)kStages * kStageBytes + kNbrBytes;
};

__device__ int g_conv_error = 0;

template <int CIN>
__global__ void __launch_bounds__(kThreads, 1)
k_conv333_tc(ConvTcArgs a) {
  using Cfg = ConvCfg<CIN>;
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  unsigned char* sB = sm;
  unsigned char* sA = sm + Cfg::kBBytes;
  int32_t* sNbr = reinterpret_cast<int32_t*>(sA + (size_t)Cfg::kStages * Cfg::kStageBytes);
  __shared__ uint64_t bar[Cfg::kStages];
  __shared__ uint64_t done_bar;
  __shared__ uint32_t tslot;
  __shared__ uint32_t tile_mask;
  __shared__ int abort_flag;

  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (w == 0) tc::tmem_alloc(&tslot, 256);
  if (t == 0) {
    for (int s = 0; s < Cfg::kStages; s++) tc::mbar_init(&bar[s], 1);
    tc::mbar_init(&done_bar, 1);
    tc::fence_mbar_init();
    abort_flag = 0;
  }
  // weights: pre-swizzled image, copied linearly
  {
    const uint4* src = reinterpret_cast<const uint4*>(a.wimg);
    uint4* dst = reinterpret_cast<uint4*>(sB);
    for (int i = t; i < Cfg::kBBytes / 16; i += kThreads) dst[i] = __ldg(src + i);
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tslot;
  const int64_t n = *a.d_n;
  const int64_t ntiles = (n + kTileM - 1) / kTileM;
  constexpr uint32_t idesc = tc::idesc_bf16(kTileM, 32);

  // epilogue constants of this thread's 16 output channels
  const int half = w >> 2;          // column half handled by this warp
  const int lrow = (w & 3) * 32 + lane;  // TMEM lane = row within the tile
  int32_t bias[16], mult[16], slope[16], ma[16], mb[16], rsl[16];
#pragma unroll
  for (int i = 0; i < 16; i++) {
    const int co = half * 16 + i;
    bias[i] = a.bias[co];
    mult[i] = a.mult[co];
    slope[i] = a.prelu ? a.slope[co] : 0;
    ma[i] = a.has_res ? a.res_mab[co] : 0;
    mb[i] = a.has_res ? a.res_mab[32 + co] : 0;
    rsl[i] = a.has_res ? a.res_slope[co] : 0;
  }

  uint32_t use = 0;    // stage uses so far (stage = use % kStages)
  uint32_t tiles_done = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * kTileM;
    // the tile's neighbour rows into shared memory (coalesced), then the
    // offsets present in the tile (OR of the rows' neighbour masks)
    if (t == 0) tile_mask = 0;
    {
      const int64_t base = r0 * 27, lim = n * 27;
      for (int i = t; i < kTileM * 27; i += kThreads)
        sNbr[i] = base + i < lim ? __ldg(a.nbr + base + i) : -1;
    }
    __syncthreads();
    if (t < kTileM) {
      uint32_t m = 0;
#pragma unroll
      for (int o = 0; o < 27; o++) m |= (uint32_t)(sNbr[t * 27 + o] >= 0) << o;
      m = __reduce_or_sync(0xffffffffu, m);
      if (lane == 0) atomicOr(&tile_mask, m);
    }
    __syncthreads();
    const uint32_t mask = tile_mask;
    const int count = __popc(mask);

    // gathers for offset #j into stage (use0 + j) % kStages; MMAs kDepth behind
    uint32_t rem = mask;
    int next_o = rem ? __ffs(rem) - 1 : 0;
    const uint32_t use0 = use;
    int mma_o[32];
    for (int j = 0; j < count + kDepth; j++) {
      if (j < count) {
        const int o = next_o;
        rem &= rem - 1;
        next_o = rem ? __ffs(rem) - 1 : 0;
        mma_o[j] = o;
        const uint32_t u = use0 + j;
        const int s = (int)(u % Cfg::kStages);
        if (u >= (uint32_t)Cfg::kStages && !abort_flag) {
          // the MMAs that last read this stage must be done
          const bool ok = tc::mbar_wait(&bar[s], ((u / Cfg::kStages) - 1) & 1);
          if (!ok) abort_flag = 1;
        }
        const uint32_t sbase = tc::smem_u32(sA + (size_t)s * Cfg::kStageBytes);
        for (int q = t; q < kTileM * Cfg::kChunks; q += kThreads) {
          const int row = q / Cfg::kChunks, c = q % Cfg::kChunks;
          const int32_t nb = sNbr[row * 27 + o];
          const bool present = nb >= 0;
          const unsigned char* src =
              reinterpret_cast<const unsigned char*>(a.xb) +
              ((present ? (int64_t)nb : 0) * a.x_stride) * 2 + c * 16;
          tc::cp_async16(sbase + tc::swz<Cfg::SW>(row * Cfg::RB + c * 16), src, present);
        }
      }
      tc::cp_async_commit();
      if (j >= kDepth - 1 && j - (kDepth - 1) < count) {
        const int jm = j - (kDepth - 1);
        tc::cp_async_wait<kDepth - 1>();
        tc::fence_async_smem();
        __syncthreads();
        if (t == 0 && !abort_flag) {
          tc::tc_fence_after();
          const int o = mma_o[jm];
          const uint32_t u = use0 + jm;
          const int s = (int)(u % Cfg::kStages);
          const int g = jm / Cfg::kPerGroup;
          const uint32_t sa = tc::smem_u32(sA + (size_t)s * Cfg::kStageBytes);
#pragma unroll
          for (int ks = 0; ks < CIN / 16; ks++) {
            const int k0 = o * CIN + ks * 16;
            const uint32_t sb = tc::smem_u32(sB) + (k0 / 64) * 4096 + (k0 % 64) * 2;
            tc::mma_bf16(tbase + g * 32, tc::smem_desc<Cfg::SW>(sa + ks * 32, 8 * Cfg::RB),
                         tc::smem_desc<128>(sb, 1024), idesc,
                         (jm % Cfg::kPerGroup != 0 || ks > 0) ? 1u : 0u);
          }
          tc::mma_commit(&bar[s]);
        }
      }
    }
    use = use0 + count;
    // all MMAs of the tile done
    if (t == 0 && !abort_flag) tc::mma_commit(&done_bar);
    bool to = false;
    if (!abort_flag) to = !tc::mbar_wait(&done_bar, tiles_done & 1);
    if (__syncthreads_or(to)) abort_flag = 1;
    tiles_done++;
    tc::tc_fence_after();

    // epilogue: sum the accumulators in INT32, bias, PReLU, requant, residual
    const int groups = (count + Cfg::kPerGroup - 1) / Cfg::kPerGroup;
    int32_t acc[16];
#pragma unroll
    for (int i = 0; i < 16; i++) acc[i] = bias[i];
    for (int g = 0; g < groups; g++) {
      float v[16];
      tc::tmem_ld16(tbase + ((uint32_t)((w & 3) * 32) << 16) + g * 32 + half * 16, v);
#pragma unroll
      for (int i = 0; i < 16; i++) acc[i] += __float2int_rn(v[i]);
    }
    const int64_t r = r0 + lrow;
    if (r < n && !abort_flag) {
      int8_t q[16];
      if (a.has_res) {
        __align__(16) int8_t y1[16];
        *reinterpret_cast<uint4*>(y1) =
            *reinterpret_cast<const uint4*>(a.y1 + r * a.y1_stride + half * 16);
#pragma unroll
        for (int i = 0; i < 16; i++) {
          int32_t v = acc[i];
          if (a.prelu) v = prelu(v, slope[i]);
          const int y2 = requant(v, mult[i], a.shift, a.z_out);
          int32_t m = (y1[i] - a.res_z1) * ma[i] + (y2 - a.res_z2) * mb[i];
          m = prelu(m, rsl[i]);
          q[i] = (int8_t)requant(m, 1, a.res_shift, a.res_z_out);
        }
      } else {
#pragma unroll
        for (int i = 0; i < 16; i++) {
          int32_t v = acc[i];
          if (a.prelu) v = prelu(v, slope[i]);
          q[i] = (int8_t)requant(v, mult[i], a.shift, a.z_out);
        }
      }
      __align__(16) int8_t qa[16];
#pragma unroll
      for (int i = 0; i < 16; i++) qa[i] = q[i];
      *reinterpret_cast<uint4*>(a.out + r * a.out_stride + a.out_col + half * 16) =
          *reinterpret_cast<const uint4*>(qa);
      if (a.outb) {
        __align__(16) __nv_bfloat16 b[16];
#pragma unroll
        for (int i = 0; i < 16; i++) b[i] = __int2bfloat16_rn((int)q[i] - a.outb_z);
        uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.outb) +
                                              r * a.outb_stride + half * 16);
        dst[0] = reinterpret_cast<const uint4*>(b)[0];
        dst[1] = reinterpret_cast<const uint4*>(b)[1];
      }
    }
    tc::tc_fence_before();
    __syncthreads();
  }
  tc::cp_async_wait<0>();
  tc::tc_fence_before();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(tbase, 256);
  if (t == 0 && abort_flag) atomicExch(&g_conv_error, 1);
}

// int8 rows -> bf16 (q - z) rows for the tensor-core gather
__global__ void k_to_bf16(const int8_t* __restrict__ x, int x_stride, int cols, int z,
                          const int64_t* d_n, __nv_bfloat16* out) {
  const int64_t n = *d_n;
  const int per = cols / 8;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * per;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / per;
    const int c = (int)(q - r * per);
    const uint2 raw = *reinterpret_cast<const uint2*>(x + r * x_stride + c * 8);
    const int8_t* b = reinterpret_cast<const int8_t*>(&raw);
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = __int2bfloat16_rn((int)b[i] - z);
    *reinterpret_cast<uint4*>(out + r * cols + c * 8) = *reinterpret_cast<const uint4*>(v);
  }
}

}  // namespace

size_t conv_tc_weight_bytes(int cin) {
  return cin == 64 ? ConvCfg<64>::kBBytes : ConvCfg<32>::kBBytes;
}

// Weight image of a 27-slice layer W[27][32][cin] (int8) as bf16, K-major
// with K = 27 * cin, in 64-element blocks of 32 rows x 128 bytes, each block
// 128-byte swizzled (the layout the MMA reads from shared memory).
void pack_conv_tc_weights(const int8_t* W, int cin, uint16_t* img) {
  const size_t bytes = conv_tc_weight_bytes(cin);
  unsigned char* p = reinterpret_cast<unsigned char*>(img);
  for (size_t i = 0; i < bytes; i++) p[i] = 0;
  const int K = 27 * cin;
  for (int co = 0; co < 32; co++)
    for (int k = 0; k < K; k++) {
      const int o = k / cin, ci = k % cin;
      const float v = (float)W[((size_t)o * 32 + co) * cin + ci];
      const __nv_bfloat16 b = __float2bfloat16_rn(v);
      const int blk = k / 64, kk = k % 64;
      uint32_t off = (uint32_t)(co * 128 + kk * 2);
      off ^= ((off >> 7) & 7) << 4;
      memcpy(p + (size_t)blk * 4096 + off, &b, 2);
    }
}

void launch_to_bf16(const int8_t* x, int x_stride, int cols, int z, const int64_t* d_n,
                    int64_t n_host, void* out, cudaStream_t st) {
  if (n_host <= 0) return;
  const int64_t work = n_host * (cols / 8);
  const int blocks = (int)std::min<int64_t>((work + 255) / 256, 148 * 8);
  k_to_bf16<<<blocks, 256, 0, st>>>(x, x_stride, cols, z, d_n,
                                    reinterpret_cast<__nv_bfloat16*>(out));
  count_launches(1);
}

void launch_conv333_tc(const ConvTcArgs& a, int cin, int64_t n_host, cudaStream_t st) {
  if (n_host <= 0) return;
  const int64_t ntiles = (n_host + kTileM - 1) / kTileM;
  const int blocks = (int)std::min<int64_t>(ntiles, 148);
  if (cin == 64) {
    cudaFuncSetAttribute(k_conv333_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)ConvCfg<64>::kSmem);
    k_conv333_tc<64><<<blocks, kThreads, ConvCfg<64>::kSmem, st>>>(a);
  } else {
    cudaFuncSetAttribute(k_conv333_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)ConvCfg<32>::kSmem);
    k_conv333_tc<32><<<blocks, kThreads, ConvCfg<32>::kSmem, st>>>(a);
  }
  count_launches(1);
}

int conv_tc_error(bool reset) {
  int e = 0;
  cudaMemcpyFromSymbol(&e, g_conv_error, sizeof(int));
  if (reset && e) {
    const int z = 0;
    cudaMemcpyToSymbol(g_conv_error, &z, sizeof(int));
  }
  return e;
}

}  // namespace lpc
