// Upsampling + Pruning (Eq. 6, 9, 11) on the tcgen05 tensor cores, exact in
// integer arithmetic: every parent row (q - z_in, as bf16) times the weights
// of all eight child slots (N = 8 x 32 = 256, K = Cin) in one M = 128 MMA
// chain per tile of 128 parents; the epilogue keeps only the slots that hold
// a child (the pruning), adds the slot's bias, applies the slot's PReLU and
// the fixed-point requantisation (Eq. 14) and writes each child's int8 row
// (and, where asked, its code embedding beside it).
//
// Exactness: |q - z| <= 255 and |w| <= 127 are exact in bf16, every product
// (|p| <= 32,385) is exact in fp32 and a row sums at most 64 of them
// (< 2^21), so the fp32 accumulator holds the integer sum exactly whatever
// the order of accumulation.
//
// Orientation: the weights are the M side (rows slot x 32 + channel, two
// M = 128 MMAs for slots 0-3 and 4-7) and the tile's 128 parents the N side,
// so an accumulator lane is one (slot, channel) and its columns the parents.
// Roles (416 threads, one persistent CTA per SM):
//  - 4 producer warps, one parent row a thread: 16-byte loads of the int8
//    row, (q - z_in) to bf16, 16-byte shared-memory stores into a ring of
//    swizzled K-major stages, then a proxy fence and an arrive on the
//    stage's "full" barrier;
//  - 8 epilogue warps, one per slot (TMEM lane quadrant x accumulator half),
//    lane = output channel: per 32 parents, a ballot of the parents whose
//    occupancy code has the warp's slot; the warp walks only those,
//    finishing one child's 32 channels per step (no divergence: every lane
//    works on the same child), with 32-byte coalesced stores;
//  - 1 MMA warp: one thread issues 2 x Cin / 16 MMAs per tile into one of
//    two 256-column accumulators and commits the stage and the accumulator.
// Every wait is bounded; a wait that gives up raises a shared abort flag and
// the CTA drains its MMAs before it frees its tensor memory.
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc_util.cuh"

namespace lpc {
namespace {

constexpr int kUM = 128;          // parents a tile
constexpr int kUProd = 128;       // producer threads (warps 0-3)
constexpr int kUEpi = 256;        // epilogue threads (warps 4-11)
constexpr int kUMmaW = 12;        // MMA warp
constexpr int kUThreads = kUProd + kUEpi + 32;
constexpr int kUStages = 4;
constexpr int kUN = 256;          // accumulator columns: 8 slots x 32 channels
constexpr int kUIlp = 4;          // children of a slot in flight per epilogue warp

template <int CIN>
struct UpCfg {
  static constexpr int RB = CIN * 2;  // bf16 row bytes
  static constexpr int SW = CIN == 64 ? 128 : 64;
  static constexpr int kStageBytes = kUM * RB;
  static constexpr int kWBytes = kUN * 128;  // one 64-element K block of 256 rows
  static constexpr size_t kSmem = 1024 + kWBytes + (size_t)kUStages * kStageBytes;
};

__device__ int g_up_tc_error = 0;

__device__ __forceinline__ bool up_try_wait(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for a phase; false when this or another thread of the CTA gave up
__device__ __forceinline__ bool up_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  const uint32_t a = tc::smem_u32(bar);
  if (up_try_wait(a, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (up_try_wait(a, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > (1ll << 31)) {
      *abort = 1;
      return false;
    }
  }
}
__device__ __forceinline__ void up_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

template <int CIN>
__global__ void __launch_bounds__(kUThreads, 1) k_up_tc(const UpTcArgs a) {
  using Cfg = UpCfg<CIN>;
  extern __shared__ unsigned char smraw[];
  // aligned to 1024 by offsetting smraw itself, so that accesses through sm
  // stay shared-memory accesses (an integer round trip would make them generic)
  unsigned char* sm = smraw + ((1024u - (tc::smem_u32(smraw) & 1023u)) & 1023u);
  unsigned char* sW = sm;  // weights: rows slot x 32 + channel, the A operand
  unsigned char* sX = sm + Cfg::kWBytes;  // parent-row stages, the B operand
  __shared__ uint64_t full_bar[kUStages], empty_bar[kUStages], acc_full[2], acc_empty[2];
  __shared__ uint64_t w_bar, drain_bar;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  __shared__ uint32_t sTr[kUEpi / 32][32 * 33];  // each epilogue warp's transposed chunk
  __shared__ __align__(16) int8_t sE[256 * 32];  // the oe embedding table
  volatile int* abort = &abort_flag;

  const int64_t n = *a.d_np;
  const int64_t ntiles = (n + kUM - 1) / kUM;
  if ((int64_t)blockIdx.x >= ntiles) return;  // capacity-sized grid: nothing here
  const int my_tiles = (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1);
  auto tile_r0 = [&](int lt) { return ((int64_t)blockIdx.x + (int64_t)lt * gridDim.x) * kUM; };

  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (w == kUMmaW) tc::tmem_alloc(&tslot, 2 * kUN);
  if (t == 0) {
    for (int s = 0; s < kUStages; s++) {
      tc::mbar_init(&full_bar[s], kUProd);
      tc::mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; b++) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], kUEpi);
    }
    tc::mbar_init(&w_bar, 1);
    tc::mbar_init(&drain_bar, 1);
    tc::fence_mbar_init();
    abort_flag = 0;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     tc::smem_u32(&w_bar)),
                 "r"(Cfg::kWBytes)
                 : "memory");
    for (int off = 0; off < Cfg::kWBytes; off += 16384)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
          "[%3];" ::"r"(tc::smem_u32(sW + off)),
          "l"(reinterpret_cast<const unsigned char*>(a.wimg) + off), "r"(16384),
          "r"(tc::smem_u32(&w_bar))
          : "memory");
  }
  const bool hi = a.hi != 0;  // mult holds the high-word form
  if (a.oe.table)
    for (int i = t; i < 256 * 32 / 16; i += kUThreads)
      reinterpret_cast<uint4*>(sE)[i] = __ldg(reinterpret_cast<const uint4*>(a.oe.table) + i);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tslot;

  if (w < kUProd / 32) {
    // ---------------------------------------------------------- producers --
    const int row = t;
    for (int lt = 0; lt < my_tiles; lt++) {
      const int sg = lt % kUStages;
      if (lt >= kUStages && !up_wait(&empty_bar[sg], ((lt / kUStages) - 1) & 1, abort)) break;
      const int64_t p = tile_r0(lt) + row;
      const uint32_t dst = tc::smem_u32(sX + (size_t)sg * Cfg::kStageBytes);
#pragma unroll
      for (int c = 0; c < CIN / 16; c++) {
        uint4 raw = make_uint4(0, 0, 0, 0);
        if (p < n) raw = __ldg(reinterpret_cast<const uint4*>(a.x + p * a.x_stride) + c);
        const int8_t* b8 = reinterpret_cast<const int8_t*>(&raw);
        __align__(16) __nv_bfloat16 v[16];
#pragma unroll
        for (int i = 0; i < 16; i++) v[i] = __int2bfloat16_rn(p < n ? (int)b8[i] - a.z_in : 0);
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const uint4 q = reinterpret_cast<const uint4*>(v)[h];
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(
                           dst + tc::swz<Cfg::SW>(row * Cfg::RB + (2 * c + h) * 16)),
                       "r"(q.x), "r"(q.y), "r"(q.z), "r"(q.w)
                       : "memory");
        }
      }
      tc::fence_async_smem();  // the stores are read by the MMA (async proxy)
      up_arrive(&full_bar[sg]);
    }
  } else if (w == kUMmaW) {
    // ---------------------------------------------------------------- MMA --
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16(kUM, kUM);
      bool ok = up_wait(&w_bar, 0, abort);
      for (int lt = 0; lt < my_tiles && ok; lt++) {
        const int b = lt & 1, sg = lt % kUStages;
        if (lt >= 2 && !up_wait(&acc_empty[b], ((lt >> 1) - 1) & 1, abort)) break;
        if (!up_wait(&full_bar[sg], (lt / kUStages) & 1, abort)) break;
        tc::tc_fence_after();
        const uint32_t sx = tc::smem_u32(sX + (size_t)sg * Cfg::kStageBytes);
#pragma unroll
        for (int mt = 0; mt < 2; mt++)
#pragma unroll
          for (int ks = 0; ks < CIN / 16; ks++)
            tc::mma_bf16(tbase + (uint32_t)(b * kUN + mt * kUM),
                         tc::smem_desc<128>(tc::smem_u32(sW) + mt * kUM * 128 + ks * 32, 1024),
                         tc::smem_desc<Cfg::SW>(sx + ks * 32, 8 * Cfg::RB), idesc,
                         ks > 0 ? 1u : 0u);
        tc::mma_commit(&empty_bar[sg]);
        tc::mma_commit(&acc_full[b]);
      }
      tc::mma_commit(&drain_bar);
      if (!tc::mbar_wait(&drain_bar, 0)) *abort = 1;
    }
    __syncwarp();
  } else {
    // ----------------------------------------------------------- epilogue --
    // warp (quadrant q, half mt) owns slot s = q + 4 mt; lane = channel
    const int q = w & 3, mt = (w - kUProd / 32) >> 2, s = q + 4 * mt;
    const int ch = s * 32 + lane;
    const int32_t bias = a.bias[ch], slope = a.slope[ch];
    const int32_t mult = a.mult[ch];
    const uint32_t below = (1u << s) - 1u;
    const uint32_t dcol = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(mt * kUM);
    uint32_t* sT = sTr[w - kUProd / 32];
    for (int lt = 0; lt < my_tiles; lt++) {
      const int b = lt & 1;
      // before the accumulators are waited for: lane l's parent in each of
      // the tile's four 32-parent chunks (first child, occupancy code = the
      // mask of its children's slots), then its child in this slot (row,
      // and with oe its code); all loads of a step in flight together
      uint32_t c0[4], m[4], cr[4], cc[4];
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const int64_t p = tile_r0(lt) + 32 * k + lane;
        c0[k] = p < n ? __ldg(a.poff + p) : 0u;
        m[k] = p < n ? (uint32_t)__ldg(a.pcode + p) : 0u;
      }
#pragma unroll
      for (int k = 0; k < 4; k++) {
        cr[k] = c0[k] + __popc(m[k] & below);
        cc[k] = (((m[k] >> s) & 1u) && a.oe.table) ? (uint32_t)__ldg(a.oe.code + cr[k]) : 0u;
      }
      if (!__all_sync(0xffffffffu, up_wait(&acc_full[b], (lt >> 1) & 1, abort))) break;
      tc::tc_fence_after();
#pragma unroll
      for (int k = 0; k < 4; k++) {  // 32 parents (accumulator columns) at a time
        uint32_t rem = __ballot_sync(0xffffffffu, (m[k] >> s) & 1u);
        if (!rem) continue;
        const uint32_t my_r = cr[k], my_code = cc[k];
        uint32_t v[2][16];
        tc::tmem_ld16_issue(dcol + (uint32_t)(b * kUN + 32 * k), v[0]);
        tc::tmem_ld16_issue(dcol + (uint32_t)(b * kUN + 32 * k + 16), v[1]);
        tc::tmem_wait_ld();
        tc::tmem_regs_ready(v[0]);
        tc::tmem_regs_ready(v[1]);
        // transposed through shared memory (row = lane, stride 33: no bank
        // conflicts either way), so that a child's column is one load
#pragma unroll
        for (int i = 0; i < 32; i++) sT[lane * 33 + i] = v[i >> 4][i & 15];
        __syncwarp();
        while (rem) {
          // up to four children at a time (warp-uniform: every lane works on
          // the same children), their chains independent
          int jj[kUIlp];
#pragma unroll
          for (int u = 0; u < kUIlp; u++) {
            jj[u] = rem ? __ffs(rem) - 1 : -1;
            rem &= rem - 1;
          }
          uint32_t r[kUIlp], code[kUIlp];
          int32_t acc[kUIlp];
#pragma unroll
          for (int u = 0; u < kUIlp; u++) {
            const int j = jj[u] < 0 ? 0 : jj[u];
            r[u] = __shfl_sync(0xffffffffu, my_r, j);
            code[u] = __shfl_sync(0xffffffffu, my_code, j);
            acc[u] = __float2int_rn(__uint_as_float(sT[lane * 33 + j])) + bias;
          }
#pragma unroll
          for (int u = 0; u < kUIlp; u++) {
            if (a.prelu) acc[u] = prelu(acc[u], slope);
            acc[u] = hi ? requant_hi(acc[u], mult, a.z_out) : requant(acc[u], mult, a.shift, a.z_out);
          }
#pragma unroll
          for (int u = 0; u < kUIlp; u++) {
            if (jj[u] < 0) break;
            int8_t* orow = a.out + (int64_t)r[u] * a.out_stride;
            orow[a.out_col + lane] = (int8_t)acc[u];
            if (a.oe.table)  // the next step's Concat(., E[Y]) half of the child's row
              orow[a.oe_col + lane] = sE[code[u] * 32 + lane];
          }
        }
        __syncwarp();  // the transposed chunk is read before the next one lands
      }
      tc::tc_fence_before();
      up_arrive(&acc_empty[b]);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (t == kUThreads - 32) tc::mbar_wait(&w_bar, 0);  // the weights' copies have landed
  if (w == kUMmaW) tc::tmem_dealloc(tbase, 2 * kUN);
  if (t == 0 && abort_flag) atomicExch(&g_up_tc_error, 1);
}

}  // namespace

size_t up_tc_weight_bytes() { return UpCfg<64>::kWBytes; }

// Weight image of an eight-slot layer W[8][32][cin] (int8) as bf16: row m =
// slot s x 32 + output channel, K = cin (at most 64, one block), 128-byte
// rows, 128-byte swizzled; the MMA reads it as the K-major A operand, rows
// 0-127 and 128-255 in two M = 128 MMAs.
void pack_up_tc_weights(const int8_t* W, int cin, uint16_t* img) {
  unsigned char* p = reinterpret_cast<unsigned char*>(img);
  memset(p, 0, up_tc_weight_bytes());
  for (int nrow = 0; nrow < kUN; nrow++)
    for (int k = 0; k < cin; k++) {
      const __nv_bfloat16 b = __float2bfloat16_rn((float)W[(size_t)nrow * cin + k]);
      uint32_t off = (uint32_t)(nrow * 128 + k * 2);
      off ^= ((off >> 7) & 7) << 4;
      memcpy(p + off, &b, 2);
    }
}

int up_tc_error(bool reset) {
  int e = 0;
  cudaMemcpyFromSymbol(&e, g_up_tc_error, sizeof(int));
  if (reset && e) {
    const int z = 0;
    cudaMemcpyToSymbol(g_up_tc_error, &z, sizeof(int));
  }
  return e;
}

void launch_up_tc(const UpTcArgs& a, int64_t np_host, cudaStream_t st) {
  if (np_host <= 0) return;
  const int blocks = (int)std::min<int64_t>((np_host + kUM - 1) / kUM, 148);
  if (a.cin == 64) {
    cudaFuncSetAttribute(k_up_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)UpCfg<64>::kSmem);
    k_up_tc<64><<<blocks, kUThreads, UpCfg<64>::kSmem, st>>>(a);
  } else {
    cudaFuncSetAttribute(k_up_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)UpCfg<32>::kSmem);
    k_up_tc<32><<<blocks, kUThreads, UpCfg<32>::kSmem, st>>>(a);
  }
  count_launches(1);
}

}  // namespace lpc
