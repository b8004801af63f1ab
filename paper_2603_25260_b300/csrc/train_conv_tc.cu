// The differentiable twin's 3x3x3 sparse conv in bf16 mode on the tcgen05
// tensor cores: the forward y[i] = b + sum_o W[o] x[nbr[i][o]] (Eq. 5) and the
// input gradient dx[i] = sum_o W[o]^T dy[nbr[i][26 - o]].  bf16 mode rounds
// both operands of every product to bf16 and accumulates in fp32, which is
// what kind::f16 MMAs with fp32 accumulators in tensor memory compute.
//
// The kernel is the inference conv's gather-GEMM (see conv_tc.cu) with a
// float epilogue: per CTA and tile of 128 output rows, 8 producer warps
// gather the bf16 rows of the tile's neighbours offset by offset (zero rows
// for absent neighbours) into a ring of swizzled stages, three offsets per
// pipeline step; one thread issues the M=128 MMAs into one fp32 accumulator
// for all 27 offsets (N = the output width, 32 or 64); 4 epilogue warps add
// the bias and store fp32 rows.  The input gradient is the same gather over
// the rounded output gradient (32 channels) with the weight slices reversed
// and transposed (slice o' = W[26 - o']^T), so it reads the same kernel map.
// Every wait is bounded; a wait that gives up raises a shared abort flag,
// the CTA drains its copies and MMAs, frees its tensor memory and sets an
// error word that lpc_t_tc_error reports.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "../../include/lpc.h"
#include "../../include/lpc_train.h"
#include "common.cuh"
#include "kernels.h"
#include "tc_util.cuh"

namespace lpc {
namespace {

constexpr int kTM = 128;
constexpr int kPWarps = 8;
constexpr int kProd = 32 * kPWarps;
constexpr int kEpi = 128;
constexpr int kMmaW = kPWarps + 4;
constexpr int kThr = kProd + kEpi + 32;

// CIN: gathered row width (bf16 elements); NOUT: output width; KO: offsets
// gathered per output row (27: the 3x3x3 conv's kernel map; 8: a parent's
// eight child slots; 1: the row itself).  Ring shapes: 64-wide rows take
// 16 KB stages (6 stages), 32-wide rows 8 KB stages (12); G offsets share a
// pipeline step (3 of 27, 2 of 8, 1 of 1).
template <int CIN, int NOUT, int KO>
struct TCfg {
  static constexpr int RB = CIN * 2;
  static constexpr int SW = CIN == 64 ? 128 : 64;
  static constexpr int kChunks = RB / 16;
  static constexpr int kBBlocks = (KO * CIN + 63) / 64;
  static constexpr int kBBlockBytes = NOUT * 128;
  static constexpr int kBBytes = kBBlocks * kBBlockBytes;
  static constexpr int kStageBytes = kTM * RB;
  static constexpr int kStages = CIN == 64 ? 6 : 12;
  static constexpr int kG = KO == 27 ? 3 : (KO == 8 ? 2 : 1);
  static constexpr int kNbrBufs = KO == 1 ? 0 : ((CIN == 64 || NOUT == 64) && KO == 27 ? 1 : 2);
  static constexpr int kNbrBytes = kTM * KO * 4;
  static constexpr size_t kSmem =
      1024 + kBBytes + (size_t)kStages * kStageBytes + kNbrBufs * kNbrBytes;
  static constexpr int kTmemCols = 2 * NOUT;  // two accumulator buffers
  static_assert(kStages % kG == 0 && KO % kG == 0, "steps must tile the ring and the offsets");
  static_assert(kTmemCols == 64 || kTmemCols == 128 || kTmemCols == 512, "TMEM allocation");
  static_assert(kSmem <= 232448, "shared memory of a training conv variant exceeds the limit");
};

__device__ int g_tconv_error = 0;

__device__ __forceinline__ bool try_wait_parity(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity,
                                              volatile int* abort) {
  const uint32_t a = tc::smem_u32(bar);
  if (try_wait_parity(a, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (try_wait_parity(a, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > (1ll << 31)) {
      *abort = 1;
      return false;
    }
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(tc::smem_u32(dst)), "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   tc::smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool producer_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 1, %2, p;\n"
      "selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kProd)
      : "memory");
  return r != 0;
}

struct TConvArgs {
  const __nv_bfloat16* xb;  // gathered rows [rows][CIN], bf16
  const int32_t* nbr;       // [n][KO] (KO > 1): the gathered row of each offset, -1 absent
  int64_t n;
  const uint16_t* wimg;     // weight image, TCfg::kBBytes
  const float* bias;        // rows: [NOUT]; scatter: [8][32] per slot; or null
  float* out;               // rows: [n][NOUT]; scatter: [children][32]
  // scatter epilogue (NOUT = 256 = 8 slots x 32): output row p is a parent
  // whose children off[p] .. off[p + 1] - 1 (slot ckey & 7) take the 32
  // columns of their slot
  const uint32_t* off;
  const uint64_t* ckey;
};

// EPI 0: output rows of NOUT floats (+ bias); EPI 1: the scatter above.
template <int CIN, int NOUT, int KO, int EPI>
__global__ void __launch_bounds__(kThr, 1) k_tconv_tc(TConvArgs a) {
  using Cfg = TCfg<CIN, NOUT, KO>;
  constexpr int S = Cfg::kStages, G = Cfg::kG, SG = S / G, NB = Cfg::kNbrBufs;
  extern __shared__ unsigned char smraw[];
  // aligned to 1024 by offsetting smraw itself, so that accesses through sm
  // stay shared-memory accesses (an integer round trip would make them generic)
  unsigned char* sm = smraw + ((1024u - (tc::smem_u32(smraw) & 1023u)) & 1023u);
  unsigned char* sB = sm;
  unsigned char* sA = sm + Cfg::kBBytes;
  int32_t* sNbr0 = reinterpret_cast<int32_t*>(sA + (size_t)S * Cfg::kStageBytes);
  __shared__ uint64_t full_bar[SG], empty_bar[SG], acc_full[2], acc_empty[2], drain_bar;
  __shared__ uint64_t w_bar, nbr_bar[2];
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  __shared__ float sBias[NOUT];
  volatile int* abort = &abort_flag;

  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (w == kMmaW) tc::tmem_alloc(&tslot, Cfg::kTmemCols);
  if (t == 0) {
    for (int s = 0; s < SG; s++) {
      tc::mbar_init(&full_bar[s], kProd);
      tc::mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; b++) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], kEpi);
    }
    tc::mbar_init(&drain_bar, 1);
    tc::mbar_init(&w_bar, 1);
    tc::mbar_init(&nbr_bar[0], 1);
    tc::mbar_init(&nbr_bar[1], 1);
    tc::fence_mbar_init();
    abort_flag = 0;
    mbar_expect(&w_bar, Cfg::kBBytes);
    for (int off = 0; off < Cfg::kBBytes; off += 16384)
      bulk_g2s(sm + off, reinterpret_cast<const unsigned char*>(a.wimg) + off,
               (uint32_t)min(16384, Cfg::kBBytes - off), &w_bar);
  }
  if (t < NOUT) sBias[t] = a.bias ? a.bias[t] : 0.f;
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tslot;
  const int64_t n = a.n;
  const int64_t ntiles = (n + kTM - 1) / kTM;
  const int my_tiles = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  auto tile_r0 = [&](int lt) { return ((int64_t)blockIdx.x + (int64_t)lt * gridDim.x) * kTM; };

  if (w < kPWarps) {
    // ---------------------------------------------------------- producers --
    // (with one offset the gathered row is the output row itself: no map)
    constexpr int NBX = NB > 0 ? NB : 1;
    int last_issued = -1, last_used = -1;
    auto issue_nbr = [&](int lt) {
      if (KO > 1 && t == 0 && lt < my_tiles && tile_r0(lt) + kTM <= n) {
        last_issued = lt;
        tc::fence_async_smem();
        uint64_t* bar = &nbr_bar[lt % NBX];
        mbar_expect(bar, Cfg::kNbrBytes);
        bulk_g2s(sNbr0 + (lt % NBX) * kTM * KO, a.nbr + tile_r0(lt) * KO, Cfg::kNbrBytes, bar);
      }
    };
    issue_nbr(0);
    constexpr int kPer = kTM * Cfg::kChunks / kProd;
    static_assert(kPer * kProd == kTM * Cfg::kChunks, "copies must split evenly");
    int prow[kPer];
    uint32_t pdst[kPer];
    const unsigned char* psrc[kPer];
#pragma unroll
    for (int k = 0; k < kPer; k++) {
      const int q = t + k * kProd;
      const int c = q % Cfg::kChunks;
      prow[k] = q / Cfg::kChunks;
      pdst[k] = tc::swz<Cfg::SW>(prow[k] * Cfg::RB + c * 16);
      psrc[k] = reinterpret_cast<const unsigned char*>(a.xb) + c * 16;
    }
    uint32_t u = 0;
    for (int lt = 0; lt < my_tiles; lt++) {
      const int64_t r0 = tile_r0(lt);
      int32_t* sNbr = sNbr0 + (lt % NBX) * kTM * KO;
      if (producer_sync_or(*abort != 0)) break;
      if (KO > 1) {
        if (NB == 2) issue_nbr(lt + 1);
        else if (lt > 0) issue_nbr(lt);
        if (r0 + kTM <= n) {
          if (producer_sync_or(!wait_or_abort(&nbr_bar[lt % NBX], (lt / NBX) & 1, abort))) break;
          last_used = lt;
        } else {
          const int64_t base = r0 * KO, lim = n * KO;
          for (int i = t; i < kTM * KO; i += kProd)
            sNbr[i] = base + i < lim ? __ldg(a.nbr + base + i) : -1;
          producer_sync_or(false);
        }
      }
      for (int og = 0; og < KO / G; og++, u++) {
        const int sg = (int)(u % SG);
        if (u >= (uint32_t)SG && !wait_or_abort(&empty_bar[sg], ((u / SG) - 1) & 1, abort))
          break;
#pragma unroll
        for (int i = 0; i < G; i++) {
          const int o = og * G + i;
          const uint32_t sbase = tc::smem_u32(sA + (size_t)(sg * G + i) * Cfg::kStageBytes);
#pragma unroll
          for (int k = 0; k < kPer; k++) {
            const int32_t nb = KO > 1 ? sNbr[prow[k] * KO + o]
                                      : (r0 + prow[k] < n ? (int32_t)(r0 + prow[k]) : -1);
            const uint32_t r = (uint32_t)max(nb, 0);
            tc::cp_async16(sbase + pdst[k], psrc[k] + (size_t)r * Cfg::RB, nb >= 0);
          }
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(
                         tc::smem_u32(&full_bar[sg]))
                     : "memory");
      }
    }
    if (t == 0 && last_issued > last_used)
      tc::mbar_wait(&nbr_bar[last_issued % NBX], (last_issued / NBX) & 1);
    tc::cp_async_wait<0>();
  } else if (w == kMmaW) {
    // ---------------------------------------------------------------- MMA --
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16(kTM, NOUT);
      uint32_t u = 0;
      const bool wok = wait_or_abort(&w_bar, 0, abort);
      for (int lt = 0; lt < my_tiles && wok && !*abort; lt++) {
        const int b = lt & 1;
        if (lt >= 2 && !wait_or_abort(&acc_empty[b], ((lt >> 1) - 1) & 1, abort)) break;
        tc::tc_fence_after();
        const uint32_t dbase = tbase + (uint32_t)(b * NOUT);
        bool ok = true;
        for (int og = 0; og < KO / G; og++, u++) {
          const int sg = (int)(u % SG);
          if (!wait_or_abort(&full_bar[sg], (u / SG) & 1, abort)) {
            ok = false;
            break;
          }
          tc::fence_async_smem();
          tc::tc_fence_after();
#pragma unroll
          for (int i = 0; i < G; i++) {
            const int o = og * G + i;
            const uint32_t sa = tc::smem_u32(sA + (size_t)(sg * G + i) * Cfg::kStageBytes);
#pragma unroll
            for (int ks = 0; ks < CIN / 16; ks++) {
              const int k0 = o * CIN + ks * 16;
              const uint32_t sb =
                  tc::smem_u32(sB) + (k0 / 64) * Cfg::kBBlockBytes + (k0 % 64) * 2;
              tc::mma_bf16(dbase, tc::smem_desc<Cfg::SW>(sa + ks * 32, 8 * Cfg::RB),
                           tc::smem_desc<128>(sb, 1024), idesc, (o > 0 || ks > 0) ? 1u : 0u);
            }
          }
          tc::mma_commit(&empty_bar[sg]);
        }
        if (!ok) break;
        tc::mma_commit(&acc_full[b]);
      }
      tc::mma_commit(&drain_bar);
      if (!tc::mbar_wait(&drain_bar, 0)) *abort = 1;
    }
    __syncwarp();
  } else {
    // ----------------------------------------------------------- epilogue --
    const int e = t - kProd;
    const uint32_t lane_off = (uint32_t)((w & 3) * 32) << 16;
    for (int lt = 0; lt < my_tiles; lt++) {
      const int b = lt & 1;
      if constexpr (EPI == 1) {
        // output row p is a parent: its first child and the slots it has,
        // read before the accumulators are waited for
        const int64_t p = tile_r0(lt) + e;
        uint32_t c0 = 0, smask = 0;
        if (p < n) {
          c0 = __ldg(a.off + p);
          const uint32_t c1 = __ldg(a.off + p + 1);
          for (uint32_t r = c0; r < c1 && r < c0 + 8; r++) smask |= 1u << (__ldg(a.ckey + r) & 7);
        }
        if (!__all_sync(0xffffffffu, wait_or_abort(&acc_full[b], (lt >> 1) & 1, abort))) break;
        tc::tc_fence_after();
        const uint32_t dbase = tbase + lane_off + (uint32_t)(b * NOUT);
        // the TMEM loads are warp-collective (one column address a warp), so
        // every lane reads every slot and stores the ones its parent has
#pragma unroll 1
        for (int s = 0; s < 8; s++) {
          uint32_t v[2][16];
          tc::tmem_ld16_issue(dbase + s * 32, v[0]);
          tc::tmem_ld16_issue(dbase + s * 32 + 16, v[1]);
          tc::tmem_wait_ld();
          tc::tmem_regs_ready(v[0]);
          tc::tmem_regs_ready(v[1]);
          if (p < n && ((smask >> s) & 1u)) {
            const uint32_t r = c0 + __popc(smask & ((1u << s) - 1u));
            float4* dst = reinterpret_cast<float4*>(a.out + (int64_t)r * 32);
#pragma unroll
            for (int c = 0; c < 32; c += 4)
              dst[c / 4] = make_float4(__uint_as_float(v[c / 16][c % 16]) + sBias[s * 32 + c],
                                       __uint_as_float(v[c / 16][c % 16 + 1]) + sBias[s * 32 + c + 1],
                                       __uint_as_float(v[c / 16][c % 16 + 2]) + sBias[s * 32 + c + 2],
                                       __uint_as_float(v[c / 16][c % 16 + 3]) + sBias[s * 32 + c + 3]);
          }
        }
        tc::tc_fence_before();
        mbar_arrive(&acc_empty[b]);
      } else {
        if (!__all_sync(0xffffffffu, wait_or_abort(&acc_full[b], (lt >> 1) & 1, abort))) break;
        tc::tc_fence_after();
        uint32_t raw[NOUT / 16][16];
        const uint32_t dbase = tbase + lane_off + (uint32_t)(b * NOUT);
#pragma unroll
        for (int g = 0; g < NOUT / 16; g++) tc::tmem_ld16_issue(dbase + g * 16, raw[g]);
        tc::tmem_wait_ld();
#pragma unroll
        for (int g = 0; g < NOUT / 16; g++) tc::tmem_regs_ready(raw[g]);
        tc::tc_fence_before();
        mbar_arrive(&acc_empty[b]);
        const int64_t r = tile_r0(lt) + e;
        if (r < n) {
          float4* dst = reinterpret_cast<float4*>(a.out + r * NOUT);
#pragma unroll
          for (int c = 0; c < NOUT; c += 4)
            dst[c / 4] = make_float4(__uint_as_float(raw[c / 16][c % 16]) + sBias[c],
                                     __uint_as_float(raw[c / 16][c % 16 + 1]) + sBias[c + 1],
                                     __uint_as_float(raw[c / 16][c % 16 + 2]) + sBias[c + 2],
                                     __uint_as_float(raw[c / 16][c % 16 + 3]) + sBias[c + 3]);
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (t == kThr - 32) tc::mbar_wait(&w_bar, 0);
  if (w == kMmaW) tc::tmem_dealloc(tbase, Cfg::kTmemCols);
  if (t == 0 && abort_flag) atomicExch(&g_tconv_error, 1);
}

// ---- backward: weight gradients, and input gradients from the same gather ---
// dW[o] = sum over rows m of G_o[m]^T Y[m] for every offset o, G_o[m] the
// gathered 32-wide bf16 row of offset o (zero where absent), Y[m] the row's
// own NY-wide bf16 row:
//  - conv: G_o[m] = dy[nbr[m][o]], Y = x, into dW[26 - o][co][ci] (the kernel
//    map is symmetric: nbr[m][o] = r exactly when nbr[r][26 - o] = m);
//  - up-step: rows are parents, G_s[p] = dy[p's child in slot s], Y = x, into
//    dW[s][co][ci];
//  - down-step: rows are parents, G_s[p] = x[p's child in slot s], Y = dy,
//    into dW[s][co][ci] (the gathered channel is ci).
// Four offsets' stages lie side by side in shared memory, so an MN-major
// descriptor reads them as the A operand of one MMA (M = 4 offsets x 32
// channels) per 16 rows against the MN-major Y tile (N = NY); every
// offset's accumulator stays in tensor memory across the CTA's tiles and is
// added into dW once at the end.  With DX the same stages also give the
// input gradient as in k_tconv_tc (K-major A, the weight image as B), so the
// conv's and the up-step's dx and dW share one gather.
template <int NY, int KO, bool DX>
struct BCfg {
  static constexpr int RB = 64;  // gathered rows: 32 bf16, 64-byte swizzle
  static constexpr int G = 4;    // offsets a pipeline step: one 128-row M group
  static constexpr int kSteps = (KO + G - 1) / G;
  static constexpr int kStageBytes = kTM * RB;
  static constexpr int SG = (NY == 64 && KO == 27 && DX) ? 2 : 3;  // ring depth in steps
  static constexpr int YRB = NY * 2, YSW = NY == 64 ? 128 : 64;
  static constexpr int kYBytes = kTM * YRB;
  static constexpr int kBBlocks = DX ? (KO * 32 + 63) / 64 : 0;
  static constexpr int kBBlockBytes = NY * 128;
  static constexpr int kBBytes = kBBlocks * kBBlockBytes;
  static constexpr int kNbrBufs = (NY == 64 && KO == 27 && DX) ? 1 : 2;
  static constexpr int kNbrBytes = kTM * KO * 4;
  static constexpr int kDwCols = kSteps * NY;
  static constexpr int kDxBufs = DX ? (kDwCols + 2 * NY <= 512 ? 2 : 1) : 0;
  static constexpr int kNeed = kDwCols + kDxBufs * NY;
  static constexpr int kTmemCols =
      kNeed <= 64 ? 64 : (kNeed <= 128 ? 128 : (kNeed <= 256 ? 256 : 512));
  static constexpr size_t kSmem = 1024 + kBBytes + (size_t)SG * G * kStageBytes + 2 * kYBytes +
                                  (size_t)kNbrBufs * kNbrBytes;
  static_assert(kNeed <= 512, "tensor memory of a backward variant exceeds 512 columns");
  static_assert(kSmem <= 232448 - 512, "shared memory of a backward variant exceeds the limit");
  static_assert(kTM * 4 == 2 * kProd && kTM * (YRB / 16) % kProd == 0, "copies split evenly");
};

struct TBwdArgs {
  const __nv_bfloat16* gb;  // gathered rows [][32], bf16
  const __nv_bfloat16* yb;  // the rows' own [n][NY], bf16
  const int32_t* map;       // [n][KO]: the gathered row of each offset, -1 absent
  int64_t n;
  const uint16_t* wimg;     // DX: weight image of the input gradient
  float* dx;                // DX: [n][NY]
  float* dw;                // [KO][32][NY] (trans) or [KO][NY][32], accumulated into
  int mirror;               // dW slice KO - 1 - o instead of o
  int trans;                // the gathered channel indexes W's rows (else its columns)
  int vec4;                 // dw is 16-byte aligned
};

template <int NY, int KO, bool DX>
__global__ void __launch_bounds__(kThr, 1) k_tbwd_tc(TBwdArgs a) {
  using Cfg = BCfg<NY, KO, DX>;
  constexpr int G = Cfg::G, SG = Cfg::SG, NB = Cfg::kNbrBufs, KS = Cfg::kSteps;
  constexpr int XB = Cfg::kDxBufs > 0 ? Cfg::kDxBufs : 1;
  extern __shared__ unsigned char smraw[];
  // aligned to 1024 by offsetting smraw itself, so that accesses through sm
  // stay shared-memory accesses (an integer round trip would make them generic)
  unsigned char* sm = smraw + ((1024u - (tc::smem_u32(smraw) & 1023u)) & 1023u);
  // ring first, the Y tiles right after it, then the weight image and maps
  unsigned char* sA = sm;
  unsigned char* sY = sA + (size_t)SG * G * Cfg::kStageBytes;
  unsigned char* sB = sY + 2 * Cfg::kYBytes;
  int32_t* sNbr0 = reinterpret_cast<int32_t*>(sB + Cfg::kBBytes);
  __shared__ uint64_t full_bar[SG], empty_bar[SG], acc_full[2], acc_empty[2], y_full[2],
      y_empty[2], dw_bar, drain_bar, w_bar, nbr_bar[2];
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  volatile int* abort = &abort_flag;

  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (w == kMmaW) tc::tmem_alloc(&tslot, Cfg::kTmemCols);
  if (t == 0) {
    for (int s = 0; s < SG; s++) {
      tc::mbar_init(&full_bar[s], kProd);
      tc::mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; b++) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], kEpi);
      tc::mbar_init(&y_full[b], kProd);
      tc::mbar_init(&y_empty[b], 1);
      tc::mbar_init(&nbr_bar[b], 1);
    }
    tc::mbar_init(&dw_bar, 1);
    tc::mbar_init(&drain_bar, 1);
    tc::mbar_init(&w_bar, 1);
    tc::fence_mbar_init();
    abort_flag = 0;
    if (DX) {
      mbar_expect(&w_bar, Cfg::kBBytes);
      for (int off = 0; off < Cfg::kBBytes; off += 16384)
        bulk_g2s(sB + off, reinterpret_cast<const unsigned char*>(a.wimg) + off,
                 (uint32_t)min(16384, Cfg::kBBytes - off), &w_bar);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tslot;
  const int64_t n = a.n;
  const int64_t ntiles = (n + kTM - 1) / kTM;
  const int my_tiles = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  auto tile_r0 = [&](int lt) { return ((int64_t)blockIdx.x + (int64_t)lt * gridDim.x) * kTM; };

  if (w < kPWarps) {
    // ---------------------------------------------------------- producers --
    int last_issued = -1, last_used = -1;
    auto issue_nbr = [&](int lt) {
      if (t == 0 && lt < my_tiles && tile_r0(lt) + kTM <= n) {
        last_issued = lt;
        tc::fence_async_smem();
        uint64_t* bar = &nbr_bar[lt % NB];
        mbar_expect(bar, Cfg::kNbrBytes);
        bulk_g2s(sNbr0 + (lt % NB) * kTM * KO, a.map + tile_r0(lt) * KO, Cfg::kNbrBytes, bar);
      }
    };
    issue_nbr(0);
    constexpr int kPer = kTM * 4 / kProd;             // gathered copies a thread, per offset
    constexpr int kYPer = kTM * (Cfg::YRB / 16) / kProd;  // Y copies a thread, per tile
    int prow[kPer];
    uint32_t pdst[kPer];
    const unsigned char* psrc[kPer];
#pragma unroll
    for (int k = 0; k < kPer; k++) {
      const int q = t + k * kProd;
      prow[k] = q >> 2;
      pdst[k] = tc::swz<64>(prow[k] * 64 + (q & 3) * 16);
      psrc[k] = reinterpret_cast<const unsigned char*>(a.gb) + (q & 3) * 16;
    }
    uint32_t u = 0;
    for (int lt = 0; lt < my_tiles; lt++) {
      const int64_t r0 = tile_r0(lt);
      int32_t* sNbr = sNbr0 + (lt % NB) * kTM * KO;
      if (producer_sync_or(*abort != 0)) break;
      // the tile's own rows (zero past the end)
      const int yb = lt & 1;
      if (lt < 2 || wait_or_abort(&y_empty[yb], ((lt >> 1) - 1) & 1, abort)) {
        const uint32_t ybase = tc::smem_u32(sY + (size_t)yb * Cfg::kYBytes);
#pragma unroll
        for (int k = 0; k < kYPer; k++) {
          const int q = t + k * kProd;
          const int row = q / (Cfg::YRB / 16), c = q % (Cfg::YRB / 16);
          const bool in = r0 + row < n;
          tc::cp_async16(ybase + tc::swz<Cfg::YSW>(row * Cfg::YRB + c * 16),
                         reinterpret_cast<const unsigned char*>(a.yb) +
                             (in ? (r0 + row) * Cfg::YRB : 0) + c * 16,
                         in);
        }
      }
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(
                       tc::smem_u32(&y_full[yb]))
                   : "memory");
      if (NB == 2) issue_nbr(lt + 1);
      else if (lt > 0) issue_nbr(lt);
      if (r0 + kTM <= n) {
        if (producer_sync_or(!wait_or_abort(&nbr_bar[lt % NB], (lt / NB) & 1, abort))) break;
        last_used = lt;
      } else {
        const int64_t base = r0 * KO, lim = n * KO;
        for (int i = t; i < kTM * KO; i += kProd)
          sNbr[i] = base + i < lim ? __ldg(a.map + base + i) : -1;
        producer_sync_or(false);
      }
      for (int st = 0; st < KS; st++, u++) {
        const int sg = (int)(u % SG);
        if (u >= (uint32_t)SG && !wait_or_abort(&empty_bar[sg], ((u / SG) - 1) & 1, abort))
          break;
#pragma unroll
        for (int i = 0; i < G; i++) {
          const int o = st * G + i;
          if (o >= KO) break;  // a padding offset: its M rows are never read out
          const uint32_t sbase = tc::smem_u32(sA + (size_t)(sg * G + i) * Cfg::kStageBytes);
#pragma unroll
          for (int k = 0; k < kPer; k++) {
            const int32_t nb = sNbr[prow[k] * KO + o];
            const uint32_t r = (uint32_t)max(nb, 0);
            tc::cp_async16(sbase + pdst[k], psrc[k] + (size_t)r * 64, nb >= 0);
          }
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(
                         tc::smem_u32(&full_bar[sg]))
                     : "memory");
      }
    }
    if (t == 0 && last_issued > last_used)
      tc::mbar_wait(&nbr_bar[last_issued % NB], (last_issued / NB) & 1);
    tc::cp_async_wait<0>();
  } else if (w == kMmaW) {
    // ---------------------------------------------------------------- MMA --
    if (lane == 0) {
      constexpr uint32_t idesc_dx = tc::idesc_bf16(kTM, NY);
      constexpr uint32_t idesc_dw = tc::idesc_bf16_mn(kTM, NY);
      constexpr uint32_t ysbo = 8 * Cfg::YRB;  // 8 rows of Y
      uint32_t u = 0;
      bool ok = DX ? wait_or_abort(&w_bar, 0, abort) : true;
      for (int lt = 0; lt < my_tiles && ok && !*abort; lt++) {
        const int yb = lt & 1, b = DX ? lt % XB : 0;
        if (!wait_or_abort(&y_full[yb], (lt >> 1) & 1, abort)) break;
        if (DX && lt >= XB && !wait_or_abort(&acc_empty[b], ((lt / XB) - 1) & 1, abort)) break;
        tc::tc_fence_after();
        const uint32_t ya = tc::smem_u32(sY + (size_t)yb * Cfg::kYBytes);
        const uint32_t dxacc = tbase + (uint32_t)(Cfg::kDwCols + b * NY);
        for (int st = 0; st < KS; st++, u++) {
          const int sg = (int)(u % SG);
          if (!wait_or_abort(&full_bar[sg], (u / SG) & 1, abort)) {
            ok = false;
            break;
          }
          tc::fence_async_smem();
          tc::tc_fence_after();
          const uint32_t s0 = tc::smem_u32(sA + (size_t)sg * G * Cfg::kStageBytes);
          if (DX) {
#pragma unroll
            for (int i = 0; i < G; i++) {
              const int o = st * G + i;
              if (o >= KO) break;
#pragma unroll
              for (int ks = 0; ks < 2; ks++) {
                const int k0 = o * 32 + ks * 16;
                const uint32_t sb =
                    tc::smem_u32(sB) + (k0 / 64) * Cfg::kBBlockBytes + (k0 % 64) * 2;
                tc::mma_bf16(dxacc,
                             tc::smem_desc<64>(s0 + i * Cfg::kStageBytes + ks * 32, 8 * 64),
                             tc::smem_desc<128>(sb, 1024), idesc_dx, (o > 0 || ks > 0) ? 1u : 0u);
              }
            }
          }
          // dW: the step's four stages (M = 4 x 32, MN-major, atoms one stage
          // apart) against the tile's Y rows, 16 rows an MMA
#pragma unroll
          for (int ks = 0; ks < kTM / 16; ks++)
            tc::mma_bf16(tbase + (uint32_t)(st * NY),
                         tc::smem_desc_mn<64>(s0 + ks * 2 * 8 * 64, Cfg::kStageBytes, 8 * 64),
                         tc::smem_desc_mn<Cfg::YSW>(ya + ks * 2 * ysbo, ysbo, ysbo), idesc_dw,
                         (lt > 0 || ks > 0) ? 1u : 0u);
          tc::mma_commit(&empty_bar[sg]);
        }
        if (!ok) break;
        tc::mma_commit(&y_empty[yb]);
        if (DX) tc::mma_commit(&acc_full[b]);
      }
      tc::mma_commit(&dw_bar);
      tc::mma_commit(&drain_bar);
      if (!tc::mbar_wait(&drain_bar, 0)) *abort = 1;
    }
    __syncwarp();
  } else {
    // ----------------------------------------------------------- epilogue --
    const int e = t - kProd;
    const uint32_t lane_off = (uint32_t)((w & 3) * 32) << 16;
    bool live = true;
    if (DX) {
      for (int lt = 0; lt < my_tiles; lt++) {
        const int b = lt % XB;
        if (!__all_sync(0xffffffffu, wait_or_abort(&acc_full[b], (lt / XB) & 1, abort))) {
          live = false;
          break;
        }
        tc::tc_fence_after();
        uint32_t raw[NY / 16][16];
        const uint32_t dbase = tbase + lane_off + (uint32_t)(Cfg::kDwCols + b * NY);
#pragma unroll
        for (int g = 0; g < NY / 16; g++) tc::tmem_ld16_issue(dbase + g * 16, raw[g]);
        tc::tmem_wait_ld();
#pragma unroll
        for (int g = 0; g < NY / 16; g++) tc::tmem_regs_ready(raw[g]);
        tc::tc_fence_before();
        mbar_arrive(&acc_empty[b]);
        const int64_t r = tile_r0(lt) + e;
        if (r < n) {
          float4* dst = reinterpret_cast<float4*>(a.dx + r * NY);
#pragma unroll
          for (int c = 0; c < NY; c += 4)
            dst[c / 4] = make_float4(__uint_as_float(raw[c / 16][c % 16]),
                                     __uint_as_float(raw[c / 16][c % 16 + 1]),
                                     __uint_as_float(raw[c / 16][c % 16 + 2]),
                                     __uint_as_float(raw[c / 16][c % 16 + 3]));
        }
      }
    }
    // dW: the warp's 32 TMEM lanes are offset 4 g + (w & 3) of group g, one
    // lane per gathered channel
    if (live && my_tiles > 0 &&
        __all_sync(0xffffffffu, wait_or_abort(&dw_bar, 0, abort)) && !*abort) {
      tc::tc_fence_after();
      const int q = w & 3;
#pragma unroll 1
      for (int g = 0; g < KS; g++) {
        const int o = g * G + q;
        if (o >= KO) break;
        uint32_t raw[NY / 16][16];
        const uint32_t dbase = tbase + lane_off + (uint32_t)(g * NY);
#pragma unroll
        for (int h = 0; h < NY / 16; h++) tc::tmem_ld16_issue(dbase + h * 16, raw[h]);
        tc::tmem_wait_ld();
#pragma unroll
        for (int h = 0; h < NY / 16; h++) tc::tmem_regs_ready(raw[h]);
        const int so = a.mirror ? KO - 1 - o : o;
        if (a.trans) {
          float* dst = a.dw + ((size_t)so * 32 + lane) * NY;
          if (a.vec4) {
#pragma unroll
            for (int c = 0; c < NY; c += 4)
              atomicAdd(reinterpret_cast<float4*>(dst + c),
                        make_float4(__uint_as_float(raw[c / 16][c % 16]),
                                    __uint_as_float(raw[c / 16][c % 16 + 1]),
                                    __uint_as_float(raw[c / 16][c % 16 + 2]),
                                    __uint_as_float(raw[c / 16][c % 16 + 3])));
          } else {
#pragma unroll
            for (int c = 0; c < NY; c++) atomicAdd(dst + c, __uint_as_float(raw[c / 16][c % 16]));
          }
        } else {
          float* dst = a.dw + (size_t)so * NY * 32 + lane;
#pragma unroll
          for (int c = 0; c < NY; c++)
            atomicAdd(dst + (size_t)c * 32, __uint_as_float(raw[c / 16][c % 16]));
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (DX && t == kThr - 32) tc::mbar_wait(&w_bar, 0);
  if (w == kMmaW) tc::tmem_dealloc(tbase, Cfg::kTmemCols);
  if (t == 0 && abort_flag) atomicExch(&g_tconv_error, 1);
}

// float rows -> bf16 rows (round to nearest even), n x cols
__global__ void k_f32_to_bf16(const float* __restrict__ x, int64_t count, __nv_bfloat16* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count / 4;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = reinterpret_cast<const float4*>(x)[i];
    __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
    reinterpret_cast<__nv_bfloat162*>(out)[2 * i] = lo;
    reinterpret_cast<__nv_bfloat162*>(out)[2 * i + 1] = hi;
  }
}

// Weight image of the gather-GEMM (K-major, 64-element blocks of nout rows x
// 128 bytes, 128-byte swizzled) from W [S][cout][cin]; k = o kper + kk:
//  mode 0, gather forward: row n = output channel, value W[o][n][kk];
//  mode 1, the conv's input gradient: row n = ci, value W[26 - o][kk][n];
//  mode 2, gather transposed (the up-step's input gradient): W[o][kk][n];
//  mode 3, expand (the up-step forward, one offset): row n = s cout + co,
//          value W[s][co][kk];
//  mode 4, expand transposed (the down-step's input gradient): row n =
//          s cin + ci, value W[s][kk][ci].
__global__ void k_pack_tw(const float* __restrict__ W, int cout, int cin, int mode, int ko,
                          int kper, int nout, unsigned char* img) {
  const int64_t total = (int64_t)ko * kper * nout;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int nrow = (int)(idx % nout);
    const int k = (int)(idx / nout);
    const int o = k / kper, kk = k % kper;
    float v;
    if (mode == 0) v = W[((size_t)o * cout + nrow) * cin + kk];
    else if (mode == 1) v = W[((size_t)(26 - o) * cout + kk) * cin + nrow];
    else if (mode == 2) v = W[((size_t)o * cout + kk) * cin + nrow];
    else if (mode == 3) v = W[((size_t)(nrow / cout) * cout + nrow % cout) * cin + kk];
    else v = W[((size_t)(nrow / cin) * cout + kk) * cin + nrow % cin];
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    const int blk = k / 64, kb = k % 64;
    uint32_t off = (uint32_t)(nrow * 128 + kb * 2);
    off ^= ((off >> 7) & 7) << 4;
    *reinterpret_cast<__nv_bfloat16*>(img + (size_t)blk * nout * 128 + off) = b;
  }
}

// A parent's eight child slots: smap[p][s] = its child in slot s, else -1.
__global__ void k_slot_map(const uint32_t* __restrict__ off, const uint64_t* __restrict__ ckey,
                           int64_t np, int32_t* smap) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
       p += (int64_t)gridDim.x * blockDim.x) {
    int32_t m[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    const uint32_t c1 = off[p + 1];
    for (uint32_t r = off[p]; r < c1; r++) m[ckey[r] & 7] = (int32_t)r;
#pragma unroll
    for (int s = 0; s < 8; s++) smap[p * 8 + s] = m[s];
  }
}

// Growable device scratch for the bf16 rows and the weight image (allocated
// on the first calls and on growth only).
struct Scratch {
  std::mutex mu;
  void* p = nullptr;
  size_t cap = 0;
};
Scratch g_rows, g_img;

void* grow(Scratch& s, size_t bytes) {
  std::lock_guard<std::mutex> g(s.mu);
  if (bytes <= s.cap) return s.p;
  if (s.p) cudaFree(s.p);
  s.cap = std::max<size_t>(bytes + bytes / 4, 1 << 16);
  if (cudaMalloc(&s.p, s.cap) != cudaSuccess) {
    cudaGetLastError();
    s.p = nullptr;
    s.cap = 0;
  }
  return s.p;
}

Scratch g_smap;

template <int CIN, int NOUT, int KO, int EPI>
int launch(const TConvArgs& a, cudaStream_t st) {
  using Cfg = TCfg<CIN, NOUT, KO>;
  const int64_t ntiles = (a.n + kTM - 1) / kTM;
  const int blocks = (int)std::min<int64_t>(ntiles, 148);
  auto* k = k_tconv_tc<CIN, NOUT, KO, EPI>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem);
  k<<<blocks, kThr, Cfg::kSmem, st>>>(a);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? LPC_OK : LPC_CUDA_ERROR;
}

// The float input rows as bf16 and the weight image (mode, ko offsets of
// kper, nout rows) in scratch; returns false if scratch is missing.
bool stage_inputs(const float* in, int64_t rows, int gw, const float* W, int cout, int cin,
                  int mode, int ko, int nout, void** xb, void** img, cudaStream_t st) {
  const size_t img_bytes = (size_t)((ko * gw + 63) / 64) * nout * 128;
  *xb = grow(g_rows, (size_t)std::max<int64_t>(rows * gw * 2, 16));
  *img = grow(g_img, img_bytes);
  if (!*xb || !*img) return false;
  const int64_t cnt = rows * gw;
  if (cnt > 0)
    k_f32_to_bf16<<<(int)std::min<int64_t>((cnt / 4 + 255) / 256, 148 * 8), 256, 0, st>>>(
        in, cnt, static_cast<__nv_bfloat16*>(*xb));
  cudaMemsetAsync(*img, 0, img_bytes, st);
  k_pack_tw<<<(int)std::min<int64_t>(((int64_t)ko * gw * nout + 255) / 256, 148 * 4), 256, 0,
              st>>>(W, cout, cin, mode, ko, gw, nout, static_cast<unsigned char*>(*img));
  count_launches(2);
  return true;
}

template <int NY, int KO, bool DX>
int launch_bwd(const TBwdArgs& a, cudaStream_t st) {
  using Cfg = BCfg<NY, KO, DX>;
  const int64_t ntiles = (a.n + kTM - 1) / kTM;
  const int blocks = (int)std::min<int64_t>(ntiles, 148);
  auto* k = k_tbwd_tc<NY, KO, DX>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem);
  k<<<blocks, kThr, Cfg::kSmem, st>>>(a);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? LPC_OK : LPC_CUDA_ERROR;
}

Scratch g_rows_y;

// cnt floats (a multiple of 4) as bf16 in scratch s, or null
void* bf16_copy(Scratch& s, const float* in, int64_t cnt, cudaStream_t st) {
  void* p = grow(s, (size_t)std::max<int64_t>(cnt * 2, 16));
  if (p && cnt > 0) {
    k_f32_to_bf16<<<(int)std::min<int64_t>((cnt / 4 + 255) / 256, 148 * 8), 256, 0, st>>>(
        in, cnt, static_cast<__nv_bfloat16*>(p));
    count_launches(1);
  }
  return p;
}

// dW (and dx when given) of one sparse op from one gather: gsrc [gn][32] the
// gathered rows, ysrc [n][ny] the rows' own, map [n][ko]; the weight image
// of dx from W [ko][cout][cin] in k_pack_tw's mode wmode.
int tbwd(const float* gsrc, int64_t gn, const float* ysrc, int64_t n, int ny, const int32_t* map,
         int ko, const float* W, int cout, int cin, int wmode, float* dx, float* dW, int mirror,
         int trans, cudaStream_t st) {
  if (n <= 0) return LPC_OK;
  void* gb = bf16_copy(g_rows, gsrc, gn * 32, st);
  void* yb = bf16_copy(g_rows_y, ysrc, n * ny, st);
  if (!gb || !yb) return LPC_CUDA_ERROR;
  void* img = nullptr;
  if (dx) {
    const size_t img_bytes = (size_t)((ko * 32 + 63) / 64) * ny * 128;
    img = grow(g_img, img_bytes);
    if (!img) return LPC_CUDA_ERROR;
    cudaMemsetAsync(img, 0, img_bytes, st);
    k_pack_tw<<<(int)std::min<int64_t>(((int64_t)ko * 32 * ny + 255) / 256, 148 * 4), 256, 0,
                st>>>(W, cout, cin, wmode, ko, 32, ny, static_cast<unsigned char*>(img));
    count_launches(1);
  }
  const TBwdArgs a{static_cast<const __nv_bfloat16*>(gb), static_cast<const __nv_bfloat16*>(yb),
                   map, n, static_cast<const uint16_t*>(img), dx, dW, mirror, trans,
                   (reinterpret_cast<uintptr_t>(dW) & 15) == 0};
#define LPC_BWD(NY_, KO_)                                                 \
  if (ny == NY_ && ko == KO_)                                             \
    return dx ? launch_bwd<NY_, KO_, true>(a, st) : launch_bwd<NY_, KO_, false>(a, st);
  LPC_BWD(32, 27)
  LPC_BWD(64, 27)
  LPC_BWD(32, 8)
  LPC_BWD(64, 8)
#undef LPC_BWD
  return LPC_INVALID_ARG;
}

// the parents' slot map [np][8] in scratch, or null
int32_t* slot_map(const uint32_t* off, const uint64_t* ckey, int64_t np, cudaStream_t st) {
  auto* smap = static_cast<int32_t*>(grow(g_smap, (size_t)np * 8 * 4));
  if (smap) {
    k_slot_map<<<(int)std::min<int64_t>((np + 255) / 256, 148 * 8), 256, 0, st>>>(off, ckey, np,
                                                                                   smap);
    count_launches(1);
  }
  return smap;
}

}  // namespace

// The conv's backward in bf16 mode: dW [27][32][cin] (accumulated) and, with
// dx, dx [n][cin], from one gather of the rounded dy rows.
int tconv_bwd_tc(const float* x, const float* dy, int64_t n, int cin, const int32_t* nbr,
                 const float* W, float* dx, float* dW, cudaStream_t st) {
  if (cin != 32 && cin != 64) return LPC_INVALID_ARG;
  return tbwd(dy, n, x, n, cin, nbr, 27, W, 32, cin, 1, dx, dW, 1, 1, st);
}

// The up-step's backward in bf16 mode (cout 32): dW [8][32][cin] and, with
// dx, the parents' dx [np][cin], from one gather of the children's dy by slot.
int tup_bwd_tc(const float* x, const float* dy, int64_t np, int64_t nc, int cin,
               const uint32_t* off, const uint64_t* ckey, const float* W, float* dx, float* dW,
               cudaStream_t st) {
  if (np <= 0) return LPC_OK;
  if (cin != 32 && cin != 64) return LPC_INVALID_ARG;
  int32_t* smap = slot_map(off, ckey, np, st);
  if (!smap) return LPC_CUDA_ERROR;
  return tbwd(dy, nc, x, np, cin, smap, 8, W, 32, cin, 2, dx, dW, 0, 1, st);
}

// The down-step's weight gradient in bf16 mode (cin 32): dW [8][cout][32]
// from the children's x gathered by slot against the parents' dy.
int tdown_dw_tc(const float* x, const float* dy, int64_t np, int64_t nc, int cout,
                const uint32_t* off, const uint64_t* ckey, float* dW, cudaStream_t st) {
  if (np <= 0) return LPC_OK;
  if (cout != 32 && cout != 64) return LPC_INVALID_ARG;
  int32_t* smap = slot_map(off, ckey, np, st);
  if (!smap) return LPC_CUDA_ERROR;
  return tbwd(x, nc, dy, np, cout, smap, 8, nullptr, cout, 32, 0, nullptr, dW, 0, 0, st);
}

// bf16-mode forward (mirror 0: x [n][cin] -> y [n][32]) or input gradient
// (mirror 1: dy [n][32] -> dx [n][cin]) of the 3x3x3 conv on tcgen05.
int tconv_tc(const float* in, int64_t n, int cin, const int32_t* nbr, const float* W,
             const float* bias, float* out, int mirror, cudaStream_t st) {
  if (n <= 0) return LPC_OK;
  const int gw = mirror ? 32 : cin;    // gathered row width
  const int nout = mirror ? cin : 32;  // output width
  void *xb, *img;
  if (!stage_inputs(in, n, gw, W, 32, cin, mirror ? 1 : 0, 27, nout, &xb, &img, st))
    return LPC_CUDA_ERROR;
  const TConvArgs a{static_cast<const __nv_bfloat16*>(xb), nbr, n,
                    static_cast<const uint16_t*>(img), bias, out, nullptr, nullptr};
  if (gw == 64) return launch<64, 32, 27, 0>(a, st);
  if (nout == 64) return launch<32, 64, 27, 0>(a, st);
  return launch<32, 32, 27, 0>(a, st);
}

// Parents from their eight child slots: the down-step forward (transpose 0:
// child rows x [][cin] -> y [np][cout], bias [cout]) or the up-step's input
// gradient (transpose 1: child rows dy [][cout] -> dx [np][cin]); W is
// [8][cout][cin], off / ckey the parents' first children and the children's
// keys (slot = ckey & 7).
int tslot_tc(const float* in, int64_t np, int64_t nc, const uint32_t* off, const uint64_t* ckey,
             const float* W, int cout, int cin, const float* bias, float* out, int transpose,
             cudaStream_t st) {
  if (np <= 0) return LPC_OK;
  const int gw = transpose ? cout : cin, nout = transpose ? cin : cout;
  if (gw != 32 || (nout != 32 && nout != 64)) return LPC_INVALID_ARG;
  auto* smap = static_cast<int32_t*>(grow(g_smap, (size_t)np * 8 * 4));
  void *xb, *img;
  if (!smap || !stage_inputs(in, nc, gw, W, cout, cin, transpose ? 2 : 0, 8, nout, &xb, &img, st))
    return LPC_CUDA_ERROR;
  k_slot_map<<<(int)std::min<int64_t>((np + 255) / 256, 148 * 8), 256, 0, st>>>(off, ckey, np, smap);
  count_launches(1);
  const TConvArgs a{static_cast<const __nv_bfloat16*>(xb), smap, np,
                    static_cast<const uint16_t*>(img), bias, out, nullptr, nullptr};
  if (nout == 64) return launch<32, 64, 8, 0>(a, st);
  return launch<32, 32, 8, 0>(a, st);
}

// Children from their parent's row: the up-step forward (transpose 0:
// parent rows x [np][cin] -> y [children][cout], per-slot bias [8][cout])
// or the down-step's input gradient (transpose 1: parent rows dy [np][cout]
// -> dx [children][cin]).  One GEMM of every parent against all eight
// slots' weights (N = 256), each child taking its slot's 32 columns.
int texpand_tc(const float* in, int64_t np, const uint32_t* off, const uint64_t* ckey,
               const float* W, int cout, int cin, const float* slot_bias, float* out,
               int transpose, cudaStream_t st) {
  if (np <= 0) return LPC_OK;
  const int gw = transpose ? cout : cin, per_child = transpose ? cin : cout;
  if (per_child != 32 || (gw != 32 && gw != 64)) return LPC_INVALID_ARG;
  void *xb, *img;
  if (!stage_inputs(in, np, gw, W, cout, cin, transpose ? 4 : 3, 1, 256, &xb, &img, st))
    return LPC_CUDA_ERROR;
  const TConvArgs a{static_cast<const __nv_bfloat16*>(xb), nullptr, np,
                    static_cast<const uint16_t*>(img), slot_bias, out, off, ckey};
  if (gw == 64) return launch<64, 256, 1, 1>(a, st);
  return launch<32, 256, 1, 1>(a, st);
}

}  // namespace lpc

extern "C" int lpc_t_tc_error(int reset) {
  int e = 0;
  cudaMemcpyFromSymbol(&e, lpc::g_tconv_error, sizeof(int));
  if (reset && e) {
    const int z = 0;
    cudaMemcpyToSymbol(lpc::g_tconv_error, &z, sizeof(int));
  }
  return e;
}
