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
// Warp-specialised and persistent: one CTA per SM walks its tiles of 128
// output nodes (Morton order) and, for each, all 27 offsets.
//  - 8 producer warps gather, for each (tile, offset), the 128 neighbour rows
//    (pre-subtracted bf16 rows, 16-byte cp.async copies, zero-filled when the
//    neighbour is absent: the exact zero padding of the sparse conv) into a
//    ring of swizzled stages (the 32-channel conv fills three offsets' stages
//    per pipeline step).  Each thread's copies of a step arrive on the
//    step's "full" barrier by themselves when they land
//    (cp.async.mbarrier.arrive), so producers never wait on their own copies;
//    the MMA thread fences the landed stage to the async proxy.
//  - 1 MMA warp: one thread waits for a full stage and issues the M=128,
//    N=32, K=16 MMAs into the offset's accumulator; tcgen05.commit releases
//    the stage ("empty" barrier) when they are done, and after the tile's
//    last offset signals the accumulator buffer full.
//  - 4 epilogue warps (one per TMEM lane quadrant, one output row a thread)
//    read the accumulators, add them in INT32 with the bias, apply the PReLU
//    and the fixed-point requantisation (Eq. 14) and the fused residual merge
//    of the ResBlock, write int8 (and optionally the next conv's bf16 input),
//    and hand the buffer back.  Two accumulator buffers let the epilogue of
//    one tile overlap the MMAs of the next.
// The weights of all 27 offsets stay in shared memory (bf16, 128-byte
// swizzled K-major).  Every wait is bounded; a wait that gives up raises a
// shared abort flag that ends every other wait, and the CTA drains its own
// copies and MMAs before it frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>

#include <string.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "tc_util.cuh"

namespace lpc {

namespace {

constexpr int kTileM = kConvTile;  // the tiles of the kernel map's present-offset masks
constexpr int kEpilogue = 128;  // 4 warps after the producers (TMEM quadrants w % 4)

// Thread roles of the two gather schedules: 8 producer warps of cp.async
// copies (GATHER 0), or one producer warp of TMA gather4 loads (GATHER 1);
// then the 4 epilogue warps and the MMA warp.
template <int GATHER>
struct Roles {
  static constexpr int kProdWarps = GATHER ? 1 : 8;  // warps 0 .. kProdWarps-1
  static constexpr int kProducers = 32 * kProdWarps;
  static constexpr int kMmaWarp = kProdWarps + 4;
  static constexpr int kThreads = kProducers + kEpilogue + 32;
};

// Variants the autotuner chooses from: the stage-ring depth and the order in
// which a CTA walks its tiles (strided over the grid, or one contiguous run
// of Morton-adjacent tiles, whose neighbour rows overlap in L2).
// Ring shapes the autotuner chooses from (alt = 0 / 1): stages, offsets per
// pipeline step, neighbour-map buffers.  32 channels: 12 stages in steps of
// three with the map a tile ahead, or 18 stages in steps of nine with one map
// buffer; 64 channels (its weights take half the shared memory): 6 stages in
// steps of three, one map buffer.
template <int CIN>
constexpr int stages_of(int alt) {
  return CIN == 64 ? 6 : (alt ? 18 : 12);
}
template <int CIN>
constexpr int step_of(int alt) {
  return CIN == 64 ? 3 : (alt ? 9 : 3);
}
template <int CIN>
constexpr int nbr_bufs_of(int alt) {
  return CIN == 64 ? 1 : (alt ? 1 : 2);
}

// Tall tiles (256 rows, 32 channels only: two 128-row MMAs per offset into
// the two halves of a 256-column accumulator buffer) halve the tile count
// and with it the per-tile work (map copy, masks, barrier round trips,
// accumulator hand-over) per row; their ring: 6 stages of 256 rows in steps
// of three, the map a tile ahead.
constexpr int kTallRows = 256;
constexpr int kTallStages = 6, kTallStep = 3, kTallNbrBufs = 2;

template <int CIN, int S_ = stages_of<CIN>(0), int G_ = step_of<CIN>(0),
          int NB_ = nbr_bufs_of<CIN>(0), int TM_ = kTileM>
struct ConvCfg {
  static constexpr int TM = TM_;                     // rows of a tile
  static constexpr int RB = CIN * 2;                 // bf16 row bytes
  static constexpr int SW = CIN == 64 ? 128 : 64;    // swizzle of the A stage
  static constexpr int kStages = S_;
  // offsets per pipeline step: their rows share one barrier round trip (one
  // wait, one arrival, one commit)
  static constexpr int kG = G_;
  // neighbour-map buffers: two (the next tile's map loads a tile ahead) or
  // one (loaded at the tile's start; leaves room for more stages)
  static constexpr int kNbrBufs = NB_;
  static_assert(kStages % kG == 0 && 27 % kG == 0, "stage groups must tile the ring and offsets");
  static constexpr int kStageBytes = TM * RB;
  static constexpr int kPerGroup = 256 / CIN;        // offsets per fp32 accumulator
  static constexpr int kGroups = (27 + kPerGroup - 1) / kPerGroup;
  static constexpr int kBufCols = 256;               // TMEM columns per accumulator buffer
  static constexpr int kBBlocks = (27 * CIN + 63) / 64;
  static constexpr int kBBytes = kBBlocks * 4096;
  static constexpr int kChunks = RB / 16;            // 16-byte chunks per row
  static constexpr int kNbrBytes = TM * 27 * 4;      // a tile's neighbour rows
  static constexpr size_t kSmem =
      1024 + kBBytes + (size_t)kStages * kStageBytes + kNbrBufs * kNbrBytes;
  static_assert(kGroups * 32 * (TM / kTileM) <= kBufCols,
                "accumulators of one tile exceed a buffer");
};

__device__ int g_conv_error = 0;


// Bounded wait that also ends as soon as another thread has raised *abort.
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
  if (try_wait_parity(a, parity)) return true;  // the usual case: no clock read
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

// One bulk (TMA) copy global -> shared counted on bar; 16-byte aligned
// addresses, size a multiple of 16.
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

// Barrier of the producer threads that also ORs a flag over them, so that
// they all take the same decision.
template <int NPROD>
__device__ __forceinline__ bool producer_sync_or(bool v) {
  if (NPROD == 32) return __any_sync(0xffffffffu, v);
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 1, %2, p;\n"
      "selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(NPROD)
      : "memory");
  return r != 0;
}

// TMA gather of four rows (one row high boxes of the 2D tensor map: columns
// from col, rows r0..r3) into 4 consecutive swizzled rows at dst, counted
// on bar.  A row at or past the map's row extent is not read: it lands as
// zeros.
__device__ __forceinline__ void tma_gather4(uint32_t dst, const void* tmap, int col, int r0,
                                            int r1, int r2, int r3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(tmap), "r"(col), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(tc::smem_u32(bar))
      : "memory");
}

template <int CIN, int ALT, int ORDER, int GATHER, int TALL = 0>
__global__ void __launch_bounds__(Roles<GATHER>::kThreads, 1)
k_conv333_tc(const __grid_constant__ ConvTcArgs a) {
  static_assert(!TALL || (CIN == 32 && !GATHER), "tall tiles: 32 channels, cp.async gather");
  constexpr int kProdWarps = Roles<GATHER>::kProdWarps;
  constexpr int kProducers = Roles<GATHER>::kProducers;
  constexpr int kMmaWarp = Roles<GATHER>::kMmaWarp;
  constexpr int kThreads = Roles<GATHER>::kThreads;
  using Cfg = typename std::conditional<
      TALL != 0, ConvCfg<CIN, kTallStages, kTallStep, kTallNbrBufs, kTallRows>,
      ConvCfg<CIN, stages_of<CIN>(ALT), step_of<CIN>(ALT), nbr_bufs_of<CIN>(ALT)>>::type;
  constexpr int TM = Cfg::TM;  // rows of a tile
  constexpr int S = Cfg::kStages;
  constexpr int G = Cfg::kG;       // offsets per pipeline step
  constexpr int SG = S / G;        // steps in the ring
  constexpr int NB = Cfg::kNbrBufs;
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
  __shared__ int32_t sBias[32], sMult[32], sSlope[32], sMa[32], sMb[32], sRsl[32];
  volatile int* abort = &abort_flag;

  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (w == kMmaWarp) tc::tmem_alloc(&tslot, 512);
  if (t == 0) {
    for (int s = 0; s < SG; s++) {
      // cp.async: every producer's copies arrive; TMA: one expect_tx arrival
      tc::mbar_init(&full_bar[s], GATHER ? 1 : kProducers);
      tc::mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; b++) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], kEpilogue);
    }
    tc::mbar_init(&drain_bar, 1);
    tc::mbar_init(&w_bar, 1);
    tc::mbar_init(&nbr_bar[0], 1);
    tc::mbar_init(&nbr_bar[1], 1);
    tc::fence_mbar_init();
    abort_flag = 0;
    // weights: the pre-swizzled image in bulk copies; only the MMA thread
    // reads it, after waiting on w_bar
    mbar_expect(&w_bar, Cfg::kBBytes);
    for (int off = 0; off < Cfg::kBBytes; off += 16384)
      bulk_g2s(sm + off, reinterpret_cast<const unsigned char*>(a.wimg) + off,
               (uint32_t)min(16384, Cfg::kBBytes - off), &w_bar);
  }
  // a.mult_hi: the multipliers in the high-word form (requant_hi)
  const bool hi = a.mult_hi != nullptr;
  const bool res_hi = hi_ok(1, a.res_shift);
  const int32_t res_ms = res_hi ? hi_scale(1, a.res_shift) : 1;
  if (t < 32) {
    sBias[t] = a.bias[t];
    sMult[t] = hi ? a.mult_hi[t] : a.mult[t];
    sSlope[t] = a.prelu ? a.slope[t] : 0;
    sMa[t] = a.has_res ? a.res_mab[t] : 0;
    sMb[t] = a.has_res ? a.res_mab[32 + t] : 0;
    sRsl[t] = a.has_res ? a.res_slope[t] : 0;
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tslot;
  const int64_t n = *a.d_n;
  const int64_t ntiles = (n + TM - 1) / TM;
  // this CTA's tiles: t_first + lt * t_step, lt < my_tiles
  int64_t t_first, t_step;
  int my_tiles;
  if (ORDER == 0) {
    t_first = blockIdx.x;
    t_step = gridDim.x;
    my_tiles = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  } else if (!TALL && a.ranges) {  // contiguous runs of about equal cost (launch_conv_ranges)
    const int2 rg = a.ranges[blockIdx.x];
    t_first = rg.x;
    t_step = 1;
    my_tiles = rg.y;
  } else {
    const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
    t_first = (int64_t)blockIdx.x * per;
    t_step = 1;
    my_tiles = (int)std::max<int64_t>(0, std::min<int64_t>(per, ntiles - t_first));
  }
  auto tile_r0 = [&](int lt) { return (t_first + (int64_t)lt * t_step) * TM; };
  // the tile's present offsets (bit o: some node of the tile has its offset-o
  // neighbour): every role walks the same sequence, the present offsets in
  // ascending order, G to a pipeline step; absent ones are neither gathered
  // nor multiplied (their rows would all be zeros)
  auto tile_mask = [&](int lt) -> uint32_t {
    if (!a.tmask) return 0x7FFFFFFu;
    const int64_t tt = t_first + (int64_t)lt * t_step;
    if (!TALL) return __ldg(a.tmask + tt);
    // a tall tile: the masks of its two 128-row tiles
    const int64_t m0 = 2 * tt, nm = (n + kTileM - 1) / kTileM;
    return __ldg(a.tmask + m0) | (m0 + 1 < nm ? __ldg(a.tmask + m0 + 1) : 0u);
  };

  if (w < kProdWarps) {
    // ---------------------------------------------------------- producers --
    // a tile's neighbour rows: one bulk copy into buffer lt & 1, issued a
    // tile ahead (a partial last tile is read with plain loads instead)
    int last_issued = -1, last_used = -1;  // thread 0's bookkeeping of nbr copies
    auto issue_nbr = [&](int lt) {
      if (t == 0 && lt < my_tiles && tile_r0(lt) + TM <= n) {
        last_issued = lt;
        tc::fence_async_smem();  // earlier reads of the buffer come first
        uint64_t* bar = &nbr_bar[lt % NB];
        mbar_expect(bar, Cfg::kNbrBytes);
        // in pieces of one 128-row tile's map (13,824 bytes) at most
#pragma unroll
        for (int pc = 0; pc < TM / kTileM; pc++)
          bulk_g2s(sNbr0 + (lt % NB) * TM * 27 + pc * kTileM * 27,
                   a.nbr + tile_r0(lt) * 27 + pc * kTileM * 27, Cfg::kNbrBytes / (TM / kTileM), bar);
      }
    };
    issue_nbr(0);
    // cp.async: this thread's copies of a stage are (row, 16-byte chunk)
    // pairs fixed for the whole kernel, so their swizzled destinations and
    // source columns are formed once; per stage only the neighbour's row
    // changes.  TMA: lane l loads rows 4l .. 4l + 3 of every stage.
    constexpr int kPer = GATHER ? 1 : TM * Cfg::kChunks / kProducers;
    static_assert(GATHER || kPer * kProducers == TM * Cfg::kChunks,
                  "copies must split evenly");
    int prow[kPer];
    uint32_t pdst[kPer];
    const unsigned char* psrc[kPer];
    const uint32_t rbytes = (uint32_t)a.x_stride * 2;
    if (!GATHER) {
#pragma unroll
      for (int k = 0; k < kPer; k++) {
        const int q = t + k * kProducers;
        const int c = q % Cfg::kChunks;
        prow[k] = q / Cfg::kChunks;
        pdst[k] = tc::swz<Cfg::SW>(prow[k] * Cfg::RB + c * 16);
        psrc[k] = reinterpret_cast<const unsigned char*>(a.xb) + c * 16;
      }
    }
    uint32_t u = 0;  // stages filled so far
    uint32_t tm_next = my_tiles > 0 ? tile_mask(0) : 0u;  // masks are read a tile ahead
    for (int lt = 0; lt < my_tiles; lt++) {
      const int64_t r0 = tile_r0(lt);
      int32_t* sNbr = sNbr0 + (lt % NB) * TM * 27;
      // every producer is done issuing the previous tile's copies; all leave
      // together if any saw the abort flag
      if (producer_sync_or<kProducers>(*abort != 0)) break;
      // the next tile's map a tile ahead (two buffers; with one buffer it
      // went out at the end of the previous tile, tile 0's before the loop)
      if (NB == 2) issue_nbr(lt + 1);
      if (r0 + TM <= n) {
        if (producer_sync_or<kProducers>(!wait_or_abort(&nbr_bar[lt % NB], (lt / NB) & 1, abort)))
          break;
        last_used = lt;
      } else {
        const int64_t base = r0 * 27, lim = n * 27;
        for (int i = t; i < TM * 27; i += kProducers)
          sNbr[i] = base + i < lim ? __ldg(a.nbr + base + i) : -1;
        producer_sync_or<kProducers>(false);
      }
      // a failed wait has raised the abort flag: the step loop ends here and
      // the producers leave together at the next tile's barrier
      const uint32_t tm = tm_next;
      if (lt + 1 < my_tiles) tm_next = tile_mask(lt + 1);
      const int nsteps = (__popc(tm) + G - 1) / G;
      uint32_t mrem = tm;  // present offsets not yet staged
      for (int og = 0; og < nsteps; og++, u++) {
        const int sg = (int)(u % SG);
        if (GATHER) {
          // one lane's failed wait ends the warp's issuing together
          if (!__all_sync(0xffffffffu, u < (uint32_t)SG ||
                                           wait_or_abort(&empty_bar[sg], ((u / SG) - 1) & 1, abort)))
            break;
          int os[G];  // this step's offsets (-1: none; the last step may have fewer)
#pragma unroll
          for (int i = 0; i < G; i++) {
            os[i] = mrem ? __ffs(mrem) - 1 : -1;
            mrem &= mrem - 1;
          }
          if (lane == 0)
            mbar_expect(&full_bar[sg], (uint32_t)(min(G, __popc(tm) - og * G) * Cfg::kStageBytes));
          __syncwarp();
          const int32_t* m = sNbr + lane * 4 * 27;
#pragma unroll
          for (int i = 0; i < G; i++) {
            const int o = os[i];
            if (o < 0) continue;
            const uint32_t dst = tc::smem_u32(sA + (size_t)(sg * G + i) * Cfg::kStageBytes) +
                                 (uint32_t)(lane * 4 * Cfg::RB);
            // absent neighbours (< 0) name the row past the map's extent
            const int32_t n0 = m[o], n1 = m[27 + o], n2 = m[54 + o], n3 = m[81 + o];
            tma_gather4(dst, &a.tmap, 0, n0 < 0 ? a.tma_rows : n0, n1 < 0 ? a.tma_rows : n1,
                        n2 < 0 ? a.tma_rows : n2, n3 < 0 ? a.tma_rows : n3, &full_bar[sg]);
          }
        } else {
          if (u >= (uint32_t)SG && !wait_or_abort(&empty_bar[sg], ((u / SG) - 1) & 1, abort))
            break;
#pragma unroll
          for (int i = 0; i < G; i++) {
            const int o = mrem ? __ffs(mrem) - 1 : -1;
            mrem &= mrem - 1;
            if (o < 0) continue;
            const uint32_t sbase = tc::smem_u32(sA + (size_t)(sg * G + i) * Cfg::kStageBytes);
#pragma unroll
            for (int k = 0; k < kPer; k++) {
              const int32_t nb = sNbr[prow[k] * 27 + o];
              // absent neighbours (nb < 0): zero-filled, the address kept valid
              const uint32_t r = (uint32_t)max(nb, 0);
              tc::cp_async16(sbase + pdst[k], psrc[k] + (size_t)r * rbytes, nb >= 0);
            }
          }
          // arrives on the step's barrier once this thread's copies have landed
          asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(
                           tc::smem_u32(&full_bar[sg]))
                       : "memory");
        }
      }
      // one map buffer: every producer has read this tile's map (its copies
      // are issued), so the next tile's goes out now, beside the last steps
      if (NB == 1 && lt + 1 < my_tiles) {
        producer_sync_or<kProducers>(false);
        issue_nbr(lt + 1);
      }
    }
    // a neighbour-row copy issued but not consumed (abort) lands before exit
    if (t == 0 && last_issued > last_used)
      tc::mbar_wait(&nbr_bar[last_issued % NB], (last_issued / NB) & 1);
    if (GATHER) {
      // the loads of the last steps issued land before the CTA exits (the
      // MMA thread has waited for them unless it stopped on abort)
      if (lane == 0)
        for (uint32_t q = u > (uint32_t)SG ? u - SG : 0; q < u; q++)
          tc::mbar_wait(&full_bar[q % SG], (q / SG) & 1);
      __syncwarp();
    } else {
      tc::cp_async_wait<0>();  // every copy of this thread has landed
    }
  } else if (w == kMmaWarp) {
    // ---------------------------------------------------------------- MMA --
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16(kTileM, 32);
      uint32_t u = 0;
      const bool wok = wait_or_abort(&w_bar, 0, abort);  // the weights have landed
      uint32_t tm_next = my_tiles > 0 ? tile_mask(0) : 0u;
      for (int lt = 0; lt < my_tiles && wok && !*abort; lt++) {
        const int b = lt & 1;
        if (lt >= 2 && !wait_or_abort(&acc_empty[b], ((lt >> 1) - 1) & 1, abort)) break;
        tc::tc_fence_after();
        const uint32_t dbase = tbase + (uint32_t)(b * Cfg::kBufCols);
        bool ok = true;
        const uint32_t tm = tm_next;
        if (lt + 1 < my_tiles) tm_next = tile_mask(lt + 1);
        const int nsteps = (__popc(tm) + G - 1) / G;
        uint32_t mrem = tm, started = 0;  // started: accumulator groups written this tile
        for (int og = 0; og < nsteps; og++, u++) {
          const int sg = (int)(u % SG);
          if (!wait_or_abort(&full_bar[sg], (u / SG) & 1, abort)) {
            ok = false;
            break;
          }
          // the step's landed cp.async copies, to the MMA's proxy (TMA
          // loads are in that proxy already)
          if (!GATHER) tc::fence_async_smem();
          tc::tc_fence_after();
#pragma unroll
          for (int i = 0; i < G; i++) {
            const int o = mrem ? __ffs(mrem) - 1 : -1;
            mrem &= mrem - 1;
            if (o < 0) continue;
            const uint32_t sa = tc::smem_u32(sA + (size_t)(sg * G + i) * Cfg::kStageBytes);
            const int g = o / Cfg::kPerGroup;
            // a group's first present offset overwrites its accumulator
            const uint32_t acc0 = (started >> g) & 1u;
            started |= 1u << g;
#pragma unroll
            for (int ks = 0; ks < CIN / 16; ks++) {
              const int k0 = o * CIN + ks * 16;
              const uint32_t sb = tc::smem_u32(sB) + (k0 / 64) * 4096 + (k0 % 64) * 2;
              tc::mma_bf16(dbase + g * 32, tc::smem_desc<Cfg::SW>(sa + ks * 32, 8 * Cfg::RB),
                           tc::smem_desc<128>(sb, 1024), idesc, (acc0 || ks > 0) ? 1u : 0u);
              if (TALL)  // rows 128..255 of the tile into the buffer's upper 128 columns
                tc::mma_bf16(dbase + kTileM + g * 32,
                             tc::smem_desc<Cfg::SW>(sa + kTileM * Cfg::RB + ks * 32, 8 * Cfg::RB),
                             tc::smem_desc<128>(sb, 1024), idesc, (acc0 || ks > 0) ? 1u : 0u);
            }
          }
          tc::mma_commit(&empty_bar[sg]);
        }
        if (!ok) break;
        tc::mma_commit(&acc_full[b]);
      }
      // every MMA this thread issued has completed before the CTA frees TMEM
      // (a plain bounded wait: this one must not end early on abort)
      tc::mma_commit(&drain_bar);
      if (!tc::mbar_wait(&drain_bar, 0)) *abort = 1;
    }
    __syncwarp();
  } else {
    // ----------------------------------------------------------- epilogue --
    const int e = ((w & 3) << 5) | lane;  // row of the tile = TMEM lane (the warp's quadrant)
    const uint32_t lane_off = (uint32_t)((w & 3) * 32) << 16;
    uint32_t tm_next = my_tiles > 0 ? tile_mask(0) : 0u;
    for (int lt = 0; lt < my_tiles; lt++) {
      const int b = lt & 1;
      const uint32_t tm = tm_next;  // groups without a present offset hold nothing
      if (lt + 1 < my_tiles) tm_next = tile_mask(lt + 1);
      // the tile's rows e and (tall tiles) e + 128, their accumulators in the
      // buffer's lower and upper 128 columns
      bool left = false;
#pragma unroll
      for (int hf = 0; hf <= TALL; hf++) {
        const int64_t r = tile_r0(lt) + e + hf * kTileM;
        // the row's inputs that do not wait for the accumulators (the
        // residual's y1 row, the embedding row) are loaded before the wait
        uint4 y1v[2] = {}, ev[2] = {};
        if (r < n) {
          if (a.has_res) {
            const uint4* ys = reinterpret_cast<const uint4*>(a.y1 + r * a.y1_stride);
            y1v[0] = ys[0];
            y1v[1] = ys[1];
          }
          if (a.emb.table) {
            const uint4* e4 = reinterpret_cast<const uint4*>(a.emb.table + (int)a.emb.code[r] * 32);
            ev[0] = __ldg(e4);
            ev[1] = __ldg(e4 + 1);
          }
        }
        // the TMEM loads below are warp-collective: the warp leaves together
        if (hf == 0) {
          if (!__all_sync(0xffffffffu, wait_or_abort(&acc_full[b], (lt >> 1) & 1, abort))) {
            left = true;
            break;
          }
          tc::tc_fence_after();
        }
        int32_t acc[32];
#pragma unroll
        for (int i = 0; i < 32; i++) acc[i] = sBias[i];
        const uint32_t dbase = tbase + lane_off + (uint32_t)(b * Cfg::kBufCols + hf * kTileM);
        // a group's 32 columns in flight per wait
#pragma unroll
        for (int g = 0; g < Cfg::kGroups; g++) {
          if (!((tm >> (g * Cfg::kPerGroup)) & ((1u << Cfg::kPerGroup) - 1))) continue;
          uint32_t v[2][16];
          tc::tmem_ld16_issue(dbase + g * 32, v[0]);
          tc::tmem_ld16_issue(dbase + g * 32 + 16, v[1]);
          tc::tmem_wait_ld();
#pragma unroll
          for (int k = 0; k < 2; k++) {
            tc::tmem_regs_ready(v[k]);
#pragma unroll
            for (int i = 0; i < 16; i++) acc[k * 16 + i] += __float2int_rn(__uint_as_float(v[k][i]));
          }
        }
        if (hf == TALL) {
          tc::tc_fence_before();
          mbar_arrive(&acc_empty[b]);  // the buffer is free for tile lt + 2
        }
        if (r < n) {
          __align__(16) int8_t q[32];
          // the requantisation form is fixed per launch: one straight loop per
          // form (HI: the layer's, RHI: the residual merge's)
          auto finish = [&](auto HI, auto RHI) {
            if (a.has_res) {
              __align__(16) int8_t y1[32];
              reinterpret_cast<uint4*>(y1)[0] = y1v[0];
              reinterpret_cast<uint4*>(y1)[1] = y1v[1];
#pragma unroll
              for (int i = 0; i < 32; i++) {
                int32_t v = acc[i];
                if (a.prelu) v = prelu(v, sSlope[i]);
                int y2;
                if constexpr (decltype(HI)::value) y2 = requant_hi(v, sMult[i], a.z_out);
                else y2 = requant(v, sMult[i], a.shift, a.z_out);
                int32_t m = (y1[i] - a.res_z1) * sMa[i] + (y2 - a.res_z2) * sMb[i];
                m = prelu(m, sRsl[i]);
                if constexpr (decltype(RHI)::value) q[i] = (int8_t)requant_hi(m, res_ms, a.res_z_out);
                else q[i] = (int8_t)requant(m, 1, a.res_shift, a.res_z_out);
              }
            } else {
#pragma unroll
              for (int i = 0; i < 32; i++) {
                int32_t v = acc[i];
                if (a.prelu) v = prelu(v, sSlope[i]);
                if constexpr (decltype(HI)::value) q[i] = (int8_t)requant_hi(v, sMult[i], a.z_out);
                else q[i] = (int8_t)requant(v, sMult[i], a.shift, a.z_out);
              }
            }
          };
          if (hi && res_hi) finish(std::true_type{}, std::true_type{});
          else if (hi) finish(std::true_type{}, std::false_type{});
          else if (res_hi) finish(std::false_type{}, std::true_type{});
          else finish(std::false_type{}, std::false_type{});
          uint4* dst = reinterpret_cast<uint4*>(a.out + r * a.out_stride + a.out_col);
          dst[0] = reinterpret_cast<const uint4*>(q)[0];
          dst[1] = reinterpret_cast<const uint4*>(q)[1];
          if (a.emb.table) {  // the next step's Concat(., E[Y]) half of the row
            uint4* de = reinterpret_cast<uint4*>(a.out + r * a.out_stride + a.emb_col);
            de[0] = ev[0];
            de[1] = ev[1];
          }
          if (a.outb) {
            __align__(16) __nv_bfloat16 bq[32];
#pragma unroll
            for (int i = 0; i < 32; i++) bq[i] = __int2bfloat16_rn((int)q[i] - a.outb_z);
            uint4* db = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.outb) +
                                                 r * a.outb_stride);
#pragma unroll
            for (int k = 0; k < 4; k++) db[k] = reinterpret_cast<const uint4*>(bq)[k];
          }
        }
      }
      if (left) break;
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (t == kThreads - 32) tc::mbar_wait(&w_bar, 0);  // the weights' copies have landed
  if (w == kMmaWarp) tc::tmem_dealloc(tbase, 512);
  if (t == 0 && abort_flag) atomicExch(&g_conv_error, 1);
}

// int8 rows -> bf16 (q - z) rows for the tensor-core gather; columns
// [0, x_cols) come from x, the rest (the concatenated second half) from x2,
// or from the embedding table row of the node's code when etab is set
__global__ void k_to_bf16(const int8_t* __restrict__ x, int x_stride, int x_cols,
                          const int8_t* __restrict__ x2, int x2_stride, int cols, int z,
                          const int64_t* d_n, __nv_bfloat16* out,
                          const int8_t* __restrict__ etab = nullptr,
                          const uint8_t* __restrict__ ecode = nullptr) {
  const int64_t n = *d_n;
  const int per = cols / 8;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * per;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / per;
    const int c = (int)(q - r * per);
    const int8_t* src = c * 8 < x_cols ? x + r * x_stride + c * 8
                        : etab ? etab + (int)ecode[r] * 32 + (c * 8 - x_cols)
                               : x2 + r * x2_stride + (c * 8 - x_cols);
    const uint2 raw = *reinterpret_cast<const uint2*>(src);
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
  k_to_bf16<<<blocks, 256, 0, st>>>(x, x_stride, cols, x, x_stride, cols, z, d_n,
                                    reinterpret_cast<__nv_bfloat16*>(out));
  count_launches(1);
}

void launch_to_bf16_emb(const int8_t* a, int a_stride, int a_cols, EmbSrc e, int z,
                        const int64_t* d_n, int64_t n_host, void* out, cudaStream_t st) {
  if (n_host <= 0) return;
  const int cols = a_cols + 32;
  const int64_t work = n_host * (cols / 8);
  const int blocks = (int)std::min<int64_t>((work + 255) / 256, 148 * 8);
  k_to_bf16<<<blocks, 256, 0, st>>>(a, a_stride, a_cols, nullptr, 0, cols, z, d_n,
                                    reinterpret_cast<__nv_bfloat16*>(out), e.table, e.code);
  count_launches(1);
}

void launch_to_bf16_cat(const int8_t* a, int a_stride, const int8_t* b, int b_stride, int z,
                        const int64_t* d_n, int64_t n_host, void* out, cudaStream_t st) {
  if (n_host <= 0) return;
  const int64_t work = n_host * 8;
  const int blocks = (int)std::min<int64_t>((work + 255) / 256, 148 * 8);
  k_to_bf16<<<blocks, 256, 0, st>>>(a, a_stride, 32, b, b_stride, 64, z, d_n,
                                    reinterpret_cast<__nv_bfloat16*>(out));
  count_launches(1);
}

namespace {

template <int CIN, int ALT, int ORDER, int GATHER>
void launch_variant(const ConvTcArgs& a, int blocks, cudaStream_t st) {
  constexpr size_t smem =
      ConvCfg<CIN, stages_of<CIN>(ALT), step_of<CIN>(ALT), nbr_bufs_of<CIN>(ALT)>::kSmem;
  static_assert(smem <= 232448, "shared memory of a conv variant exceeds the limit");
  auto* k = k_conv333_tc<CIN, ALT, ORDER, GATHER>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<blocks, Roles<GATHER>::kThreads, smem, st>>>(a);
}

template <int CIN, int ORDER>
void launch_tall(const ConvTcArgs& a, int blocks, cudaStream_t st) {
  constexpr size_t smem = ConvCfg<CIN, kTallStages, kTallStep, kTallNbrBufs, kTallRows>::kSmem;
  static_assert(smem <= 232448, "shared memory of a conv variant exceeds the limit");
  auto* k = k_conv333_tc<CIN, 0, ORDER, 0, 1>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<blocks, Roles<0>::kThreads, smem, st>>>(a);
}

template <int CIN, int GATHER>
void launch_cin(const ConvTcArgs& a, int blocks, int variant, cudaStream_t st) {
  if (variant >= 8) {  // tall tiles (32 channels); 64 channels take 0 / 2
    if constexpr (CIN == 32 && !GATHER) {
      if (variant & 1) launch_tall<32, 1>(a, blocks, st);
      else launch_tall<32, 0>(a, blocks, st);
      return;
    }
    variant = (variant & 1) ? 2 : 0;
  }
  switch (variant & 3) {
    case 1: launch_variant<CIN, 1, 0, GATHER>(a, blocks, st); break;
    case 2: launch_variant<CIN, 0, 1, GATHER>(a, blocks, st); break;
    case 3: launch_variant<CIN, 1, 1, GATHER>(a, blocks, st); break;
    default: launch_variant<CIN, 0, 0, GATHER>(a, blocks, st); break;
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime.
EncodeTiled encoder() {
  static EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// The bf16 input rows as a 2D tensor (cin columns, rows rows, row pitch
// x_stride elements) with one-row boxes of the whole row, swizzled like the
// A stages (64-byte rows: 64B swizzle, 128-byte rows: 128B).
bool encode_rows(ConvTcArgs& a, int cin, int64_t rows) {
  static_assert(sizeof(TmaDesc) == sizeof(CUtensorMap), "tensor map size");
  const EncodeTiled fn = encoder();
  if (!fn || rows <= 0 || rows > 0x7fffffff || ((uintptr_t)a.xb & 15) || (a.x_stride * 2) % 16)
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cin, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)a.x_stride * 2};
  const cuuint32_t box[2] = {(cuuint32_t)cin, 1};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(reinterpret_cast<CUtensorMap*>(&a.tmap), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                        2, const_cast<void*>(a.xb), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE,
                        cin == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  a.tma_rows = (int)rows;
  return r == CUDA_SUCCESS;
}

}  // namespace

int conv_ctas(int64_t n_host) { return (int)std::min<int64_t>((n_host + kTileM - 1) / kTileM, 148); }

// Tile runs of about equal cost for the contiguous tile order: a tile costs
// its present offsets plus kTileCost for its fixed work (map, epilogue,
// hand-offs).  With the exclusive cost prefix P_t, the tile's midpoint
// K_t = P_t + floor(c_t / 2) and the total T, CTA b starts at the first tile
// with K_t >= floor(b T / ctas) (a tile goes to the run its cost's middle
// falls in): tile t starts the CTAs b in [cnt(K_{t-1}), cnt(K_t)) (K_{-1} =
// -1), cnt(K) = #{b : floor(b T / ctas) <= K} = ceil((K + 1) ctas / T), so
// every tile finds its CTAs at once.
constexpr int kTileCost = 12;

__global__ void __launch_bounds__(1024)
k_conv_ranges(const uint32_t* __restrict__ tmask, const int64_t* d_n, int ctas, int2* ranges) {
  __shared__ uint32_t sm[32];
  __shared__ int start[149];
  const int64_t n = *d_n;
  const int nt = (int)((n + kTileM - 1) / kTileM);
  auto cost = [&](int t) { return (uint32_t)(__popc(tmask[t]) + kTileCost); };
  uint32_t total = 0;
  for (int t = threadIdx.x; t < nt; t += 1024) total += cost(t);
  total = __reduce_add_sync(0xffffffffu, total);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = total;
  for (int b = threadIdx.x; b <= ctas; b += 1024) start[b] = nt;  // CTAs past the last tile
  __syncthreads();
  total = 0;
  for (int i = 0; i < 32; i++) total += sm[i];
  __syncthreads();
  auto cnt = [&](int64_t P) -> int {  // CTAs whose boundary is at most P
    const int64_t c = ((P + 1) * ctas + total - 1) / total;
    return c < ctas ? (int)c : ctas;
  };
  uint32_t run = 0;
  for (int base = 0; base < nt; base += 1024) {
    const int t = base + threadIdx.x;
    const uint32_t c = t < nt ? cost(t) : 0u;
    uint32_t x = c;  // block-inclusive scan of the costs
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if ((threadIdx.x & 31) >= d) x += y;
    }
    if ((threadIdx.x & 31) == 31) sm[threadIdx.x >> 5] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int i = 0; i < (int)(threadIdx.x >> 5); i++) before += sm[i];
    const uint32_t blk = sm[0] + sm[1] + sm[2] + sm[3] + sm[4] + sm[5] + sm[6] + sm[7] + sm[8] +
                         sm[9] + sm[10] + sm[11] + sm[12] + sm[13] + sm[14] + sm[15] + sm[16] +
                         sm[17] + sm[18] + sm[19] + sm[20] + sm[21] + sm[22] + sm[23] + sm[24] +
                         sm[25] + sm[26] + sm[27] + sm[28] + sm[29] + sm[30] + sm[31];
    if (t < nt) {
      const int64_t P = (int64_t)run + before + x - c;  // exclusive prefix of tile t
      const int64_t K = P + c / 2;
      int64_t Kp = -1;  // the midpoint of tile t - 1
      if (t > 0) {
        const uint32_t cp = cost(t - 1);
        Kp = P - cp + cp / 2;
      }
      for (int b = cnt(Kp); b < cnt(K); b++) start[b] = t;
    }
    run += blk;
    __syncthreads();
  }
  __syncthreads();
  for (int b = threadIdx.x; b < ctas; b += 1024) ranges[b] = make_int2(start[b], start[b + 1] - start[b]);
}

void launch_conv_ranges(const uint32_t* tmask, const int64_t* d_n, int64_t n_host, int2* ranges,
                        cudaStream_t st) {
  if (n_host <= 0) return;
  k_conv_ranges<<<1, 1024, 0, st>>>(tmask, d_n, conv_ctas(n_host), ranges);
  count_launches(1);
}

void launch_conv333_tc(const ConvTcArgs& a, int cin, int64_t n_host, cudaStream_t st,
                       int variant) {
  if (n_host <= 0) return;
  const int blocks = conv_ctas(n_host);
  if (variant & 4) {
    // TMA gather: the map covers rows [0, n_host), every neighbour index the
    // kernel reads is below the level's size <= n_host.  An input the
    // encoder rejects (unaligned rows) takes the copy gather of the same ring.
    ConvTcArgs b = a;
    if (encode_rows(b, cin, n_host)) {
      if (cin == 64) launch_cin<64, 1>(b, blocks, variant, st);
      else launch_cin<32, 1>(b, blocks, variant, st);
      count_launches(1);
      return;
    }
  }
  if (cin == 64) launch_cin<64, 0>(a, blocks, variant, st);
  else launch_cin<32, 0>(a, blocks, variant, st);
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
