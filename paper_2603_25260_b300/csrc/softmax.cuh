// The integer softmax of one row (Eq. 15), one warp per row, used by the
// CUDA-core predictor and the softmax-only kernel; the tensor-core
// predictor's per-half-row form shares its constants and helpers.
#pragma once

#include "common.cuh"

namespace lpc {

// ------------------------------------------- integer softmax -> CDF row --
// One warp per row; lane l holds the logits of symbols s = 8l + i, i = 0..7;
// symbol 255 (lane 31, i = 7) is not a class and takes no frequency.
//   M = max l_s; e_s = lut[M - l_s]; S = sum e_s (2^16 <= S < 2^24, as
//   lut[0] = 2^16 and lut is nonincreasing);
//   f_s = 1 + q_s with q_s = floor(e_s (2^16 - 255) / S) (the product fits
//   in 32 bits); the remainder R = 2^16 - sum f_s goes to the lowest s with
//   l_s = M.
// M and its lowest index come from one reduction of the keys 256 l_s +
// (255 - s).  The divisions share one reciprocal inv = floor((2^32 - 1) / S):
// for x < 2^32, umulhi(x, inv) is floor(x / S) or one less (x inv / 2^32 >
// x / S - x / 2^32), and one conditional step makes it exact.
constexpr uint32_t kQScale = kFreqTotal - kNsym;

__device__ __forceinline__ uint32_t div_by(uint32_t x, uint32_t S, uint32_t inv) {
  uint32_t q = __umulhi(x, inv);
  if (x - q * S >= S) q++;
  return q;
}

// floor((2^32 - 1) / S).  For 2^16 <= S < 2^24 the fp32 reciprocal scaled
// by 2^32 is within 2^-8 of 2^32 / S, so its truncation is within one of
// the result and one correction either way makes it exact; other S take
// the integer division.
__device__ __forceinline__ uint32_t recip32(uint32_t S) {
  if (S < (1u << 16) || S >= (1u << 24)) return 0xFFFFFFFFu / S;
  uint32_t g = __float2uint_rz(__frcp_rn((float)S) * 4294967296.0f);
  const unsigned long long gs = (unsigned long long)g * S;
  if (gs > 0xFFFFFFFFull)
    g--;
  else if (gs + S <= 0xFFFFFFFFull)
    g++;
  return g;
}

struct SoftRow {
  uint32_t r[8];  // this lane's running sums q_{8l} + ... + q_{8l+i}
  uint32_t tot;   // sum of q over the row
  int first;      // lowest symbol with the maximum logit
};

// Byte i of w, sign-extended (a byte permute whose upper selectors
// replicate the byte's sign bit).
__device__ __forceinline__ int sext_byte(uint32_t w, int i) {
  const uint32_t sel = (uint32_t)(i | ((8 | i) << 4) | ((8 | i) << 8) | ((8 | i) << 12));
  uint32_t r;
  asm("prmt.b32 %0, %1, 0, %2;" : "=r"(r) : "r"(w), "r"(sel));
  return (int)r;
}

// Per-lane tie-break constants 255 - (8 lane + i) of the max keys.
__device__ __forceinline__ void tie_keys(int lane, int (&ck)[8]) {
#pragma unroll
  for (int i = 0; i < 8; i++) ck[i] = 255 - (8 * lane + i);
}

// l: this lane's logits (lane 31's l[7], the padding, is ignored).
__device__ __forceinline__ void softmax_row(int (&l)[8], const int (&ck)[8], bool last,
                                            const uint32_t* slut, SoftRow& o) {
  if (last) l[7] = -128;  // key -32768: loses every tie
  int key = l[0] * 256 + ck[0];
#pragma unroll
  for (int i = 1; i < 8; i++) key = max(key, l[i] * 256 + ck[i]);
  key = __reduce_max_sync(0xffffffffu, key);
  const int mx = key >> 8;  // floor: the low byte is the tie-break
  o.first = 255 - (key & 255);
  uint32_t e[8];
  uint32_t S = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    e[i] = slut[mx - l[i]];
    S += e[i];
  }
  if (last) {
    S -= e[7];
    e[7] = 0;
  }
  S = __reduce_add_sync(0xffffffffu, S);
  const uint32_t inv = recip32(S);
  uint32_t run = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    run += div_by(e[i] * kQScale, S, inv);
    o.r[i] = run;
  }
  o.tot = __reduce_add_sync(0xffffffffu, run);
}

// The row of cumulative values C_{s+1} = f_0 + ... + f_s as u16, entries
// 254 and 255 = 0xFFFF (C_{s+1} <= 65535 for s <= 253 since every f >= 1).
__device__ __forceinline__ void cdf_values(const SoftRow& o, int lane, uint32_t (&h)[8]) {
  uint32_t x = o.r[7];
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  const uint32_t R = kQScale - o.tot;
  const uint32_t base = x - o.r[7] + 8 * lane + 1;  // q before this lane; f = 1 + q
  const int thr = o.first - 8 * lane;              // symbols from the first maximum on take R
#pragma unroll
  for (int i = 0; i < 8; i++) h[i] = o.r[i] + base + i + (i >= thr ? R : 0u);
}

__device__ __forceinline__ void store_cdf_row(const SoftRow& o, int lane, uint16_t* row) {
  uint32_t h[8];
  cdf_values(o, lane, h);
  if (lane == 31) h[6] = h[7] = 0xFFFFu;
  uint4 v;
  v.x = h[0] | (h[1] << 16);
  v.y = h[2] | (h[3] << 16);
  v.z = h[4] | (h[5] << 16);
  v.w = h[6] | (h[7] << 16);
  reinterpret_cast<uint4*>(row)[lane] = v;
}

// The encoder's interval (C_s, f_s) of symbol s (0..254) packed as
// C_s | f_s << 16; every lane takes part, the result is lane s / 8's.
__device__ __forceinline__ uint32_t enc_pair(const SoftRow& o, int lane, int s) {
  const int sl = s >> 3, si = s & 7;
  const uint32_t before = __reduce_add_sync(0xffffffffu, lane < sl ? o.r[7] : 0u);
  uint32_t rs = 0, rp = 0;  // r_si and r_{si-1}, by masks (no indexed access)
#pragma unroll
  for (int k = 0; k < 8; k++) {
    rs |= o.r[k] & (0u - (uint32_t)(k == si));
    rp |= o.r[k] & (0u - (uint32_t)(k + 1 == si));
  }
  const uint32_t R = kQScale - o.tot;
  const uint32_t fs = 1 + (rs - rp) + (s == o.first ? R : 0u);
  const uint32_t cs = (uint32_t)s + before + rp + (s > o.first ? R : 0u);
  return cs | (fs << 16);
}


// ---------------------------------------------- key rows (predictor) --
// The tensor-core predictor runs the same softmax one thread per half row:
// its epilogue writes each logit l_s as the 16-bit key (127 - l_s) 128 +
// (s & 127), whose bits 7..14 are the byte offset of lut[127 - l_s] in a
// copy of the exp table with one word per bank (word 32 d + lane holds
// lut[d]); a thread reads lut[(127 - l_s) - (127 - M)] from its own bank, so
// the 32 loads of a warp never conflict.
constexpr uint32_t kKeyOff = 0x7F80u;  // the (127 - l) 128 bits of a key
constexpr uint32_t kKeyOff2 = 0x7F807F80u;  // the same in both halves of a word

__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// A read of the (read-only) bank-replicated table.
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
  uint32_t v;
  asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

}  // namespace lpc
