#include "coder.h"

#if defined(__x86_64__)
#include <immintrin.h>
#endif

namespace lpc {

void RangeEncoder::shift_low() {
  if ((uint32_t)low_ < 0xFF000000u || (low_ >> 32) != 0) {
    const uint8_t carry = (uint8_t)(low_ >> 32);
    uint8_t b = cache_;
    for (; pending_ > 0; pending_--) {
      put((uint8_t)(b + carry));
      b = 0xFF;
    }
    cache_ = (uint8_t)(low_ >> 24);
  }
  pending_++;
  low_ = (low_ & 0x00FFFFFFull) << 8;
}

void RangeEncoder::finish() {
  // the multiple of 2^k in [low, low + range) with k largest (k >= 24)
  const uint64_t end = low_ + range_;
  for (int k = 32; k > 0; k--) {
    const uint64_t v = ((low_ + ((uint64_t{1} << k) - 1)) >> k) << k;
    if (v < end) {
      low_ = v;
      break;
    }
  }
  for (int i = 0; i < 5; i++) shift_low();
  for (size_t i = 0; i < RangeDecoder::kPad && len_ > 0 && len_ <= cap_ && out_[len_ - 1] == 0;
       i++)
    len_--;
}

RangeDecoder::RangeDecoder(const uint8_t* p, size_t n) : p_(p), n_(n) {
  code_ = (at(0) << 24) | (at(1) << 16) | (at(2) << 8) | at(3);
  pos_ = 4;
}

// Renormalisation without a loop: after an update range >= 255 (the
// smallest interval of an adaptive total <= 65568), so at most three bytes
// come in; they are read before the count is known.
void RangeDecoder::update(uint32_t lo, uint32_t f) {
  code_ -= r_ * lo;
  range_ = r_ * f;
  if (code_ >= range_) bad_ = true;
  const int nb = (range_ < (1u << 24)) + (range_ < (1u << 16)) + (range_ < (1u << 8));
  const uint64_t b0 = at(pos_), b1 = at(pos_ + 1), b2 = at(pos_ + 2);
  const uint64_t c = ((uint64_t)code_ << 24) | (b0 << 16) | (b1 << 8) | b2;
  code_ = (uint32_t)(c >> (24 - 8 * nb));
  range_ <<= 8 * nb;
  pos_ += nb;
}

int RangeDecoder::decode_row(const uint16_t* row) {
  r_ = range_ >> 16;
  uint32_t v = code_ / r_;
  if (v > 65535u) v = 65535u;
  // first index in [0, 254) whose cumulative C_{s+1} exceeds v
  int lo = 0, hi = 254;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (row[mid] <= v) lo = mid + 1;
    else hi = mid;
  }
  const uint32_t a = lo ? row[lo - 1] : 0u;
  const uint32_t b = lo == 254 ? 65536u : row[lo];
  update(a, b - a);
  return lo;
}

AdaptiveModel::AdaptiveModel() {
  for (int i = 0; i < 255; i++) f_[i] = 1;
  f_[255] = 0;
  total_ = 255;
  rebuild();
}

void AdaptiveModel::rebuild() {
  uint32_t c = 0;
  for (int g = 0; g < 16; g++) {
    cg_[g] = c;
    uint32_t w = 0;
    for (int i = 0; i < 16; i++) {
      cw_[16 * g + i] = w;
      w += f_[16 * g + i];
    }
    c += w;
  }
}

namespace {
#if defined(__x86_64__)
// AVX2 forms, used when the host has AVX2 (checked once at load).
__attribute__((target("avx2"))) inline int count_above_avx2(const uint32_t* a, uint32_t v) {
  const __m256i vv = _mm256_set1_epi32((int)v);
  const __m256i* p = reinterpret_cast<const __m256i*>(a);
  const unsigned m0 = (unsigned)_mm256_movemask_ps(_mm256_castsi256_ps(
      _mm256_cmpgt_epi32(_mm256_load_si256(p), vv)));
  const unsigned m1 = (unsigned)_mm256_movemask_ps(_mm256_castsi256_ps(
      _mm256_cmpgt_epi32(_mm256_load_si256(p + 1), vv)));
  return __builtin_popcount(m0 | (m1 << 8));
}
__attribute__((target("avx2"))) inline void add_after_avx2(uint32_t* a, int j) {
  const __m256i jj = _mm256_set1_epi32(j), inc = _mm256_set1_epi32(32);
  __m256i* p = reinterpret_cast<__m256i*>(a);
  const __m256i i0 = _mm256_setr_epi32(0, 1, 2, 3, 4, 5, 6, 7);
  const __m256i i1 = _mm256_setr_epi32(8, 9, 10, 11, 12, 13, 14, 15);
  _mm256_store_si256(p, _mm256_add_epi32(_mm256_load_si256(p),
                                         _mm256_and_si256(_mm256_cmpgt_epi32(i0, jj), inc)));
  _mm256_store_si256(p + 1, _mm256_add_epi32(_mm256_load_si256(p + 1),
                                             _mm256_and_si256(_mm256_cmpgt_epi32(i1, jj), inc)));
}
const bool g_avx2 = __builtin_cpu_supports("avx2");
#endif

// Number of the 16 values a[0..15] (< 2^31) that exceed v.
inline int count_above(const uint32_t* a, uint32_t v) {
#if defined(__x86_64__)
  if (g_avx2) return count_above_avx2(a, v);
#endif
  int n = 0;
  for (int i = 0; i < 16; i++) n += a[i] > v;
  return n;
}

// a[i] += 32 for i > j (i < 16).
inline void add_after(uint32_t* a, int j) {
#if defined(__x86_64__)
  if (g_avx2) return add_after_avx2(a, j);
#endif
  for (int i = j + 1; i < 16; i++) a[i] += 32;
}
}  // namespace

void AdaptiveModel::bump(int s) {
  f_[s] += 32;
  total_ += 32;
  if (total_ > 65536u) {
    total_ = 0;
    for (int i = 0; i < 255; i++) {
      f_[i] = (f_[i] + 1) >> 1;
      total_ += f_[i];
    }
    rebuild();
    return;
  }
  add_after(cg_, s >> 4);
  add_after(cw_ + (s & ~15), s & 15);
}

void AdaptiveModel::encode(RangeEncoder& e, int s) {
  e.code_total(cg_[s >> 4] + cw_[s], f_[s], total_);
  bump(s);
}

int AdaptiveModel::decode(RangeDecoder& d) {
  const uint32_t v = d.target(total_);
  // the last group whose lower bound is <= v, then the last symbol in it;
  // symbol 255 (count 0) shares its bound with the end of the range, never
  // below v, so it is never chosen
  const int g = 15 - count_above(cg_, v);
  int s = 16 * g + 15 - count_above(cw_ + 16 * g, v - cg_[g]);
  if (s > 254) s = 254;
  d.update(cg_[g] + cw_[s], f_[s]);
  bump(s);
  return s;
}

size_t encode_packed(const uint32_t* lofreq, size_t n, uint8_t* out, size_t cap) {
  RangeEncoder e(out, cap);
  for (size_t i = 0; i < n; i++) e.code16(lofreq[i] & 0xFFFFu, lofreq[i] >> 16);
  e.finish();
  return e.size();
}

size_t encode_adaptive(const uint8_t* syms, size_t n, uint8_t* out, size_t cap) {
  RangeEncoder e(out, cap);
  AdaptiveModel m;
  for (size_t i = 0; i < n; i++) m.encode(e, syms[i]);
  e.finish();
  return e.size();
}

size_t encode_adaptive_codes(const uint8_t* codes, size_t n, uint8_t* out, size_t cap) {
  RangeEncoder e(out, cap);
  AdaptiveModel m;
  for (size_t i = 0; i < n; i++) m.encode(e, codes[i] - 1);
  e.finish();
  return e.size();
}

// The tables were just written to host memory by DMA, so they are not in any
// CPU cache: the eight 64-byte lines of a row are prefetched a few rows ahead
// of the binary search.
static inline void prefetch_row(const uint16_t* row) {
  const char* p = reinterpret_cast<const char*>(row);
  for (int k = 0; k < 512; k += 64) __builtin_prefetch(p + k, 0, 3);
}

bool decode_rows(const uint16_t* rows, size_t n, const uint8_t* in, size_t len, uint8_t* syms) {
  constexpr size_t kAhead = 8;
  RangeDecoder d(in, len);
  for (size_t i = 0; i < n && i < kAhead; i++) prefetch_row(rows + i * 256);
  for (size_t i = 0; i < n; i++) {
    if (i + kAhead < n) prefetch_row(rows + (i + kAhead) * 256);
    syms[i] = (uint8_t)d.decode_row(rows + i * 256);
  }
  return !d.bad();
}

bool decode_adaptive(size_t n, const uint8_t* in, size_t len, uint8_t* syms) {
  RangeDecoder d(in, len);
  AdaptiveModel m;
  for (size_t i = 0; i < n; i++) syms[i] = (uint8_t)m.decode(d);
  return !d.bad();
}

}  // namespace lpc

// ------------------------------------------------ C ABI (lpc_ops.h) --
#include "../../include/lpc.h"
#include "../../include/lpc_ops.h"

extern "C" int lpc_rc_encode_rows(const uint16_t* h_rows, const uint8_t* h_syms, int64_t n,
                                  uint8_t* h_out, size_t cap, size_t* out_len) {
  if (n < 0 || !out_len || (n > 0 && (!h_rows || !h_syms)) || (cap > 0 && !h_out))
    return LPC_INVALID_ARG;
  lpc::RangeEncoder e(h_out, cap);
  for (int64_t i = 0; i < n; i++) {
    const int s = h_syms[i];
    if (s > 254) return LPC_INVALID_ARG;
    const uint16_t* row = h_rows + i * 256;
    const uint32_t lo = s ? row[s - 1] : 0u;
    const uint32_t hi = s == 254 ? 65536u : row[s];
    if (hi <= lo) return LPC_INVALID_ARG;
    e.code16(lo, hi - lo);
  }
  e.finish();
  *out_len = e.size();
  return e.overflow() ? LPC_CAPACITY : LPC_OK;
}

extern "C" int lpc_rc_decode_rows(const uint16_t* h_rows, int64_t n, const uint8_t* h_in,
                                  size_t len, uint8_t* h_syms) {
  if (n < 0 || (n > 0 && (!h_rows || !h_syms)) || (len > 0 && !h_in)) return LPC_INVALID_ARG;
  return lpc::decode_rows(h_rows, (size_t)n, h_in, len, h_syms) ? LPC_OK : LPC_CORRUPT_STREAM;
}
