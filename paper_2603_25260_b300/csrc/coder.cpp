#include "coder.h"

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
  for (int i = 0; i < 5; i++) shift_low();
}

RangeDecoder::RangeDecoder(const uint8_t* p, size_t n) : p_(p), end_(p + n) {
  for (int i = 0; i < 5; i++) code_ = (code_ << 8) | next();
}

void RangeDecoder::update(uint32_t lo, uint32_t f) {
  code_ -= r_ * lo;
  range_ = r_ * f;
  if (code_ >= range_) bad_ = true;
  while (range_ < (1u << 24)) {
    code_ = (code_ << 8) | next();
    range_ <<= 8;
  }
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
  for (int i = 0; i <= 256; i++) tree_[i] = 0;
  for (int i = 0; i < 255; i++) {
    for (int k = i + 1; k <= 255; k += k & (-k)) tree_[k] += f_[i];
  }
}

uint32_t AdaptiveModel::prefix(int s) const {
  uint32_t r = 0;
  for (int k = s; k > 0; k -= k & (-k)) r += tree_[k];
  return r;
}

void AdaptiveModel::add(int s, int32_t v) {
  for (int k = s + 1; k <= 255; k += k & (-k)) tree_[k] += (uint32_t)v;
}

void AdaptiveModel::bump(int s) {
  f_[s] += 32;
  total_ += 32;
  add(s, 32);
  if (total_ > 65536u) {
    total_ = 0;
    for (int i = 0; i < 255; i++) {
      f_[i] = (f_[i] + 1) >> 1;
      total_ += f_[i];
    }
    rebuild();
  }
}

void AdaptiveModel::encode(RangeEncoder& e, int s) {
  e.code_total(prefix(s), f_[s], total_);
  bump(s);
}

int AdaptiveModel::decode(RangeDecoder& d) {
  const uint32_t v = d.target(total_);
  // largest s with prefix(s) <= v (binary lifting over the Fenwick tree)
  int pos = 0;
  uint32_t rem = v;
  for (int step = 128; step; step >>= 1) {
    if (pos + step <= 255 && tree_[pos + step] <= rem) {
      pos += step;
      rem -= tree_[pos];
    }
  }
  if (pos > 254) pos = 254;
  d.update(v - rem, f_[pos]);
  bump(pos);
  return pos;
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
