// Host entropy coding: a range coder with a 32-bit range and byte-wise carry
// propagation (low kept to 33 bits; a settled byte is held back in a cache
// together with a count of pending 0xFF bytes until the carry is known).
// Stream version 3 substreams: the cache's initial byte (always 0, since no
// carry can reach it) is not written, the decoder starts from the first four
// bytes, and the flush codes the value with the most trailing zero bits in
// the final interval and leaves out up to four trailing zero bytes, which
// the decoder reads back as zero.
// Two probability sources: the device-made 16-bit cumulative tables of the
// network levels, and an adaptive symbol-frequency model for the coarse
// levels below b (supplement, "Detailed Model Structure").
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <vector>

namespace lpc {

// Writes into a caller-provided byte range; bytes past `cap` are counted but
// not stored (overflow() reports it).
class RangeEncoder {
 public:
  RangeEncoder(uint8_t* out, size_t cap) : out_(out), cap_(cap) {}
  size_t size() const { return len_; }
  bool overflow() const { return len_ > cap_; }
  // Code the interval [lo, lo + f) of a total 2^16.
  inline void code16(uint32_t lo, uint32_t f) { code(range_ >> 16, lo, f); }
  // Code the interval [lo, lo + f) of an arbitrary total (<= 2^16).
  inline void code_total(uint32_t lo, uint32_t f, uint32_t total) { code(range_ / total, lo, f); }
  void finish();

 private:
  inline void code(uint32_t r, uint32_t lo, uint32_t f) {
    low_ += (uint64_t)r * lo;
    range_ = r * f;
    while (range_ < (1u << 24)) {
      range_ <<= 8;
      shift_low();
    }
  }
  void shift_low();
  inline void put(uint8_t b) {
    if (skip_) {  // the leading cache byte
      skip_ = false;
      return;
    }
    if (len_ < cap_) out_[len_] = b;
    len_++;
  }
  uint8_t* out_;
  size_t cap_, len_ = 0;
  bool skip_ = true;
  uint64_t low_ = 0;
  uint32_t range_ = 0xFFFFFFFFu;
  uint8_t cache_ = 0;
  uint64_t pending_ = 1;
};

class RangeDecoder {
 public:
  RangeDecoder(const uint8_t* p, size_t n);
  // Decode with a table row (u16[256], entry s = C_{s+1}, s = 0..253).
  int decode_row(const uint16_t* row);
  // Range division and update for an arbitrary total (adaptive model).
  inline uint32_t target(uint32_t total) {
    r_ = range_ / total;
    uint32_t v = code_ / r_;
    return v < total ? v : total - 1;
  }
  void update(uint32_t lo, uint32_t f);
  bool bad() const { return bad_ || pos_ > n_ + kPad; }
  // bytes a substream may be short of at its end (read as zero)
  static constexpr size_t kPad = 4;

 private:
  inline uint32_t at(size_t i) const { return i < n_ ? p_[i] : 0u; }
  const uint8_t* p_;
  size_t n_, pos_ = 0;
  uint32_t range_ = 0xFFFFFFFFu, code_ = 0, r_ = 0;
  bool bad_ = false;
};

// Adaptive frequencies of the 255 symbols: start at 1, +32 per coded symbol,
// every count halved (rounding up) once the total exceeds 2^16.  Cumulative
// counts are kept in two levels, 16 groups of 16 symbols: cg[g] = counts
// before group g, cw[s] = counts before s within its group.  The decoder's
// search compares the target with the 16 group bounds, then with the 16
// bounds inside the group (AVX2 compares and a popcount where the host has
// AVX2, plain loops elsewhere); a coded symbol adds 32 to the bounds after
// it (masked adds over 16 lanes).
class AdaptiveModel {
 public:
  AdaptiveModel();
  void encode(RangeEncoder& e, int s);
  int decode(RangeDecoder& d);

 private:
  void rebuild();
  void bump(int s);
  alignas(32) uint32_t cg_[16];
  alignas(32) uint32_t cw_[256];
  uint32_t f_[256];
  uint32_t total_;
};

// Upper bound of the coded size of n symbols: every coded interval is at
// least 2^-16 of the range (at most 2 bytes per symbol) plus the flush.
inline size_t coded_bound(size_t n) { return 2 * n + 8; }
// Encode symbols with per-node (lo, f) pairs packed as lo | f << 16 into
// out[0..cap); returns the byte count (> cap means overflow).
size_t encode_packed(const uint32_t* lofreq, size_t n, uint8_t* out, size_t cap);
// Encode symbols with the adaptive model (one model per substream).
size_t encode_adaptive(const uint8_t* syms, size_t n, uint8_t* out, size_t cap);
// The same from occupancy codes 1..255 (symbol = code - 1).
size_t encode_adaptive_codes(const uint8_t* codes, size_t n, uint8_t* out, size_t cap);
// Decode n symbols with table rows; returns false on a corrupt stream.
bool decode_rows(const uint16_t* rows, size_t n, const uint8_t* in, size_t len, uint8_t* syms);
bool decode_adaptive(size_t n, const uint8_t* in, size_t len, uint8_t* syms);

}  // namespace lpc
