// Host-side launchers of the codec's CUDA kernels.  Every launcher only
// enqueues work on the given stream; sizes that are known only on the device
// are passed as device pointers (int64) so that a whole encode can be queued
// without host round trips.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lpc {

// Process-wide count of kernel launches issued by this library (every
// launcher adds the number of kernels it enqueues).
void count_launches(int n);
int64_t launches_total();

// ---------------------------------------------------------------- octree --
// Radix sort scratch for up to n_max keys.
struct SortScratch {
  uint64_t* alt = nullptr;     // n_max keys
  uint32_t* hist = nullptr;    // 256 * tiles(n_max)
  int64_t n_max = 0;
};
int64_t sort_tiles(int64_t n);
// Sort n keys (bits = significant low bits of the key).  Returns the buffer
// holding the result (keys or scratch.alt).
uint64_t* radix_sort(uint64_t* keys, int64_t n, int bits, const SortScratch& s, cudaStream_t st);

// xyz int32 [n][3] -> Morton keys; out-of-range coordinates set err.
void launch_morton(const int32_t* xyz, int64_t n, int L, uint64_t* keys, int* err,
                   cudaStream_t st);
// Morton keys of depth L -> xyz int32 [N][3] (N on the device).
void launch_keys_to_xyz(const uint64_t* keys, const int64_t* d_n, int64_t cap, int L,
                        int32_t* xyz, cudaStream_t st);

// Device-wide scan scratch (tile sums).
struct ScanScratch {
  uint32_t* tiles = nullptr;
  int64_t max_tiles = 0;
};
int64_t scan_tiles_for(int64_t cap);

// Unique of sorted keys[0..n) (n on device) -> out[0..*d_nout).
void launch_unique(const uint64_t* keys, const int64_t* d_n, int64_t cap, uint64_t* out,
                   int64_t* d_nout, const ScanScratch& s, cudaStream_t st);
// One level up: children (sorted, unique) -> parents, codes, child offsets,
// parent index of every child.
void launch_level_up(const uint64_t* ckeys, const int64_t* d_nc, int64_t cap_c, uint64_t* pkeys,
                     uint8_t* pcodes, uint32_t* poff, uint32_t* cpar, int64_t* d_np,
                     const ScanScratch& s, cudaStream_t st);
// Decoder expansion: parents + codes -> children keys (Morton order), parent
// index of every child, child offsets of every parent.
void launch_expand(const uint64_t* pkeys, const uint8_t* pcodes, const int64_t* d_np,
                   int64_t cap_p, uint64_t* ckeys, uint32_t* cpar, uint32_t* poff,
                   int64_t* d_nc, const ScanScratch& s, int* err, cudaStream_t st);

// ------------------------------------------------------------------ hash --
struct HashTable {
  uint64_t* keys = nullptr;
  uint32_t* vals = nullptr;
  int64_t cap = 0;  // allocated slots (power of two)
};
// Clear `slots` (power of two <= cap) slots, insert the N keys of one depth,
// then write the 27-neighbour map nbr[N][27].  If pairs != nullptr, the
// number of present (node, neighbour) pairs, centre included, is added to it.
void launch_kernel_map(const uint64_t* keys, const int64_t* d_n, int64_t n_host, int depth,
                       const HashTable& h, int64_t slots, int32_t* nbr, int* err,
                       cudaStream_t st, uint64_t* pairs = nullptr);

// ---------------------------------------------------------------- layers --
// Device-resident INT8 layer (blob kinds 1 and 4) in dp4a layout.
struct DLayer {
  int S, cin, cout, z_in, z_out, shift, prelu, per_slice;
  const int32_t* Wp;     // [S][cin/4][cout] packed int8x4 words (output channel fastest)
  const int32_t* wsum;   // [S][cout] sum over input channels of W
  const int32_t* bias;   // [P][cout], P = S if per_slice else 1
  const int32_t* mult;   // [P][cout]
  const int16_t* slope;  // [P][cout]
};
struct DEmb {
  int cout, z_out;
  const int8_t* table;   // [256][cout]
};
struct DRes {
  int z1, z2, z_out, shift;
  const int32_t* mab;    // [2][C]
  const int16_t* slope;  // [C]
};
// Predictor second layer in the per-lane layout: s = lane * 8 + i.
struct DPred2 {
  int z_in, z_out, shift;
  const int32_t* Wp;     // [8][C/4][32]
  const int32_t* wsum;   // [256]
  const int32_t* bias;   // [256]
  const int32_t* mult;   // [256]
};

// Write E[codes[i]] into columns [col, col + C) of out (row stride `stride`).
void launch_embed(const DEmb& E, const uint8_t* codes, const int64_t* d_n, int64_t n_host,
                  int8_t* out, int stride, int col, cudaStream_t st);

// Upsampling + Pruning: every child r of V_d gets slice (ckey[r] & 7) of the
// layer applied to its parent row x[par[r]] (cin columns, stride x_stride).
void launch_up_prune(const DLayer& W, const uint64_t* ckey, const uint32_t* cpar,
                     const int64_t* d_nc, int64_t nc_host, const int8_t* x, int x_stride,
                     int8_t* out, int out_stride, int out_col, cudaStream_t st);

// Stride-2 down conv: parent p sums slices (ckey & 7) over its children
// off[p]..off[p+1]-1 of x (child rows).
void launch_down(const DLayer& W, const uint64_t* ckey, const uint32_t* poff, const int64_t* d_np,
                 int64_t np_host, const int8_t* x, int x_stride, int8_t* out, int out_stride,
                 int out_col, cudaStream_t st);

// 3x3x3 conv over the kernel map; with res != nullptr the residual merge of
// the ResBlock is fused into the epilogue (y1 = the first conv's output).
void launch_conv333(const DLayer& W, const int32_t* nbr, const int64_t* d_n, int64_t n_host,
                    const int8_t* x, int x_stride, int8_t* out, int out_stride, int out_col,
                    const DRes* res, const int8_t* y1, int y1_stride, cudaStream_t st);

// Predictor + integer softmax + cumulative table.
enum PredMode { kPredCdf = 0, kPredEnc = 1, kPredLogits = 2 };
void launch_predictor(const DLayer& P1, const DPred2& P2, const uint32_t* lut, const int8_t* F,
                      int f_stride, const int64_t* d_n, int64_t n_host, int mode,
                      const uint8_t* codes, uint16_t* cdf, uint32_t* enc, int8_t* logits,
                      cudaStream_t st);

// Integer softmax only (logits given), CDF rows out.
void launch_softmax_cdf(const int8_t* logits, int64_t n, const uint32_t* lut, uint16_t* cdf,
                        cudaStream_t st);

}  // namespace lpc
