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
  uint32_t* hist = nullptr;    // 256 * (tiles(n_max) + 1): per-tile counts, digit totals
  int64_t n_max = 0;
};
int64_t sort_tiles(int64_t n);
// Sort n keys by their low `bits` bits and, if frame_bits, by the frame
// bits 58..63 (8-bit digits; digits that are zero for every key are skipped).
// Returns the buffer holding the result (keys or scratch.alt).
uint64_t* radix_sort(uint64_t* keys, int64_t n, int bits, bool frame_bits, const SortScratch& s,
                     cudaStream_t st);

// One frame of a batch, as the device sees it.
struct DevFrame {
  const int32_t* xyz;  // encoder input [n][3]
  int32_t* out;        // decoder output [n][3]
  int64_t n;           // points (encoder) / voxels (decoder)
  int64_t pre;         // first point of the frame in the batch
  int L;               // octree depth
  int pad;
};
// Morton keys of every frame, frame index in bits 58..63.
void launch_morton_batch(const DevFrame* fr, int nf, int64_t total, uint64_t* keys, int* err,
                         cudaStream_t st);
// Level arrays by height (0 = leaves) for the frame-offset search.
constexpr int kHeights = 7;  // heights 0..6 (depths L .. L-6 = b-1 of every frame)
struct LevelPtrs {
  const uint64_t* key[kHeights];
  const int64_t* n[kHeights];
};
void launch_frame_offsets(const LevelPtrs& lv, int nh, int nf, int64_t* foff, cudaStream_t st);
void launch_keys_to_xyz_batch(const uint64_t* keys, const int64_t* d_n, int64_t n_host,
                              const DevFrame* fr, const int64_t* foff0, cudaStream_t st);

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
// parent index of every child (poff and cpar may be null).
void launch_level_up(const uint64_t* ckeys, const int64_t* d_nc, int64_t cap_c, uint64_t* pkeys,
                     uint8_t* pcodes, uint32_t* poff, uint32_t* cpar, int64_t* d_np,
                     const ScanScratch& s, cudaStream_t st);
// Decoder expansion: parents + codes -> children keys (Morton order), parent
// index of every child, child offsets of every parent.  At most cap_c
// children are written (kErrCapacity beyond).
void launch_expand(const uint64_t* pkeys, const uint8_t* pcodes, const int64_t* d_np,
                   int64_t cap_p, uint64_t* ckeys, uint32_t* cpar, uint32_t* poff, int64_t cap_c,
                   int64_t* d_nc, const ScanScratch& s, int* err, cudaStream_t st);

// Coarse heights in one launch each (see octree.cu).
// scan_heights: how many of the lowest coarse heights (7, 8, ...) take the
// multi-block scan (large batches) before the single-block kernel; cap
// bounds their sizes.
// Encoder's coarse heights 7..top from the sorted keys of height 6 (count on
// the device, at most cap6): codes of height h into codes + (h - 7) *
// stride, sizes into cN[h], frame offsets into foff[h * (nf + 1) + f];
// scratch holds 32 * coarse_up_blocks(cap6) words.
int64_t coarse_up_blocks(int64_t cap6);
void launch_coarse_up(const uint64_t* key6, const int64_t* d_n6, int64_t cap6, int top,
                      uint8_t* codes, int64_t stride, int64_t* cN, int nf, int64_t* foff,
                      uint32_t* scratch, cudaStream_t st);
// counts: host copy of the coarse level sizes by height, d_counts the same
// on the device (the large heights expand with the multi-block scan).
void launch_coarse_down(const uint64_t* roots, int top, const uint8_t* codes, int64_t stride,
                        const int64_t* counts, const int64_t* d_counts, int64_t cap, uint64_t* k0,
                        uint64_t* k1, uint64_t* key6, int64_t* n6, const ScanScratch& s, int* err,
                        cudaStream_t st);

// ------------------------------------------------- coarse-level decoding --
// One coarse substream: n symbols of the adaptive model from in[in_off ..
// in_off + in_len) into out[0 .. n) (device) as codes (symbol + 1); fill != 0
// instead writes n copies of the code `fill` (no stream).
struct CoarseChunk {
  int64_t in_off;
  int64_t in_len;
  uint8_t* out;
  int32_t n;
  int32_t fill;
};
// Decode every chunk, one warp each; a corrupt substream sets kErrStream.
void launch_coarse_decode(const CoarseChunk* ck, int n, const uint8_t* in, int* err,
                          cudaStream_t st);
// The popcounts of n codes must add up to expect (kErrStream otherwise).
struct CoarseCheck {
  const uint8_t* codes;
  int64_t n;
  int64_t expect;
};
void launch_coarse_check(const CoarseCheck* ck, int n, int* err, cudaStream_t st);

// ------------------------------------------------------ device range coding --
// One substream: `rows` symbols starting at table / interval row `row`, its
// bytes at `byte_off` of the byte buffer (`byte_len` = stream length when
// decoding, capacity when encoding).
struct RcChunk {
  int64_t row;
  int64_t rows;
  int64_t byte_off;
  int64_t byte_len;
};
// Range-encode every chunk (one thread each) from packed intervals
// lo | f << 16 of a total 2^16; lens[k] = bytes written (kErrCapacity past
// the capacity).  Same bytes as the host encoder.
void launch_rc_encode(const RcChunk* ck, int n, const uint32_t* lofreq, uint8_t* out,
                      uint32_t* lens, int* err, cudaStream_t st);
// Per decoded frame, for the device-built substream tables: the frame's
// substreams are subs[2 (sub0 + s)] (offset in its stream) and
// subs[2 (sub0 + s) + 1] (length), s < nsub; `next` is the first substream
// not yet given to a chunk (advanced level by level); in_base is the frame's
// first byte in the device stream buffer.
struct DevSubFrame {
  int64_t sub0, nsub, chunk, in_base, next;
};
// The substream table of one network level, built on the device: frame f's
// rows foff[f] .. foff[f + 1] - 1 in chunks of its chunk size, each taking
// the frame's next substream.  *d_nck = chunk count.  kErrStream when a
// frame runs out of substreams, kErrCapacity past cap chunks or maxp rows
// of a frame (the table is then cut short).
void launch_rc_chunks(const int64_t* foff, int nf, DevSubFrame* fr, const int64_t* subs,
                      RcChunk* out, int64_t cap, int64_t maxp, int64_t* d_nck, int* err,
                      cudaStream_t st);
// Range-decode every chunk (one warp each) against the cumulative tables
// (u16[256] rows, entry s = C_{s+1}); codes[row + i] = symbol + 1.  A corrupt
// substream sets kErrStream.  Same symbols as the host decoder.
void launch_rc_decode(const RcChunk* ck, int n, const uint16_t* cdf, const uint8_t* in,
                      uint8_t* codes, int* err, cudaStream_t st);
// The same with the chunk count on the device (*d_n <= cap; grid of cap).
void launch_rc_decode_dev(const RcChunk* ck, const int64_t* d_n, int64_t cap, const uint16_t* cdf,
                          const uint8_t* in, uint8_t* codes, int* err, cudaStream_t st);

// ------------------------------------------------------------------ hash --
struct HashTable {
  ulonglong2* slots = nullptr;  // {key, row} pairs
  int64_t cap = 0;              // allocated slots (power of two)
};
// Clear `slots` (power of two <= cap) slots, insert the N keys of one level,
// then write the 27-neighbour map nbr[N][27].  Node depth: Lf[frame] - depth
// for a frame batch (Lf = per-frame octree depths on the device), else
// `depth`.  If pairs != nullptr, the number of present (node, neighbour)
// pairs, centre included, is added to it.  If tmask != nullptr (at least
// conv_tiles(n_host) words), tmask[t] gets bit o set when some node of tile
// t (nodes t kConvTile .. (t + 1) kConvTile - 1) has its offset-o neighbour:
// the conv skips the offsets a tile lacks.
constexpr int kConvTile = 128;  // output nodes per tile of the tensor-core conv
inline int64_t conv_tiles(int64_t n) { return (n + kConvTile - 1) / kConvTile; }
void launch_kernel_map(const uint64_t* keys, const int64_t* d_n, int64_t n_host, const int* Lf,
                       int depth, const HashTable& h, int64_t slots, int32_t* nbr, int* err,
                       cudaStream_t st, uint64_t* pairs = nullptr, uint32_t* tmask = nullptr);
// The 27-neighbour map of a level from its parents' map: ckeys / cpar are the
// children's keys and parent rows (*d_n children), pnbr[Np][27] the parents'
// map, pcode / poff their occupancy codes and first child rows.  Same output
// as launch_kernel_map on the children; no hash table.
void launch_kernel_map_child(const uint64_t* ckeys, const uint32_t* cpar, const int64_t* d_n,
                             int64_t n_host, const int32_t* pnbr, const uint8_t* pcode,
                             const uint32_t* poff, int32_t* nbr, cudaStream_t st,
                             uint64_t* pairs = nullptr, uint32_t* tmask = nullptr);

// ---------------------------------------------------------------- layers --
// Device-resident INT8 layer (blob kinds 1 and 4) in dp4a layout.
struct DLayer {
  int S, cin, cout, z_in, z_out, shift, prelu, per_slice;
  const int32_t* Wp;     // [S][cin/4][cout] packed int8x4 words (output channel fastest)
  const int32_t* wsum;   // [S][cout] sum over input channels of W
  const int32_t* bias;   // [P][cout], P = S if per_slice else 1
  const int32_t* mult;   // [P][cout]
  const int16_t* slope;  // [P][cout]
  const uint16_t* Wtc;   // 27-slice layers, eight-slot up-steps and the predictor's first
                         // layer: packed bf16 weights for the tensor cores
  const int32_t* mult_hi;  // [P][cout] mult x 2^(32 - shift) when every multiplier
                           // admits the high-word requantisation (requant_hi), else null
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

// A code embedding E[Y]: node r's row is the 32-column row code[r] of table
// (its occupancy code's embedding).  A kernel that writes a node's row can
// write its embedding half too, and one that reads it can take it from the
// table, so that no kernel of its own copies it.
struct EmbSrc {
  const int8_t* table = nullptr;  // [256][32]
  const uint8_t* code = nullptr;  // the nodes' codes (the rows' level)
};
// Predictor second layer in the per-lane layout: s = lane * 8 + i.
struct DPred2 {
  int z_in, z_out, shift;
  const int32_t* Wp;     // [8][C/4][32]
  const int32_t* wsum;   // [256]
  const int32_t* bias;   // [256]
  const int32_t* mult;   // [256]
  const uint16_t* Wtc;   // [256][32] bf16, K-major 64-byte swizzled rows (row 255 zero)
};
// Predictor weights for the tensor cores: W [rows][32] int8 -> bf16 rows of
// 64 bytes, K-major, 64-byte swizzled; rows_total >= rows (extra rows zero).
void pack_pred_tc_weights(const int8_t* W, int rows, int rows_total, uint16_t* img);
// Non-zero if a tensor-core predictor gave up on a bounded wait (optionally reset).
int pred_tc_error(bool reset);

// Write E[codes[i]] into columns [col, col + C) of out (row stride `stride`).
void launch_embed(const DEmb& E, const uint8_t* codes, const int64_t* d_n, int64_t n_host,
                  int8_t* out, int stride, int col, cudaStream_t st);



// Upsampling + Pruning: every child r of V_d gets slice (ckey[r] & 7) of the
// layer applied to its parent row x[par[r]] (cin columns, stride x_stride);
// with oe, the output row's columns [oe_col, oe_col + 32) get E[Y] of the
// child's code (the next step's Concat half).
void launch_up_prune(const DLayer& W, const uint64_t* ckey, const uint32_t* cpar,
                     const int64_t* d_nc, int64_t nc_host, const int8_t* x, int x_stride,
                     int8_t* out, int out_stride, int out_col, cudaStream_t st, EmbSrc oe = {},
                     int oe_col = 0);

// The same layer on the tensor cores, walked by parent: every parent row
// times all eight slots' weights (the layer's Wtc image), then the present
// children's rows.  poff [np + 1]: each parent's first child; pcode: each
// parent's occupancy code (bit s = a child in slot s, the children in slot
// order from poff[p]); bias, mult, slope: [8][32] per slot.
struct UpTcArgs {
  int cin, z_in, prelu, shift, z_out;
  int hi;  // mult holds the high-word form
  const uint16_t* wimg;
  const int32_t* bias;
  const int32_t* mult;
  const int16_t* slope;
  const int8_t* x;
  int x_stride;
  const int64_t* d_np;
  const uint32_t* poff;
  const uint8_t* pcode;
  int8_t* out;
  int out_stride, out_col;
  EmbSrc oe;
  int oe_col;
};
void launch_up_tc(const UpTcArgs& a, int64_t np_host, cudaStream_t st);
size_t up_tc_weight_bytes();
void pack_up_tc_weights(const int8_t* W, int cin, uint16_t* img);
// Non-zero if a tensor-core up-step gave up on a bounded wait (optionally reset).
int up_tc_error(bool reset);
// up-step variants: 0 CUDA cores (dp4a, one warp per child), 1 tensor cores
constexpr int kUpVariants = 2;

// Stride-2 down conv: parent p sums slices (ckey & 7) over its children
// off[p]..off[p+1]-1 of x (child rows).
void launch_down(const DLayer& W, const uint64_t* ckey, const uint32_t* poff, const int64_t* d_np,
                 int64_t np_host, const int8_t* x, int x_stride, int8_t* out, int out_stride,
                 int out_col, cudaStream_t st);

// 3x3x3 conv on the tcgen05 tensor cores (conv_tc.cu).  Inputs are bf16 rows
// holding (q - z_in); absent neighbours contribute zero.  With has_res the
// ResBlock's residual merge is fused into the epilogue (y1 = the first conv's
// int8 output).  outb (optional) receives bf16 (q - outb_z) rows for the next
// conv.

// A TMA tensor map (the driver's 128-byte CUtensorMap), kept opaque here.
struct alignas(64) TmaDesc {
  unsigned long long q[16];
};
struct ConvTcArgs {
  TmaDesc tmap;          // the bf16 input rows, set by the launcher (TMA gather)
  int tma_rows;          // the map's row extent: a row index here reads as zeros
  const uint16_t* wimg;  // packed weights, conv_tc_weight_bytes(cin)
  const int32_t* bias;
  const int32_t* mult;
  const int32_t* mult_hi;  // or null: see DLayer::mult_hi
  const int16_t* slope;
  int prelu, shift, z_out;
  const int32_t* nbr;
  const uint32_t* tmask;  // per tile of kConvTile nodes: its present offsets (null: all 27)
  const int2* ranges;     // contiguous order: each CTA's tile run (null: equal tile counts)
  const int64_t* d_n;
  const void* xb;
  int x_stride;  // elements
  int8_t* out;
  int out_stride, out_col;
  void* outb;
  int outb_stride, outb_z;
  int has_res;
  EmbSrc emb;   // optional: E[Y] of the rows' codes into columns [emb_col, emb_col + 32) of out
  int emb_col;
  const int8_t* y1;
  int y1_stride;
  const int32_t* res_mab;
  const int16_t* res_slope;
  int res_z1, res_z2, res_z_out, res_shift;
};
size_t conv_tc_weight_bytes(int cin);
void pack_conv_tc_weights(const int8_t* W, int cin, uint16_t* img);
// variant in [0, kConvVariants): 0..7 are 128-row tiles with ring shape
// (bit 0), tile order (bit 1) and gather schedule (bit 2: cp.async copies,
// or TMA gather4 loads); 8 and 9 are 256-row tiles (32 input channels; with
// 64 the 128-row variants 0 and 2 run instead) in strided or contiguous
// order.  Chosen by the codec's autotuner; every variant gives the same
// result.
constexpr int kConvVariants = 10;
// CTAs of a conv launch over n_host nodes (its grid), and their tile runs
// of about equal cost from the tiles' present-offset masks (ranges[ctas]),
// which the contiguous tile order takes when given.
int conv_ctas(int64_t n_host);
void launch_conv_ranges(const uint32_t* tmask, const int64_t* d_n, int64_t n_host, int2* ranges,
                        cudaStream_t st);
void launch_conv333_tc(const ConvTcArgs& a, int cin, int64_t n_host, cudaStream_t st,
                       int variant = 0);
// int8 rows (stride x_stride) -> bf16 (q - z) rows of `cols` elements.
void launch_to_bf16(const int8_t* x, int x_stride, int cols, int z, const int64_t* d_n,
                    int64_t n_host, void* out, cudaStream_t st);
// The same for the 64 columns of Concat(a, b): 32 int8 columns from each.
void launch_to_bf16_cat(const int8_t* a, int a_stride, const int8_t* b, int b_stride, int z,
                        const int64_t* d_n, int64_t n_host, void* out, cudaStream_t st);
// bf16 rows of Concat(a, E[code]) (a_cols = 32) or of E[code] alone
// (a_cols = 0): the embedding read from its table.
void launch_to_bf16_emb(const int8_t* a, int a_stride, int a_cols, EmbSrc e, int z,
                        const int64_t* d_n, int64_t n_host, void* out, cudaStream_t st);
// Non-zero if a tensor-core conv gave up on a bounded wait (optionally reset).
int conv_tc_error(bool reset);

// The differentiable twin's 3x3x3 conv in bf16 mode on tcgen05: forward
// (mirror 0: in = x [n][cin], out = y [n][32], plus bias) or input gradient
// (mirror 1: in = dy [n][32], out = dx [n][cin], no bias); W [27][32][cin]
// float; operands rounded to bf16, fp32 accumulation.
int tconv_tc(const float* in, int64_t n, int cin, const int32_t* nbr, const float* W,
             const float* bias, float* out, int mirror, cudaStream_t st);
// The up- and down-steps of the twin in bf16 mode on tcgen05 (W [8][cout][cin],
// off [np + 1] the parents' first children, ckey the children's keys):
// tslot_tc gathers each parent's eight child slots (transpose 0: the
// down-step forward, in = child rows [nc][cin], out [np][cout] + bias; 1:
// the up-step's input gradient, in = dy [nc][cout], out [np][cin]);
// texpand_tc multiplies each parent's row by all eight slots and scatters
// each child its slot's 32 columns (transpose 0: the up-step forward, in =
// x [np][cin], out [nc][cout] + per-slot bias [8][cout]; 1: the down-step's
// input gradient, in = dy [np][cout], out [nc][cin]).
int tslot_tc(const float* in, int64_t np, int64_t nc, const uint32_t* off, const uint64_t* ckey,
             const float* W, int cout, int cin, const float* bias, float* out, int transpose,
             cudaStream_t st);
int texpand_tc(const float* in, int64_t np, const uint32_t* off, const uint64_t* ckey,
               const float* W, int cout, int cin, const float* slot_bias, float* out,
               int transpose, cudaStream_t st);
// Weight gradients in bf16 mode on tcgen05, accumulated into dW, each from
// one gather that also gives the input gradient where dx is not null:
// tconv_bwd_tc the conv (dW [27][32][cin], dx [n][cin] from dy [n][32]);
// tup_bwd_tc the up-step (x [np][cin] parents, dy [nc][32] children; dW
// [8][32][cin], dx [np][cin]); tdown_dw_tc the down-step's dW [8][cout][32]
// (x [nc][32] children, dy [np][cout] parents).
int tconv_bwd_tc(const float* x, const float* dy, int64_t n, int cin, const int32_t* nbr,
                 const float* W, float* dx, float* dW, cudaStream_t st);
int tup_bwd_tc(const float* x, const float* dy, int64_t np, int64_t nc, int cin,
               const uint32_t* off, const uint64_t* ckey, const float* W, float* dx, float* dW,
               cudaStream_t st);
int tdown_dw_tc(const float* x, const float* dy, int64_t np, int64_t nc, int cout,
                const uint32_t* off, const uint64_t* ckey, float* dW, cudaStream_t st);

// Predictor + integer softmax + cumulative table.
enum PredMode { kPredCdf = 0, kPredEnc = 1, kPredLogits = 2 };
// variant 0: CUDA cores (dp4a, warp per row); 1: tcgen05 for both linear
// layers (needs the packed bf16 weights).  Same results; the codec's
// autotuner picks.
constexpr int kPredVariants = 2;
void launch_predictor(const DLayer& P1, const DPred2& P2, const uint32_t* lut, const int8_t* F,
                      int f_stride, const int64_t* d_n, int64_t n_host, int mode,
                      const uint8_t* codes, uint16_t* cdf, uint32_t* enc, int8_t* logits,
                      cudaStream_t st, int variant = 0);

// Integer softmax only (logits given), CDF rows out.
void launch_softmax_cdf(const int8_t* logits, int64_t n, const uint32_t* lut, uint16_t* cdf,
                        cudaStream_t st);

}  // namespace lpc
