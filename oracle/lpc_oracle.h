/*
 * CPU oracle of the integer-only LiDAR geometry codec (arXiv 2603.25260).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-pass restatement
 * of the paper's integer pipeline and of the entropy coder the codec uses.
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no source with the CUDA path.
 *
 * Parity status per function is stated at each declaration ("pinned by ...").
 * The paper prints no worked example of the network as a whole (the level
 * recurrences with their weights): each op is pinned separately, the
 * pipeline by the lossless round trip, and the integer logits of every level
 * and architecture by the separately written FP64 float twin run on the
 * parameters the blob was exported from (within quantisation rounding).
 *
 * All functions return 0 on success or a negative status:
 */
#ifndef LPC_ORACLE_H
#define LPC_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#define OR_OK 0
#define OR_INVALID_ARG (-1)
#define OR_CAPACITY (-2)
#define OR_CORRUPT_STREAM (-4)
#define OR_WEIGHTS_MISMATCH (-5)

#ifdef __cplusplus
extern "C" {
#endif

/* Number of OpenMP threads used by the per-node loops (1 = single thread). */
void or_set_threads(int n);
int or_get_threads(void);
/* Seconds spent by the calling thread's last or_encode / or_decode in the
 * network with its softmax tables and in range coding (CPU-baseline split). */
void or_last_phase_times(double* network_s, double* coding_s);

/* ---- integer primitives (Sec. 3.3, Eq. 13-14; pinned against exact
 *      rational arithmetic in the tests) ---- */
/* clip(round_half_up(acc * m / 2^r) + z, -128, 127) */
int or_requant(int64_t acc, int32_t m, int r, int z);
/* acc >= 0 ? acc : round_half_up(acc * a / 2^15)  (a = Q15 slope) */
int64_t or_prelu(int64_t acc, int a);

/* ---- octree (supplement, "Implementation of Octree Operations") ---- */
/* Morton key of (x, y, z) with `bits` bits per axis; x is the most
 * significant bit of each 3-bit group. */
uint64_t or_morton(uint32_t x, uint32_t y, uint32_t z, int bits);
/* Sorted unique leaf keys of the cloud.  keys_out must hold n entries.
 * Returns the unique count in *n_out.  Pinned by a set-based brute force. */
int or_leaf_keys(const int32_t* xyz, int64_t n, int L, uint64_t* keys_out, int64_t* n_out);
/* All levels: counts[d] = N_d for d = 0..L; keys_out concatenates V_0..V_L,
 * codes_out concatenates Y_0..Y_{L-1}.  cap bounds both concatenations.
 * Pinned by a set-based octree and the kernel-2 stride-2 convolution identity. */
int or_build_levels(const int32_t* xyz, int64_t n, int L, int64_t* counts, uint64_t* keys_out,
                    uint8_t* codes_out, int64_t cap);

/* ---- sparse layers on Morton-sorted node arrays (Eq. 13-14 per node;
 *      pinned against dense integer convolutions on small grids) ---- */
/* 3x3x3 sparse conv at one depth: keys[N] (3*depth-bit Morton keys, sorted),
 * x[N][cin] int8, W[27][cout][cin], per-channel bias/mult/slope.
 * out[N][cout] = requant(prelu(bias + sum_{o, present nb} W[o] (x[nb] - z_in)))
 * offset o = 9(dx+1) + 3(dy+1) + (dz+1).  slope may be NULL (no PReLU). */
int or_conv333(const uint64_t* keys, int64_t N, int depth, const int8_t* x, int cin, int z_in,
               const int8_t* W, const int32_t* bias, const int32_t* mult, int shift,
               const int16_t* slope, int z_out, int cout, int8_t* out);
/* Kernel-2 stride-2 conv from children (depth k+1) to parents (depth k):
 * out[p] = requant(prelu(bias + sum_{child r of p} W[key_r & 7] (x[r] - z_in))) */
int or_down_s2(const uint64_t* ckeys, int64_t Nc, const uint64_t* pkeys, int64_t Np,
               const int8_t* x, int cin, int z_in, const int8_t* W, const int32_t* bias,
               const int32_t* mult, int shift, const int16_t* slope, int z_out, int cout,
               int8_t* out);
/* Up-sampling (8 slices) + pruning: for each parent p and each set bit c of
 * codes[p], the child (pkey << 3 | c) row of ckeys receives
 * requant_c(prelu_c(bias[c] + W[c] (x[p] - z_in))). */
int or_up_prune(const uint64_t* pkeys, const uint8_t* codes, int64_t Np, const uint64_t* ckeys,
                int64_t Nc, const int8_t* x, int cin, int z_in, const int8_t* W,
                const int32_t* bias, const int32_t* mult, int shift, const int16_t* slope,
                int z_out, int cout, int8_t* out);

/* ---- integer softmax -> CDF (Eq. 15 with the exp table; pinned by its
 *      normalisation, floor, monotonicity and float-softmax error bound) ----
 * logits[N][255] int8, lut[256]; cdf[N][256] u16: entry s = C_{s+1} for
 * s = 0..253 (C_0 = 0 and C_255 = 65536 implicit), entries 254, 255 = 0xFFFF. */
int or_softmax_cdf(const int8_t* logits, int64_t N, const uint32_t* lut, uint16_t* cdf);

/* ---- range coder (pinned by round trip and ideal code length) ---- */
/* Code syms[i] in 0..254 with cdf rows (format above).  Returns byte count. */
int or_rc_encode_cdf(const uint16_t* cdf, const uint8_t* syms, int64_t n, uint8_t* out,
                     size_t cap, size_t* out_len);
int or_rc_decode_cdf(const uint16_t* cdf, int64_t n, const uint8_t* in, size_t len,
                     uint8_t* syms);
/* Adaptive frequency model for the coarse levels (one model per call). */
int or_rc_encode_adaptive(const uint8_t* syms, int64_t n, uint8_t* out, size_t cap,
                          size_t* out_len);
int or_rc_decode_adaptive(int64_t n, const uint8_t* in, size_t len, uint8_t* syms);

/* ---- whole codec ---- */
uint64_t or_fnv1a64(const void* data, size_t len);
/* Validate a weight blob; returns 0 or OR_INVALID_ARG. */
int or_check_blob(const void* blob, size_t len);
/* CDF table of level d (b <= d <= L-1) for the cloud: cdf[N_d][256]. */
int or_probs_level(const void* blob, size_t blob_len, const int32_t* xyz, int64_t n, int L,
                   int d, uint16_t* cdf, int64_t cap_nodes, int64_t* n_nodes);
/* Logits (int8 [N_d][255]) of level d, for debugging op chains. */
int or_logits_level(const void* blob, size_t blob_len, const int32_t* xyz, int64_t n, int L,
                    int d, int8_t* logits, int64_t cap_nodes, int64_t* n_nodes);
/* Bitstream of the cloud.  chunk = nodes per network substream. */
int or_encode(const void* blob, size_t blob_len, const int32_t* xyz, int64_t n, int L,
              int chunk, uint8_t* out, size_t cap, size_t* out_len);
/* Decoded voxels (Morton order) as int32 xyz [n_out][3]. */
int or_decode(const void* blob, size_t blob_len, const uint8_t* in, size_t len,
              int32_t* xyz_out, int64_t cap, int64_t* n_out);

#ifdef __cplusplus
}
#endif
#endif
