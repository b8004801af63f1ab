/*
 * lpc_train.h -- differentiable (quantisation-aware) twin of the codec's
 * network ops, for training on the rate loss (the occupancy cross-entropy of
 * the supplement's training section, in bits).
 *
 * Every op has a forward and a hand-written backward kernel.  Tensors are
 * device float32, row-major [rows][channels]; "bf16" = 1 rounds the operands
 * of every product to bf16 before multiplying (accumulation stays float32).
 * Weight layouts follow the integer blob: W[slices][cout][cin].  Backward
 * calls ADD into dW / db / dE / da (zero them first); dx is overwritten and
 * may be NULL when not needed.  All calls return LPC_* statuses (lpc.h) and
 * are asynchronous on `stream`.
 *
 * Index structures (integer, not differentiated) come from the codec's octree
 * and kernel-map builders: nbr[N][27] neighbour rows (-1 absent); par[r] the
 * parent row of child r; off[p]..off[p+1] the child rows of parent p;
 * ckey[r] & 7 the child slot of r.
 */
#ifndef LPC_TRAIN_H
#define LPC_TRAIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Sparse 3x3x3 conv (Eq. 5): y[i] = b + sum_o W[o] x[nbr[i][o]].  With
 * bf16 = 1 the forward and the input gradient run as gather-GEMMs on the
 * tcgen05 tensor cores (bf16 operands, fp32 accumulators in tensor memory);
 * they use a device scratch the library grows on demand (cudaMalloc on the
 * first calls and on growth only).  lpc_t_tc_error reports (and with
 * reset = 1 clears) a tensor-core launch that gave up on a bounded wait. */
int lpc_t_conv_fwd(const float* x, int64_t N, int cin, const int32_t* nbr, const float* W,
                   const float* b, int cout, float* y, int bf16, uint64_t stream);
/* dx[i] = sum_o W[o]^T dy[nbr[i][26 - o]] (mirror offset); dW[o] += sum_i
 * dy[i] x[nbr[i][o]]^T; db += sum_i dy[i]. */
int lpc_t_conv_bwd(const float* x, const float* dy, int64_t N, int cin, const int32_t* nbr,
                   const float* W, int cout, float* dx, float* dW, float* db, int bf16,
                   uint64_t stream);
int lpc_t_tc_error(int reset);

/* Upsampling + Pruning (Eq. 6): y[r] = b[c] + W[c] x[par[r]], c = ckey[r] & 7.
 * x [Np][cin]; off [Np + 1] the parents' first children (children of parent
 * p: off[p] .. off[p + 1] - 1).  bf16 mode with cout = 32 runs on the tensor
 * cores: every parent against all eight slots' weights, each child taking
 * its slot's columns. */
int lpc_t_up_fwd(const float* x, int64_t Np, int cin, const uint32_t* off, const uint32_t* par,
                 const uint64_t* ckey, int64_t Nc, const float* W, const float* b, int cout,
                 float* y, int bf16, uint64_t stream);
/* dx[p] = sum over children r of W[c_r]^T dy[r]; dW[c] += sum_{c_r = c} dy[r]
 * x[par r]^T; db[c] += sum_{c_r = c} dy[r].  bf16 mode with cout = 32 takes dx
 * on the tensor cores (a gather of each parent's eight child slots). */
int lpc_t_up_bwd(const float* x, const float* dy, int64_t Np, int cin, const uint32_t* off,
                 const uint32_t* par, const uint64_t* ckey, int64_t Nc, const float* W, int cout,
                 float* dx, float* dW, float* db, int bf16, uint64_t stream);

/* Stride-2 down conv (Eq. 4): y[p] = b + sum_{r child of p} W[c_r] x[r].
 * bf16 mode with cin = 32 runs on the tensor cores (a gather of each
 * parent's eight child slots). */
int lpc_t_down_fwd(const float* x, int64_t Nc, int cin, const uint32_t* off, const uint64_t* ckey,
                   int64_t Np, const float* W, const float* b, int cout, float* y, int bf16,
                   uint64_t stream);
/* dx[r] = W[c_r]^T dy[par r]; dW[c] += sum_{c_r = c} dy[par r] x[r]^T;
 * db += sum_p dy[p].  off [Np + 1] as for lpc_t_up_fwd; bf16 mode with
 * cin = 32 takes dx on the tensor cores (every parent's dy against all eight
 * slots' transposed weights, each child taking its slot's columns). */
int lpc_t_down_bwd(const float* x, const float* dy, int64_t Nc, int cin, const uint32_t* off,
                   const uint32_t* par, const uint64_t* ckey, int64_t Np, const float* W,
                   int cout, float* dx, float* dW, float* db, int bf16, uint64_t stream);

/* Occupancy-code embedding: y[i] = E[codes[i]]; dE[codes[i]] += dy[i]. */
int lpc_t_embed_fwd(const uint8_t* codes, int64_t N, const float* E, int C, float* y,
                    uint64_t stream);
int lpc_t_embed_bwd(const uint8_t* codes, int64_t N, const float* dy, int C, float* dE,
                    uint64_t stream);

/* PReLU with a per-channel slope a[C]. */
int lpc_t_prelu_fwd(const float* x, int64_t N, int C, const float* a, float* y, uint64_t stream);
int lpc_t_prelu_bwd(const float* x, const float* dy, int64_t N, int C, const float* a, float* dx,
                    float* da, uint64_t stream);

/* Fake quantisation of Eq. 12 with a straight-through gradient:
 * y = (clip(round(x / s) + z, -128, 127) - z) s; mask[i] = 1 where the clip
 * is inactive; dx = dy * mask. */
int lpc_t_fq_fwd(const float* x, int64_t n, float s, int z, float* y, uint8_t* mask,
                 uint64_t stream);
int lpc_t_fq_bwd(const float* dy, const uint8_t* mask, int64_t n, float* dx, uint64_t stream);
/* Weight fake quantisation with the scale found on the device: s = max|w|/127
 * (max|w| at least 1e-12; formed in double, rounded to float), then the same
 * as lpc_t_fq_fwd with z = 0 (no host round trip for the scale).  w, y, mask
 * device arrays of n elements owned by the caller. */
int lpc_t_fq_w(const float* w, int64_t n, float* y, uint8_t* mask, uint64_t stream);

/* Predictor (Eq. 7) and rate loss (supplement, Training, Eq. 16), fused:
 * per row i of F [N][32], x = q(F[i]), h = prelu(W1 x + b1, a1), l = W2 q(h)
 * + b2 (255 logits), and bits += -log2 softmax(l)[codes[i] - 1].  W1 [32][32],
 * b1, a1 [32], W2 [255][32], b2 [255]; codes u8 [N] in 1..255; q = the fake
 * quantiser of lpc_t_fq_fwd at s = 1/32, z = 0 when qat = 1, else identity.
 * *bits (device double) is added to; logits, if not NULL, receives l [N][255]
 * (float).  The backward recomputes the rows and, from the device scalar
 * *dbits = d(loss)/d(bits), writes dF [N][32] (may be NULL) and adds into dW1,
 * db1, da1, dW2, db2 (zero them first); the logits and their gradients never
 * reach device memory. */
int lpc_t_pred_fwd(const float* F, int64_t N, const float* W1, const float* b1, const float* a1,
                   const float* W2, const float* b2, const uint8_t* codes, int qat, int bf16,
                   float* logits, double* bits, uint64_t stream);
int lpc_t_pred_bwd(const float* F, int64_t N, const float* W1, const float* b1, const float* a1,
                   const float* W2, const float* b2, const uint8_t* codes, int qat, int bf16,
                   const float* dbits, float* dF, float* dW1, float* db1, float* da1, float* dW2,
                   float* db2, uint64_t stream);

/* Octree levels with parent rows and child offsets, for the index
 * structures above: concatenations over depths 0..L (keys, par) and
 * 0..L-1 (codes, off with N_d + 1 entries each); counts[d] = N_d. */
int lpc_t_levels(const int32_t* d_xyz, int64_t n, int L, uint64_t* d_keys, uint8_t* d_codes,
                 uint32_t* d_par, uint32_t* d_off, int64_t* h_counts, int64_t cap,
                 uint64_t stream);

#ifdef __cplusplus
}
#endif
#endif /* LPC_TRAIN_H */
