/*
 * lpc_ops.h -- op-level entry points of the B300 codec, for parity tests.
 *
 * Each function runs one step of the hot path on the device, exactly as the
 * codec does inside encode_frame / decode_frame, on caller-provided data.
 * Data arrays are device pointers ("d_"); layer parameters are host pointers
 * ("h_") in the weight-blob layout.  Unlike the codec, these hooks allocate
 * their temporaries (cudaMalloc) per call and synchronise the stream before
 * returning.  Status codes are the LPC_* codes of lpc.h.
 *
 * Node arrays are Morton-sorted u64 keys of one depth (3 bits per level, x
 * the most significant bit of each group).  Activations are int8 row-major
 * [rows][channels].
 */
#ifndef LPC_OPS_H
#define LPC_OPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Octree levels (supplement, "Implementation of Octree Operations"): sort the
 * Morton keys of d_xyz, drop duplicates, then repeatedly halve (key >> 3) and
 * drop consecutive duplicates; the code of a parent ORs 1 << (child key & 7)
 * (the kernel-2 stride-2 all-ones convolution).  Outputs, concatenated over
 * depths: d_keys = V_0..V_L, d_codes = Y_0..Y_{L-1}; h_counts[d] = N_d
 * (L+1 entries).  cap bounds both concatenations. */
int lpc_build_levels(const int32_t* d_xyz, int64_t n, int L, uint64_t* d_keys, uint8_t* d_codes,
                     int64_t* h_counts, int64_t cap, uint64_t stream);

/* Voxel hash + 3x3x3 kernel map at one depth: d_nbr[N][27] = row of the
 * neighbour at offset o = 9(dx+1) + 3(dy+1) + (dz+1), or -1 if absent or
 * outside the cube (Sec. 3.3, sparse conv as indexed linear transforms).
 * table_log2 = log2 of the hash capacity (0 = automatic, >= 2N slots).
 * Errors: LPC_HASH_FULL when the bounded probe sequence finds no slot. */
int lpc_kernel_map(const uint64_t* d_keys, int64_t N, int depth, int32_t* d_nbr, int table_log2,
                   uint64_t stream);

/* The kernel map of a level from the map of its parent level (the octree
 * neighbour rule; Sec. 3.3 builds maps at V_b and V_t, and V_t is the level
 * below V_b): d_ckeys / d_cpar are the Nc children's keys and parent rows,
 * d_pnbr the parents' map [Np][27], d_pcode their occupancy codes and d_poff
 * their first child rows (exclusive scan of the code popcounts).  Writes the
 * same d_nbr[Nc][27] as lpc_kernel_map on the children, without a hash
 * table.  All pointers are device memory owned by the caller; inconsistent
 * inputs (a parent row or child offset out of range) are not detected. */
int lpc_kernel_map_child(const uint64_t* d_ckeys, const uint32_t* d_cpar, int64_t Nc,
                         const int32_t* d_pnbr, const uint8_t* d_pcode, const uint32_t* d_poff,
                         int32_t* d_nbr, uint64_t stream);

/* Kernel map that allocates nothing (the paper has no counterpart; this is a
 * deployment convenience).  Same inputs, output and statuses as
 * lpc_kernel_map with automatic table size, for callers that may not call
 * cudaMalloc at this point (a real-time loop whose memory is fixed at start-up,
 * a component that does not own the CUDA allocator).  The voxel hash table is
 * a file-scope device array of 2^19 slots that every GPU loading the library
 * holds until exit; N above 262,144 nodes returns LPC_CAPACITY.  The first
 * call on each device loads the array's module (CUDA loads modules lazily by
 * default, so that is when the 8 MiB is committed, and it may synchronise
 * the device) and looks up the array's device address: make that first call
 * at start-up, before any stream capture; later calls allocate nothing.  The
 * address is cached per device and goes stale after cudaDeviceReset.  All
 * calls share the array, which keeps
 * the previous call's contents (each call clears what it uses): calls whose
 * GPU work overlaps race with each other and must be serialised by the
 * caller.  Synchronises the stream before returning. */
int lpc_kernel_map_noalloc(const uint64_t* d_keys, int64_t N, int depth, int32_t* d_nbr,
                           uint64_t stream);

/* 3x3x3 sparse conv (Eq. 13-14): out[n] = requant(prelu(bias +
 * sum_{o, present} W[o] (x[nb] - z_in))).  h_W: int8 [27][cout][cin];
 * h_bias, h_mult: int32 [cout]; h_slope: int16 [cout] Q15 or NULL (no PReLU).
 * cin in {32, 64}, cout = 32. */
int lpc_conv333(const uint64_t* d_keys, int64_t N, int depth, const int8_t* d_x, int cin,
                int z_in, const int8_t* h_W, const int32_t* h_bias, const int32_t* h_mult,
                int shift, const int16_t* h_slope, int z_out, int cout, int8_t* d_out,
                uint64_t stream);
/* The same with an explicit kernel variant of the tensor-core conv (0..7,
 * 128-row tiles: bit 0 the alternative ring shape (32 channels: 18 stages
 * in steps of nine offsets), bit 1 contiguous tile order, bit 2 the
 * neighbour rows gathered by TMA gather4 loads (absent neighbours read as
 * zeros without a memory access) instead of 16-byte cp.async copies; 8, 9:
 * 256-row tiles in strided or contiguous order, 32 channels only (with 64
 * channels they run variants 0 and 2); the codec's autotuner picks among
 * them).  Every variant gives the same result; others: LPC_INVALID_ARG. */
int lpc_conv333_variant(const uint64_t* d_keys, int64_t N, int depth, const int8_t* d_x, int cin,
                        int z_in, const int8_t* h_W, const int32_t* h_bias,
                        const int32_t* h_mult, int shift, const int16_t* h_slope, int z_out,
                        int cout, int8_t* d_out, int variant, uint64_t stream);

/* Kernel-2 stride-2 sparse conv from the children (depth k+1, d_ckeys[Nc])
 * to the parents (depth k, d_pkeys[Np]), part of Downsampling (Eq. 4).
 * h_W: int8 [8][cout][cin], slice = child index key & 7. */
int lpc_down_s2(const uint64_t* d_ckeys, int64_t Nc, const uint64_t* d_pkeys, int64_t Np,
                const int8_t* d_x, int cin, int z_in, const int8_t* h_W, const int32_t* h_bias,
                const int32_t* h_mult, int shift, const int16_t* h_slope, int z_out, int cout,
                int8_t* d_out, uint64_t stream);

/* Upsampling + Pruning (Eq. 6): parent p with code d_codes[p]; each set bit c
 * gives the child row (pkey << 3 | c) of d_ckeys with
 * requant_c(prelu_c(bias[c] + W[c] (x[p] - z_in))).  h_W int8 [8][cout][cin];
 * h_bias, h_mult int32 [8][cout]; h_slope int16 [8][cout] or NULL. */
int lpc_up_prune(const uint64_t* d_pkeys, const uint8_t* d_codes, int64_t Np,
                 const uint64_t* d_ckeys, int64_t Nc, const int8_t* d_x, int cin, int z_in,
                 const int8_t* h_W, const int32_t* h_bias, const int32_t* h_mult, int shift,
                 const int16_t* h_slope, int z_out, int cout, int8_t* d_out, uint64_t stream);
/* The same with an explicit kernel variant: 0 CUDA cores (one warp per
 * child, dp4a; what lpc_up_prune runs), 1 tensor cores (each parent row
 * times all eight slots' weights in bf16 MMAs with fp32 accumulators, exact
 * for these magnitudes, then the present children's rows; LPC_TIMEOUT if a
 * bounded wait gave up).  Both give the same bytes. */
int lpc_up_prune_variant(const uint64_t* d_pkeys, const uint8_t* d_codes, int64_t Np,
                         const uint64_t* d_ckeys, int64_t Nc, const int8_t* d_x, int cin,
                         int z_in, const int8_t* h_W, const int32_t* h_bias,
                         const int32_t* h_mult, int shift, const int16_t* h_slope, int z_out,
                         int cout, int8_t* d_out, int variant, uint64_t stream);

/* Integer softmax to cumulative table (Eq. 15): d_logits int8 [N][255],
 * h_lut u32 [256] (lut[0] = 2^16, non-increasing) -> d_cdf u16 [N][256] in
 * the probs_level row format. */
int lpc_softmax_cdf(const int8_t* d_logits, int64_t N, const uint32_t* h_lut, uint16_t* d_cdf,
                    uint64_t stream);

/* Host range coding of one substream with caller tables (the coder the
 * network levels use, Sec. 3.3: the 16-bit cumulative tables drive an
 * entropy coder; stream version 3 framing).  h_rows: host u16 [n][256],
 * entry s = C_{s+1} for s = 0..253 (C_0 = 0, C_255 = 2^16 implicit; entries
 * 254, 255 unused), strictly increasing; h_syms: host symbols 0..254.
 * lpc_rc_encode_rows writes the substream to h_out[0..cap) and its length to
 * *out_len (LPC_CAPACITY, with the required length, if cap is too small;
 * LPC_INVALID_ARG for a symbol above 254).  lpc_rc_decode_rows decodes n
 * symbols from h_in[0..len) with the given rows into h_syms; LPC_CORRUPT_STREAM
 * if the stream is inconsistent with the rows (an interval the decoder's
 * value falls outside of, or reads beyond the four zero bytes a flush may
 * leave out) -- the symbols are then whatever the decoder produced.  Host
 * memory only, no CUDA calls. */
int lpc_rc_encode_rows(const uint16_t* h_rows, const uint8_t* h_syms, int64_t n, uint8_t* h_out,
                       size_t cap, size_t* out_len);
int lpc_rc_decode_rows(const uint16_t* h_rows, int64_t n, const uint8_t* h_in, size_t len,
                       uint8_t* h_syms);

#ifdef __cplusplus
}
#endif
#endif /* LPC_OPS_H */
