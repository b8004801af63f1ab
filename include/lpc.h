/*
 * lpc.h -- C ABI of the B300 integer-only LiDAR geometry codec
 * (arXiv 2603.25260, "Towards Practical Lossless Neural Compression for
 * LiDAR Point Clouds").
 *
 * The codec turns integer voxel coordinates into a bitstream and back.  The
 * GPU builds the octree (supplement, "Implementation of Octree Operations"),
 * runs the integer network of Sec. 3 (GRED, Eq. 4-7; XFP, Eq. 8-11; integer
 * linear / sparse conv / requantisation, Eq. 13-14) and the integer softmax
 * (Eq. 15) that turns logits into 16-bit cumulative frequency tables; the
 * host range coder consumes those tables.  All arithmetic that decides a
 * bit of the stream is integer, so a stream written on one device decodes on
 * any other (Sec. 3.3).
 *
 * Conventions for every entry point:
 *  - Return value: an LPC_* status (0 = success, negative = failure).  On
 *    failure `codec_last_error` gives a one-line message.  No entry point
 *    aborts the process; kernels never trap, they record an error word that
 *    the host turns into a status.
 *  - "d_" arguments are device pointers (CUDA global memory on the device the
 *    codec was created on); "h_" arguments are host pointers.  The caller
 *    owns every buffer it passes; the codec owns its internal workspace.
 *  - Coordinates are int32 triples (x, y, z), row-major [n][3], each in
 *    [0, 2^L).  Duplicate points are allowed; the codec works on the set of
 *    occupied voxels.
 *  - All GPU work is issued on the stream given at creation.  Calls return
 *    only after every host buffer they fill is complete; device outputs are
 *    complete in stream order.  A codec is not thread-safe: use one codec per
 *    host thread.
 */
#ifndef LPC_H
#define LPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LPC_OK 0
#define LPC_INVALID_ARG (-1)      /* bad argument, out-of-range coordinate, bad blob */
#define LPC_CAPACITY (-2)         /* an output buffer or the workspace is too small */
#define LPC_HASH_FULL (-3)        /* voxel hash table probe limit reached */
#define LPC_CORRUPT_STREAM (-4)   /* bitstream fails to parse or decode */
#define LPC_WEIGHTS_MISMATCH (-5) /* bitstream written with a different weight blob */
#define LPC_CUDA_ERROR (-6)       /* a CUDA runtime call failed */
#define LPC_TIMEOUT (-7)          /* a bounded device wait gave up */

typedef struct lpc_codec codec_t;

typedef struct {
  int L;              /* maximum octree depth handled (6..19); frames may use L' <= L */
  int C;              /* network width; must equal the blob's (32) */
  int b_off;          /* base level offset: b = L - b_off (5) */
  int t_off;          /* threshold offset: t = L - t_off (4 or 3), Sec. 3.2 and supplement;
                         must equal the blob's */
  int64_t max_points; /* largest point count of one frame */
  int max_frames;     /* largest batch for encode_batch / decode_batch (1..64) */
  int chunk;          /* nodes per entropy-coded substream of a network level (256) */
  int host_threads;   /* host threads for range coding (0 = hardware concurrency) */
  uint64_t cuda_stream; /* cudaStream_t as an integer (0 = legacy default stream) */
  int64_t max_batch_points; /* points of one batch, all frames (0 = max_points * max_frames);
                               sizes the device workspace */
  int host_coding;    /* 0 (default): the network levels are range coded on the device,
                         one thread (encode) or warp (decode) per substream; 1: on host
                         threads from tables copied to the host.  Same bitstream. */
} lpc_config;

/* Create a codec.  `blob` is the integer weight blob (format in the Python
 * package's synth module docstring: exp table, then per-layer INT8 weights,
 * INT32 biases, multipliers, shifts, zero points and Q15 PReLU slopes).  Its
 * header names the architecture -- GRED + XFP (Sec. 3.1-3.2), or one of the
 * ablations of Sec. 4.3: GRED without cross-scale propagation, or neither --
 * and the threshold offset t = L - 4 or L - 3; the same kernels run all of
 * them.  The
 * codec validates it, copies it to the device and keeps its 64-bit FNV-1a
 * hash, which every bitstream header carries.  Allocates all device and
 * pinned-host workspace once, sized by cfg->L and cfg->max_points.
 * Errors: LPC_INVALID_ARG (config or blob), LPC_CUDA_ERROR (allocation). */
int codec_create(const lpc_config* cfg, const void* blob, size_t blob_len, codec_t** out);

/* Free every resource of the codec (NULL is allowed). */
void codec_destroy(codec_t* codec);

/* Message of the last failure on this codec ("" after success). */
const char* codec_last_error(codec_t* codec);

/* Encode one frame.  d_xyz: device int32 [n][3].  The bitstream goes to the
 * caller's host buffer h_out of `cap` bytes; *out_len receives its length.
 * Stream (version 3): "LPC1", version, L, b, t, C, flags, the blob's hash,
 * then varints: network chunk, coarse chunk (512), the coarse levels' sizes
 * N_1 .. N_{b-1}, the substream count, and each substream's length as the
 * zigzag-coded difference to the previous one's; then the substreams: the
 * coarse levels in coarse chunks (adaptive symbol frequencies, a fresh model
 * each), the network levels in network chunks (the integer softmax tables).
 * A substream is range coded without the coder's always-zero leading byte
 * and ends with the shortest flush (up to four trailing zero bytes left out
 * and read back as zero). 
 * If cap is too small, returns LPC_CAPACITY with the required length in
 * *out_len.  n = 0 gives an empty-frame stream.
 * Errors: LPC_INVALID_ARG (coordinate outside [0, 2^L)), LPC_CAPACITY
 * (n > max_points or small h_out), LPC_HASH_FULL, LPC_CUDA_ERROR. */
int encode_frame(codec_t* codec, const int32_t* d_xyz, int64_t n, uint8_t* h_out, size_t cap,
                 size_t* out_len);

/* Decode one bitstream (host bytes) into device int32 [n_out][3] voxel
 * coordinates, unique and in Morton order (x the most significant bit of each
 * 3-bit group).  cap = capacity of d_xyz_out in points; if too small,
 * returns LPC_CAPACITY with the voxel count in *n_out.
 * Errors: LPC_CORRUPT_STREAM, LPC_WEIGHTS_MISMATCH, LPC_CAPACITY,
 * LPC_CUDA_ERROR. */
int decode_frame(codec_t* codec, const uint8_t* h_in, size_t len, int32_t* d_xyz_out,
                 int64_t cap, int64_t* n_out);

/* Parity hook: the cumulative frequency table of network level d
 * (b <= d <= L-1) for a frame, on the device.  d_cdf_out: u16 [N_d][256];
 * row entry s = C_{s+1} = f_0 + ... + f_s for s = 0..253 (C_0 = 0 and
 * C_255 = 65536 are implicit), entries 254 and 255 are 0xFFFF.  The f_s are
 * the 16-bit integer softmax frequencies of Eq. 15 (every f_s >= 1, sum 2^16).
 * cap_nodes: rows available; *n_nodes receives N_d (LPC_CAPACITY if larger).
 * d_cdf_out must be 16-byte aligned (LPC_INVALID_ARG otherwise).
 * Only the network runs; nothing is entropy coded. */
int probs_level(codec_t* codec, const int32_t* d_xyz, int64_t n, int d, uint16_t* d_cdf_out,
                int64_t cap_nodes, int64_t* n_nodes);

/* Batched encode: nf frames (nf <= max_frames), frame i has n[i] points at
 * d_xyz[i] (device) and depth Ls[i] (6..cfg->L).  All frames share the level
 * arrays (frame index in the top key bits) and are aligned by relative level
 * d - b, so every network level of every frame goes through one launch
 * sequence; the host codes all frames' substreams in parallel.  The output
 * for frame i is byte-identical to encode_frame of that frame: h_out[i]
 * (capacity caps[i]) receives out_lens[i] bytes.  Returns the first failing
 * status (per-frame CAPACITY reports the needed length). */
int encode_batch(codec_t* codec, int nf, const int32_t* const* d_xyz, const int64_t* n,
                 const int* Ls, uint8_t* const* h_out, const size_t* caps, size_t* out_lens);

/* Batched decode: the mirror of encode_batch.  Frame i's voxels go to
 * d_xyz_out[i] (capacity caps[i] points), count in n_out[i]. */
int decode_batch(codec_t* codec, int nf, const uint8_t* const* h_in, const size_t* lens,
                 int32_t* const* d_xyz_out, const int64_t* caps, int64_t* n_out);

/* Per-frame statistics of the last encode_frame / decode_frame call:
 * counts[d] = N_d for d = 0..L (L+1 entries), and the time split in
 * microseconds (GPU part, host coding part).  Returns the depth L. */
int codec_last_stats(codec_t* codec, int64_t* counts, double* gpu_us, double* host_us);

/* Kernel-family profiler.  codec_profile(mask) resets the counters and times
 * every later launch of the families whose bit is set in `mask` with CUDA
 * events on the codec's stream (0 turns it off).  Families: 0 sort (Morton +
 * radix sort + unique), 1 levels (level build / decoder expansion), 2 hash_kmap,
 * 3 embed (code embeddings and the bf16 conversions of the conv inputs),
 * 4 up_prune, 5 down_s2, 6 conv333, 7 predictor_cdf, 8 range_coder.
 * codec_profile_read returns, for one family, the summed launch time (ms),
 * the launch count, and the algorithmic bytes and integer ops those launches
 * must touch (counted from level sizes and neighbour pairs, not from the
 * kernels' actual traffic).  codec_profile_staged returns the bytes those
 * launches actually move in this implementation's layouts (for the 3x3x3
 * conv: bf16 gathered rows, the 27-entry map rows, the bf16 copy of the
 * output and the bf16 weight image; for every other family the algorithmic
 * figure).  codec_profile_name gives the family's name. */
int codec_profile(codec_t* codec, unsigned family_mask);
int codec_profile_read(codec_t* codec, int family, double* ms, int64_t* launches, double* bytes,
                       double* ops);
int codec_profile_staged(codec_t* codec, int family, double* bytes);
const char* codec_profile_name(int family);

/* Autotuner state (variants[5], ms[26]): variants[0], variants[1] = the
 * chosen variant of the tensor-core 3x3x3 conv for 32- and 64-channel inputs
 * (-1 while untuned), ms[c * 10 + v] = the timed milliseconds of variant v
 * (v < 8: 128-row tiles, bit 0: alternative ring shape, bit 1: contiguous
 * tile order, bit 2: the neighbour rows gathered by TMA gather4 loads
 * instead of cp.async copies; v = 8, 9: 256-row tiles in strided or
 * contiguous order, for 64-channel inputs the 128-row variants 0 and 2);
 * variants[2] = the predictor's (0 CUDA cores, 1 tensor cores), ms[20 + v]
 * its timings; variants[3], variants[4] = the Upsampling + Pruning step's
 * for 32- and 64-channel inputs (0 CUDA cores, the children slot by slot;
 * 1 tensor cores, each parent against all eight slots), ms[22 + 2 c + v]
 * their timings.
 * Tuning runs on the first encode or decode; every variant gives the same
 * result. */
int codec_tuning(codec_t* codec, int* variants, float* ms);
/* Fix the variants (conv 32, conv 64, predictor, up 32, up 64) instead of
 * tuning them; -1 leaves one to the tuner.  LPC_INVALID_ARG for an unknown
 * variant. */
int codec_set_tuning(codec_t* codec, const int* variants);

/* Host timeline of the last encode / decode, microseconds (diagnostic):
 * [0] octree ready, [1] launches issued, [2] coding done, [3] encode total;
 * [4] coarse levels decoded, [5] network issue, [6] level decoding,
 * [7] expansion issue (sums over levels), [8] decode total; encode again:
 * [9] coarse keys on the host, [10] device work done, [11] host coding done;
 * decode again: [12] streams parsed and sent to the device, [13] coarse
 * substreams decoded, [14] coarse sizes checked (then [4] after their
 * expansion on the device). */
int codec_last_phases(codec_t* codec, double* us, int n);

/* Number of CUDA kernels this library has launched in this process so far
 * (all codecs and op entry points together). */
int64_t lpc_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* LPC_H */
