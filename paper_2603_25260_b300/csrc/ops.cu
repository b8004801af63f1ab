// Op-level entry points (lpc_ops.h): the codec's own kernels run on
// caller-provided device data, for element-wise parity tests.  These hooks
// allocate their temporaries per call and synchronise before returning.
#include <string.h>

#include <vector>

#include "../../include/lpc_ops.h"
#include "../../include/lpc_train.h"
#include "common.cuh"
#include "kernels.h"
#include "model.h"

using namespace lpc;

namespace {

struct Tmp {
  std::vector<void*> ptrs;
  ~Tmp() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  T* get(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, count * sizeof(T) + 256) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
};

int finish(cudaStream_t st, const int* d_err) {
  int e = 0;
  if (d_err) cudaMemcpyAsync(&e, d_err, 4, cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return LPC_CUDA_ERROR;
  if (e == kErrCoord) return LPC_INVALID_ARG;
  if (e == kErrHashFull) return LPC_HASH_FULL;
  if (e) return LPC_CORRUPT_STREAM;
  return LPC_OK;
}

int64_t* dev_count(Tmp& t, int64_t v, cudaStream_t st) {
  int64_t* p = t.get<int64_t>(1);
  if (p) cudaMemcpyAsync(p, &v, 8, cudaMemcpyHostToDevice, st), cudaStreamSynchronize(st);
  return p;
}

// Layer record for the upload helper: kind 1 (slices summed) or 4 (selected).
int layer_from_host(int kind, int S, int cin, int cout, int z_in, int z_out, int shift,
                    const int8_t* W, const int32_t* bias, const int32_t* mult,
                    const int16_t* slope, DLayer& d, void** mem) {
  const int P = kind == 4 ? S : 1;
  std::vector<int16_t> zero((size_t)P * cout, 0);
  BlobRecord r;
  r.kind = kind;
  r.S = S;
  r.cin = cin;
  r.cout = cout;
  r.z_in = z_in;
  r.z_in2 = 0;
  r.z_out = z_out;
  r.shift = shift;
  r.prelu = slope != nullptr;
  r.W = W;
  r.bias = bias;
  r.mult = mult;
  r.slope = slope ? slope : zero.data();
  return upload_layer(r, d, mem);
}

bool bad_layer(int cin, int cout, int shift) {
  return !(cin == 32 || cin == 64) || cout != 32 || shift < 1 || shift > 62;
}

}  // namespace

extern "C" {

int lpc_build_levels(const int32_t* d_xyz, int64_t n, int L, uint64_t* d_keys, uint8_t* d_codes,
                     int64_t* h_counts, int64_t cap, uint64_t stream) {
  return lpc_t_levels(d_xyz, n, L, d_keys, d_codes, nullptr, nullptr, h_counts, cap, stream);
}

int lpc_t_levels(const int32_t* d_xyz, int64_t n, int L, uint64_t* d_keys, uint8_t* d_codes,
                 uint32_t* d_par, uint32_t* d_off, int64_t* h_counts, int64_t cap,
                 uint64_t stream) {
  if (L < 1 || L > 19 || n < 0 || !h_counts) return LPC_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) {
    for (int d = 0; d <= L; d++) h_counts[d] = 0;
    return LPC_OK;
  }
  Tmp t;
  const int64_t nn = n;
  int64_t* d_n = dev_count(t, nn, st);
  int64_t* d_N = t.get<int64_t>(kMaxDepth + 1);
  int* d_err = t.get<int>(1);
  uint64_t* k0 = t.get<uint64_t>(nn);
  SortScratch ss;
  ss.n_max = nn;
  ss.alt = t.get<uint64_t>(nn);
  ss.hist = t.get<uint32_t>(256 * (sort_tiles(nn) + 1));
  ScanScratch sc;
  sc.max_tiles = scan_tiles_for(nn);
  sc.tiles = t.get<uint32_t>(sc.max_tiles);
  uint64_t* key[kMaxDepth + 1];
  uint8_t* code[kMaxDepth + 1];
  uint32_t *off[kMaxDepth + 1], *par[kMaxDepth + 1];
  int64_t capd[kMaxDepth + 1];
  int64_t c8 = 1;
  for (int d = 0; d <= L; d++) {
    capd[d] = std::min<int64_t>(nn, c8);
    c8 = c8 < ((int64_t)1 << 40) ? c8 * 8 : c8;
    key[d] = t.get<uint64_t>(capd[d]);
    code[d] = t.get<uint8_t>(capd[d]);
    off[d] = t.get<uint32_t>(capd[d] + 1);
    par[d] = t.get<uint32_t>(capd[d]);
  }
  if (!d_n || !d_N || !d_err || !k0 || !ss.alt || !ss.hist || !sc.tiles || !key[L])
    return LPC_CUDA_ERROR;
  cudaMemsetAsync(d_err, 0, 4, st);
  launch_morton(d_xyz, nn, L, k0, d_err, st);
  uint64_t* sorted = radix_sort(k0, nn, 3 * L, false, ss, st);
  launch_unique(sorted, d_n, nn, key[L], d_N + L, sc, st);
  for (int d = L - 1; d >= 0; d--)
    launch_level_up(key[d + 1], d_N + d + 1, capd[d + 1], key[d], code[d], off[d], par[d + 1],
                    d_N + d, sc, st);
  int s = finish(st, d_err);
  if (s) return s;
  cudaMemcpy(h_counts, d_N, 8 * (L + 1), cudaMemcpyDeviceToHost);
  int64_t tot = 0;
  for (int d = 0; d <= L; d++) tot += h_counts[d];
  if (tot > cap) return LPC_CAPACITY;
  int64_t kp = 0, cp = 0, op = 0;
  for (int d = 0; d <= L; d++) {
    if (d_keys)
      cudaMemcpyAsync(d_keys + kp, key[d], 8 * h_counts[d], cudaMemcpyDeviceToDevice, st);
    if (d_par && d > 0)
      cudaMemcpyAsync(d_par + kp, par[d], 4 * h_counts[d], cudaMemcpyDeviceToDevice, st);
    kp += h_counts[d];
    if (d < L) {
      if (d_codes) cudaMemcpyAsync(d_codes + cp, code[d], h_counts[d], cudaMemcpyDeviceToDevice, st);
      if (d_off)
        cudaMemcpyAsync(d_off + op, off[d], 4 * (h_counts[d] + 1), cudaMemcpyDeviceToDevice, st);
      cp += h_counts[d];
      op += h_counts[d] + 1;
    }
  }
  return finish(st, nullptr);
}

int lpc_kernel_map(const uint64_t* d_keys, int64_t N, int depth, int32_t* d_nbr, int table_log2,
                   uint64_t stream) {
  if (N < 0 || depth < 0 || depth > kMaxDepth || table_log2 < 0 || table_log2 > 30)
    return LPC_INVALID_ARG;
  if (N == 0) return LPC_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Tmp t;
  int64_t slots = 1024;
  if (table_log2) slots = (int64_t)1 << table_log2;
  else
    while (slots < 2 * N) slots <<= 1;
  HashTable h;
  h.cap = slots;
  h.slots = t.get<ulonglong2>(slots);
  int64_t* d_n = dev_count(t, N, st);
  int* d_err = t.get<int>(1);
  if (!h.slots || !d_n || !d_err) return LPC_CUDA_ERROR;
  cudaMemsetAsync(d_err, 0, 4, st);
  launch_kernel_map(d_keys, d_n, N, nullptr, depth, h, slots, d_nbr, d_err, st);
  return finish(st, d_err);
}

int lpc_kernel_map_child(const uint64_t* d_ckeys, const uint32_t* d_cpar, int64_t Nc,
                         const int32_t* d_pnbr, const uint8_t* d_pcode, const uint32_t* d_poff,
                         int32_t* d_nbr, uint64_t stream) {
  if (Nc < 0 || (Nc > 0 && (!d_ckeys || !d_cpar || !d_pnbr || !d_pcode || !d_poff || !d_nbr)))
    return LPC_INVALID_ARG;
  if (Nc == 0) return LPC_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Tmp t;
  int64_t* d_n = dev_count(t, Nc, st);
  if (!d_n) return LPC_CUDA_ERROR;
  launch_kernel_map_child(d_ckeys, d_cpar, d_n, Nc, d_pnbr, d_pcode, d_poff, d_nbr, st);
  return finish(st, nullptr);
}

int lpc_conv333_variant(const uint64_t* d_keys, int64_t N, int depth, const int8_t* d_x, int cin,
                        int z_in, const int8_t* h_W, const int32_t* h_bias,
                        const int32_t* h_mult, int shift, const int16_t* h_slope, int z_out,
                        int cout, int8_t* d_out, int variant, uint64_t stream) {
  if (N < 0 || bad_layer(cin, cout, shift) || !h_W || !h_bias || !h_mult || variant < 0 ||
      variant >= kConvVariants)
    return LPC_INVALID_ARG;
  if (N == 0) return LPC_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Tmp t;
  int32_t* nbr = t.get<int32_t>(27 * N);
  if (!nbr) return LPC_CUDA_ERROR;
  int s = lpc_kernel_map(d_keys, N, depth, nbr, 0, stream);
  if (s) return s;
  DLayer L;
  void* mem = nullptr;
  s = layer_from_host(1, 27, cin, cout, z_in, z_out, shift, h_W, h_bias, h_mult, h_slope, L, &mem);
  if (s) return s;
  t.ptrs.push_back(mem);
  int64_t* d_n = dev_count(t, N, st);
  uint16_t* xb = t.get<uint16_t>((size_t)N * cin);
  if (!d_n || !xb || !L.Wtc) return LPC_CUDA_ERROR;
  launch_to_bf16(d_x, cin, cin, z_in, d_n, N, xb, st);
  ConvTcArgs a{};
  a.wimg = L.Wtc;
  a.bias = L.bias;
  a.mult = L.mult;
  a.mult_hi = L.mult_hi;
  a.slope = L.slope;
  a.prelu = L.prelu;
  a.shift = L.shift;
  a.z_out = L.z_out;
  a.nbr = nbr;
  a.d_n = d_n;
  a.xb = xb;
  a.x_stride = cin;
  a.out = d_out;
  a.out_stride = cout;
  launch_conv333_tc(a, cin, N, st, variant);
  s = finish(st, nullptr);
  if (conv_tc_error(true)) return LPC_TIMEOUT;
  return s;
}

int lpc_conv333(const uint64_t* d_keys, int64_t N, int depth, const int8_t* d_x, int cin,
                int z_in, const int8_t* h_W, const int32_t* h_bias, const int32_t* h_mult,
                int shift, const int16_t* h_slope, int z_out, int cout, int8_t* d_out,
                uint64_t stream) {
  return lpc_conv333_variant(d_keys, N, depth, d_x, cin, z_in, h_W, h_bias, h_mult, shift,
                             h_slope, z_out, cout, d_out, 0, stream);
}

int lpc_down_s2(const uint64_t* d_ckeys, int64_t Nc, const uint64_t* d_pkeys, int64_t Np,
                const int8_t* d_x, int cin, int z_in, const int8_t* h_W, const int32_t* h_bias,
                const int32_t* h_mult, int shift, const int16_t* h_slope, int z_out, int cout,
                int8_t* d_out, uint64_t stream) {
  (void)d_pkeys;
  if (Nc < 0 || Np < 0 || bad_layer(cin, cout, shift) || !h_W || !h_bias || !h_mult)
    return LPC_INVALID_ARG;
  if (Np == 0) return LPC_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Tmp t;
  ScanScratch sc;
  sc.max_tiles = scan_tiles_for(Nc);
  sc.tiles = t.get<uint32_t>(sc.max_tiles);
  uint64_t* pk = t.get<uint64_t>(Nc);
  uint8_t* pc = t.get<uint8_t>(Nc);
  uint32_t* poff = t.get<uint32_t>(Nc + 1);
  uint32_t* cpar = t.get<uint32_t>(Nc);
  int64_t* d_nc = dev_count(t, Nc, st);
  int64_t* d_np = t.get<int64_t>(1);
  if (!sc.tiles || !pk || !pc || !poff || !cpar || !d_nc || !d_np) return LPC_CUDA_ERROR;
  launch_level_up(d_ckeys, d_nc, Nc, pk, pc, poff, cpar, d_np, sc, st);
  DLayer L;
  void* mem = nullptr;
  int s = layer_from_host(1, 8, cin, cout, z_in, z_out, shift, h_W, h_bias, h_mult, h_slope, L,
                          &mem);
  if (s) return s;
  t.ptrs.push_back(mem);
  launch_down(L, d_ckeys, poff, d_np, Np, d_x, cin, d_out, cout, 0, st);
  return finish(st, nullptr);
}

int lpc_up_prune(const uint64_t* d_pkeys, const uint8_t* d_codes, int64_t Np,
                 const uint64_t* d_ckeys, int64_t Nc, const int8_t* d_x, int cin, int z_in,
                 const int8_t* h_W, const int32_t* h_bias, const int32_t* h_mult, int shift,
                 const int16_t* h_slope, int z_out, int cout, int8_t* d_out, uint64_t stream) {
  return lpc_up_prune_variant(d_pkeys, d_codes, Np, d_ckeys, Nc, d_x, cin, z_in, h_W, h_bias,
                              h_mult, shift, h_slope, z_out, cout, d_out, 0, stream);
}

int lpc_up_prune_variant(const uint64_t* d_pkeys, const uint8_t* d_codes, int64_t Np,
                         const uint64_t* d_ckeys, int64_t Nc, const int8_t* d_x, int cin,
                         int z_in, const int8_t* h_W, const int32_t* h_bias,
                         const int32_t* h_mult, int shift, const int16_t* h_slope, int z_out,
                         int cout, int8_t* d_out, int variant, uint64_t stream) {
  (void)d_pkeys;
  (void)d_codes;
  if (Nc < 0 || Np < 0 || bad_layer(cin, cout, shift) || !h_W || !h_bias || !h_mult ||
      variant < 0 || variant >= kUpVariants)
    return LPC_INVALID_ARG;
  if (Nc == 0) return LPC_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Tmp t;
  ScanScratch sc;
  sc.max_tiles = scan_tiles_for(Nc);
  sc.tiles = t.get<uint32_t>(sc.max_tiles);
  uint64_t* pk = t.get<uint64_t>(Nc);
  uint8_t* pc = t.get<uint8_t>(Nc);
  uint32_t* poff = t.get<uint32_t>(Nc + 1);
  uint32_t* cpar = t.get<uint32_t>(Nc);
  int64_t* d_nc = dev_count(t, Nc, st);
  int64_t* d_np = t.get<int64_t>(1);
  if (!sc.tiles || !pk || !pc || !poff || !cpar || !d_nc || !d_np) return LPC_CUDA_ERROR;
  launch_level_up(d_ckeys, d_nc, Nc, pk, pc, poff, cpar, d_np, sc, st);
  DLayer L;
  void* mem = nullptr;
  int s = layer_from_host(4, 8, cin, cout, z_in, z_out, shift, h_W, h_bias, h_mult, h_slope, L,
                          &mem);
  if (s) return s;
  t.ptrs.push_back(mem);
  if (variant == 1) {
    if (!L.Wtc) return LPC_CUDA_ERROR;
    const UpTcArgs a{cin,  L.z_in, L.prelu, L.shift, L.z_out, L.mult_hi != nullptr, L.Wtc,  L.bias,
                     L.mult_hi ? L.mult_hi : L.mult, L.slope, d_x,
                     cin,  d_np,   poff,    pc,      d_out,   cout,   0,      EmbSrc{}, 0};
    launch_up_tc(a, std::max<int64_t>(Np, 1), st);
  } else {
    launch_up_prune(L, d_ckeys, cpar, d_nc, Nc, d_x, cin, d_out, cout, 0, st);
  }
  const int s2 = finish(st, nullptr);
  if (up_tc_error(true)) return LPC_TIMEOUT;
  return s2;
}

int lpc_softmax_cdf(const int8_t* d_logits, int64_t N, const uint32_t* h_lut, uint16_t* d_cdf,
                    uint64_t stream) {
  if (N < 0 || !h_lut) return LPC_INVALID_ARG;
  if (N == 0) return LPC_OK;
  if (h_lut[0] != (uint32_t)kFreqTotal) return LPC_INVALID_ARG;
  for (int i = 1; i < 256; i++)
    if (h_lut[i] > h_lut[i - 1]) return LPC_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Tmp t;
  uint32_t* lut = t.get<uint32_t>(256);
  if (!lut) return LPC_CUDA_ERROR;
  cudaMemcpyAsync(lut, h_lut, 1024, cudaMemcpyHostToDevice, st);
  launch_softmax_cdf(d_logits, N, lut, d_cdf, st);
  return finish(st, nullptr);
}

}  // extern "C"
