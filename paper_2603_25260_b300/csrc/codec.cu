// Codec orchestration: workspace, octree build, the per-level network
// schedule of Sec. 3 (GRED + XFP), and host range coding of the
// device-made cumulative tables.  Exported through the C ABI of lpc.h.
#include "codec.h"

#include <string.h>

#include <algorithm>
#include <chrono>

#include "coder.h"

namespace lpc {

// ------------------------------------------------------------------ pool --
Pool::Pool(int workers) {
  for (int i = 0; i < workers; i++) th_.emplace_back([this] { loop(); });
}

Pool::~Pool() {
  {
    std::lock_guard<std::mutex> g(mu_);
    stop_ = true;
  }
  cv_.notify_all();
  for (auto& t : th_) t.join();
}

// Runs the next queued task (lock held on entry and on return).
bool Pool::run_one(std::unique_lock<std::mutex>& lk) {
  if (head_ >= q_.size()) return false;
  std::function<void()> f = std::move(q_[head_++]);
  lk.unlock();
  f();
  lk.lock();
  if (--pending_ == 0) {
    q_.clear();
    head_ = 0;
    done_.notify_all();
  }
  return true;
}

void Pool::loop() {
  std::unique_lock<std::mutex> lk(mu_);
  for (;;) {
    cv_.wait(lk, [&] { return stop_ || head_ < q_.size(); });
    if (stop_) return;
    run_one(lk);
  }
}

void Pool::submit(std::function<void()> task) {
  if (th_.empty()) {
    task();
    return;
  }
  {
    std::lock_guard<std::mutex> g(mu_);
    q_.push_back(std::move(task));
    pending_++;
  }
  cv_.notify_one();
}

void Pool::wait() {
  std::unique_lock<std::mutex> lk(mu_);
  while (pending_ > 0) {
    if (!run_one(lk)) done_.wait(lk, [&] { return pending_ == 0 || head_ < q_.size(); });
  }
}

// ------------------------------------------------------------ bitstream --
// "LPC1", u8 version, u8 L, u8 b, u8 t, u8 C, u8 flags (bit0: empty frame),
// u64 blob hash (little endian), varint chunk, varint n_sub, n_sub varint
// lengths, then the substreams: coarse levels 0..b-1 (adaptive model, one
// each), then every network level d = b..L-1 in chunks of `chunk` nodes.
namespace {

constexpr int kHdr = 18;

void put_varint(std::vector<uint8_t>& o, uint64_t v) {
  while (v >= 0x80) {
    o.push_back((uint8_t)(v | 0x80));
    v >>= 7;
  }
  o.push_back((uint8_t)v);
}

bool get_varint(const uint8_t* in, size_t len, size_t& pos, uint64_t& v) {
  v = 0;
  for (int sh = 0; sh < 64; sh += 7) {
    if (pos >= len) return false;
    const uint8_t c = in[pos++];
    v |= (uint64_t)(c & 0x7F) << sh;
    if (!(c & 0x80)) return true;
  }
  return false;
}

double now_us() {
  return std::chrono::duration<double, std::micro>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace

// ---------------------------------------------------------------- create --
Codec::~Codec() {
  delete pool_;
  for (auto e : ev_) cudaEventDestroy(e);
  if (dmem_) cudaFree(dmem_);
  if (hmem_) cudaFreeHost(hmem_);
  model_free(M_);
}

int Codec::cuda_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LPC_CUDA_ERROR, std::string(what) + ": " + cudaGetErrorString(e));
  return LPC_OK;
}

int64_t Codec::hash_slots(int64_t n) const {
  int64_t s = 1024;
  while (s < 2 * n) s <<= 1;
  return std::min<int64_t>(s, hash_.cap);
}

int Codec::create(const lpc_config& cfg, const void* blob, size_t len) {
  cfg_ = cfg;
  if (cfg.L < 6 || cfg.L > kMaxDepth || cfg.C != 32 || cfg.b_off != 5 || cfg.t_off != 4 ||
      cfg.max_points < 1 || cfg.max_points > (int64_t)1 << 31 || cfg.max_frames < 1 ||
      cfg.chunk < 1)
    return fail(LPC_INVALID_ARG,
                "config: need 6 <= L <= 21, C = 32, b_off = 5, t_off = 4, max_points >= 1, "
                "max_frames >= 1, chunk >= 1");
  st_ = reinterpret_cast<cudaStream_t>(cfg.cuda_stream);
  int s = model_load(blob, len, M_, err);
  if (s) return s;
  const int64_t P = cfg.max_points;
  const int L = cfg.L;
  // ---- device workspace (one allocation, 256-byte aligned slices) ----
  struct Slice {
    void** p;
    size_t bytes;
  };
  std::vector<Slice> sl;
  auto add = [&](void** p, size_t bytes) { sl.push_back({p, bytes}); };
  int64_t cap = 1;
  for (int d = 0; d <= L; d++) {
    lv_.cap[d] = std::min<int64_t>(P, cap);
    if (cap < ((int64_t)1 << 40)) cap *= 8;
    add((void**)&lv_.key[d], 8 * lv_.cap[d]);
    add((void**)&lv_.code[d], lv_.cap[d] + 16);
    add((void**)&lv_.off[d], 4 * (lv_.cap[d] + 1));
    add((void**)&lv_.par[d], 4 * lv_.cap[d]);
  }
  add((void**)&d_N_, 8 * (kMaxDepth + 2));
  add((void**)&d_err_, 16);
  add((void**)&d_pairs_, 16);
  add((void**)&d_keys0_, 8 * P);
  sort_.n_max = P;
  add((void**)&sort_.alt, 8 * P);
  add((void**)&sort_.hist, 4 * 256 * sort_tiles(P));
  scan_.max_tiles = scan_tiles_for(P);
  add((void**)&scan_.tiles, 4 * scan_.max_tiles);
  hash_.cap = 1024;
  while (hash_.cap < 2 * P) hash_.cap <<= 1;
  add((void**)&hash_.keys, 8 * hash_.cap);
  add((void**)&hash_.vals, 4 * hash_.cap);
  add((void**)&nbr_b_, 4 * 27 * P);
  add((void**)&nbr_t_, 4 * 27 * P);
  add((void**)&fb_, 32 * P);
  add((void**)&xb_, 64 * P);
  add((void**)&xt_, 64 * P);
  add((void**)&y1_, 32 * P);
  add((void**)&xb16_, 2 * 64 * P);
  add((void**)&y1b16_, 2 * 32 * P);
  add((void**)&xe_, 32 * P);
  add((void**)&g_[0], 32 * P);
  add((void**)&g_[1], 32 * P);
  add((void**)&hx_[0], 64 * P);
  add((void**)&hx_[1], 64 * P);
  add((void**)&fo_, 32 * P);
  add((void**)&d_cdf_, 512 * P);
  add((void**)&d_enc_, 4 * 5 * P);
  size_t total = 0;
  for (auto& x : sl) total += (x.bytes + 255) / 256 * 256;
  if (cudaMalloc(&dmem_, total) != cudaSuccess) {
    cudaGetLastError();
    dmem_ = nullptr;
    return fail(LPC_CUDA_ERROR, "workspace allocation failed");
  }
  size_t off = 0;
  for (auto& x : sl) {
    *x.p = static_cast<uint8_t*>(dmem_) + off;
    off += (x.bytes + 255) / 256 * 256;
  }
  // ---- pinned host workspace ----
  // The coded substreams of one frame fit in 2 bytes per symbol plus 8 per
  // substream (coded_bound); the arena is pinned so that host threads write
  // it without page faults.
  const int64_t max_subs = L + (5 * P) / cfg.chunk + 5;
  arena_cap_ = (size_t)2 * (L + 1) * P + (size_t)8 * max_subs + 1024;
  const size_t hN = 8 * (kMaxDepth + 2), hE = 16, hC = (size_t)(L + 1) * P + 64,
               hEnc = (size_t)4 * 5 * P, hCdf = (size_t)512 * P;
  const size_t hA = (arena_cap_ + 255) / 256 * 256;
  const size_t htotal = hN + hE + (hC + 255) / 256 * 256 + hEnc + hCdf + hA + 1024;
  if (cudaMallocHost(&hmem_, htotal) != cudaSuccess) {
    cudaGetLastError();
    hmem_ = nullptr;
    return fail(LPC_CUDA_ERROR, "pinned host allocation failed");
  }
  uint8_t* h = static_cast<uint8_t*>(hmem_);
  h_N_ = reinterpret_cast<int64_t*>(h);
  h_err_ = reinterpret_cast<int*>(h + hN);
  h_codes_ = h + hN + hE;
  h_enc_ = reinterpret_cast<uint32_t*>(h + hN + hE + (hC + 255) / 256 * 256);
  h_cdf_ = reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(h_enc_) + hEnc);
  h_arena_ = reinterpret_cast<uint8_t*>(h_cdf_) + hCdf;
  const int nev = (int)(P / cfg.chunk) + 8;
  ev_.resize(nev);
  for (auto& e : ev_) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  int threads = cfg.host_threads > 0 ? cfg.host_threads : (int)std::thread::hardware_concurrency();
  pool_ = new Pool(std::max(0, threads - 1));
  return cuda_check("codec_create");
}

// ------------------------------------------------------------ per frame --
void Codec::begin_frame(int L) {
  L_ = L;
  b_ = L - cfg_.b_off;
  t_ = L - cfg_.t_off;
  have_Fb_ = have_Ft_ = have_nbr_t_ = false;
  if (prof.mask) cudaMemsetAsync(d_pairs_, 0, 16, st_);
}

// Algorithmic bytes of the level build once the sizes are known.
void Codec::level_bytes(int L) {
  double b = 0;
  for (int d = 0; d < L; d++) b += 8.0 * N_[d + 1] + 4.0 * N_[d + 1] + 13.0 * N_[d] + 4.0;
  for (auto it = marks_.rbegin(); it != marks_.rend(); ++it)
    if (it->f == kFamLevels) {
      it->bytes = b;
      break;
    }
}

int Codec::check_device_error() {
  if (conv_tc_error(true)) return fail(LPC_TIMEOUT, "tensor-core conv gave up on a bounded wait");
  const int e = *h_err_;
  if (e == 0) return LPC_OK;
  if (e == kErrCoord) return fail(LPC_INVALID_ARG, "coordinate outside [0, 2^L)");
  if (e == kErrHashFull) return fail(LPC_HASH_FULL, "voxel hash probe limit reached");
  return fail(LPC_CORRUPT_STREAM, "decoded occupancy code is invalid");
}

// --------------------------------------------------------------- profiler --
void Codec::profile_reset(unsigned mask) {
  prof = Profile();
  prof.mask = mask;
  marks_.clear();
  pev_used_ = 0;
  if (mask && pev_.empty()) {
    pev_.resize(2048);
    for (auto& e : pev_) cudaEventCreate(&e);
  }
}

void Codec::pbeg(int f) {
  if (!(prof.mask >> f & 1) || pev_used_ + 2 > (int)pev_.size()) return;
  cudaEventRecord(pev_[pev_used_], st_);
  marks_.push_back(Mark{f, pev_used_, -1, -1, 0, 0, 0, 0});
  pev_used_ += 2;
}

void Codec::pend(int f, double bytes, double ops, int pair_slot, double ppo, double ppb) {
  if (!(prof.mask >> f & 1) || marks_.empty() || marks_.back().e1 >= 0 || marks_.back().f != f)
    return;
  Mark& m = marks_.back();
  m.e1 = m.e0 + 1;
  cudaEventRecord(pev_[m.e1], st_);
  m.bytes = bytes;
  m.ops = ops;
  m.pair_slot = pair_slot;
  m.ppo = ppo;
  m.ppb = ppb;
}

// After the frame's final synchronisation: fold the marks into the totals.
void Codec::prof_collect() {
  if (!prof.mask) return;
  uint64_t pairs[2] = {0, 0};
  cudaMemcpy(pairs, d_pairs_, sizeof(pairs), cudaMemcpyDeviceToHost);
  for (const Mark& m : marks_) {
    if (m.e1 < 0) continue;
    float ms = 0;
    cudaEventElapsedTime(&ms, pev_[m.e0], pev_[m.e1]);
    prof.ms[m.f] += ms;
    prof.launches[m.f] += 1;
    double P = m.pair_slot >= 0 ? (double)pairs[m.pair_slot] : 0.0;
    prof.bytes[m.f] += m.bytes + P * m.ppb;
    prof.ops[m.f] += m.ops + P * m.ppo;
  }
  marks_.clear();
  pev_used_ = 0;
}

void Codec::build_octree(const int32_t* d_xyz, int64_t n, int L) {
  cudaMemsetAsync(d_err_, 0, 4, st_);
  h_N_[kMaxDepth + 1] = n;
  cudaMemcpyAsync(d_N_ + kMaxDepth + 1, h_N_ + kMaxDepth + 1, 8, cudaMemcpyHostToDevice, st_);
  pbeg(kFamSort);
  launch_morton(d_xyz, n, L, d_keys0_, d_err_, st_);
  uint64_t* sorted = radix_sort(d_keys0_, n, 3 * L, sort_, st_);
  launch_unique(sorted, d_N_ + kMaxDepth + 1, n, lv_.key[L], d_N_ + L, scan_, st_);
  const int passes = (3 * L + 7) / 8;
  pend(kFamSort, 12.0 * n + 8.0 * n + 16.0 * n * passes + 16.0 * n, 0);
  pbeg(kFamLevels);
  for (int d = L - 1; d >= 0; d--)
    launch_level_up(lv_.key[d + 1], d_N_ + d + 1, lv_.cap[d + 1], lv_.key[d], lv_.code[d],
                    lv_.off[d], lv_.par[d + 1], d_N_ + d, scan_, st_);
  // level sizes are not known on the host yet: bytes are filled in by the
  // caller once they are (see level_bytes)
  pend(kFamLevels, 0, 0);
}

// Launch wrappers: one kernel each, bracketed by the profiler with the
// algorithmic work of that launch.
void Codec::embed(const DEmb& E, int d, int8_t* out, int stride, int col) {
  pbeg(kFamEmbed);
  launch_embed(E, lv_.code[d], d_N_ + d, N_[d], out, stride, col, st_);
  pend(kFamEmbed, 33.0 * N_[d], 0);
}

// Pruning(Upsampling(x)) from V_d to V_{d+1}
void Codec::up(const DLayer& W, int d, const int8_t* x, int xs, int8_t* out, int os) {
  pbeg(kFamUp);
  launch_up_prune(W, lv_.key[d + 1], lv_.par[d + 1], d_N_ + d + 1, N_[d + 1], x, xs, out, os, 0,
                  st_);
  pend(kFamUp, (double)W.cin * N_[d] + 32.0 * N_[d + 1] + 8.0 * N_[d + 1],
       2.0 * N_[d + 1] * W.cin * 32);
}

// int8 activations -> bf16 (q - z) rows, the tensor-core conv's input
void Codec::to_bf16(const int8_t* x, int xs, int cols, int z, int d) {
  pbeg(kFamEmbed);
  launch_to_bf16(x, xs, cols, z, d_N_ + d, N_[d], xb16_, st_);
  pend(kFamEmbed, 3.0 * cols * N_[d], 0);
}

// 3x3x3 conv on V_d: bf16 input rows xb (stride xbs elements); with res the
// residual merge reads y1_; outb (optional) gets the next conv's bf16 input.
void Codec::conv(const DLayer& W, int d, const int32_t* nbr, int slot, const void* xb, int xbs,
                 int8_t* out, int os, int oc, const DRes* res, void* outb, int outb_z) {
  ConvTcArgs a{};
  a.wimg = W.Wtc;
  a.bias = W.bias;
  a.mult = W.mult;
  a.slope = W.slope;
  a.prelu = W.prelu;
  a.shift = W.shift;
  a.z_out = W.z_out;
  a.nbr = nbr;
  a.d_n = d_N_ + d;
  a.xb = xb;
  a.x_stride = xbs;
  a.out = out;
  a.out_stride = os;
  a.out_col = oc;
  a.outb = outb;
  a.outb_stride = 32;
  a.outb_z = outb_z;
  if (res) {
    a.has_res = 1;
    a.y1 = y1_;
    a.y1_stride = 32;
    a.res_mab = res->mab;
    a.res_slope = res->slope;
    a.res_z1 = res->z1;
    a.res_z2 = res->z2;
    a.res_z_out = res->z_out;
    a.res_shift = res->shift;
  }
  pbeg(kFamConv);
  launch_conv333_tc(a, W.cin, N_[d], st_);
  // per neighbour pair: 2 Cin C ops and 2 Cin bytes gathered; per node: the
  // int8 output (+ the residual's y1 and the bf16 copy when present)
  pend(kFamConv,
       N_[d] * (32.0 + (res ? 32.0 : 0.0) + (outb ? 64.0 : 0.0)) + 27.0 * W.cin * 32 * 2, 0,
       slot, 2.0 * W.cin * 32, 2.0 * W.cin + 4.0);
}

void Codec::kmap(int d, int32_t* nbr, int slot) {
  pbeg(kFamHash);
  const int64_t slots = hash_slots(N_[d]);
  launch_kernel_map(lv_.key[d], d_N_ + d, N_[d], d, hash_, slots, nbr, d_err_, st_,
                    prof.mask ? d_pairs_ + slot : nullptr);
  pend(kFamHash, 12.0 * slots + 20.0 * N_[d] + 27.0 * N_[d] * (4 + 8), 0);
}

// F^b = Pruning(Upsampling(E_0[Y_{b-1}]), Y_{b-1})
void Codec::ensure_Fb() {
  if (have_Fb_) return;
  const int b = b_;
  embed(M_.E0, b - 1, xe_, 32, 0);
  up(M_.UP0, b - 1, xe_, 32, fb_, 32);
  have_Fb_ = true;
}

// S^b = ResBlock(F^b) (Eq. 8); F^t = Pruning(Upsampling(Concat(S^b, Y_b)), Y_b) (Eq. 9)
void Codec::ensure_Ft() {
  if (have_Ft_) return;
  ensure_Fb();
  const int b = b_;
  kmap(b, nbr_b_, 0);
  to_bf16(fb_, 32, 32, M_.RA[1].z_in, b);
  conv(M_.RA[1], b, nbr_b_, 0, xb16_, 32, y1_, 32, 0, nullptr, y1b16_, M_.RB[1].z_in);
  conv(M_.RB[1], b, nbr_b_, 0, y1b16_, 32, xb_, 64, 0, &M_.RM[1], nullptr, 0);
  embed(M_.E1, b, xb_, 64, 32);
  up(M_.UP1, b, xb_, 64, xt_, 64);
  have_Ft_ = true;
}

void Codec::ensure_nbr_t() {
  if (have_nbr_t_) return;
  kmap(t_, nbr_t_, 1);
  have_nbr_t_ = true;
}

// Network of level d (b <= d <= L-1): needs V_0..V_d and Y_0..Y_{d-1}.
void Codec::net_level(int d, int mode, uint16_t* cdf, uint32_t* enc, int8_t* logits) {
  auto pred = [&](int j, const int8_t* F, int stride) {
    pbeg(kFamPred);
    launch_predictor(M_.P1[j], M_.P2[j], M_.d_lut, F, stride, d_N_ + d, N_[d], mode, lv_.code[d],
                     cdf, enc, logits, st_);
    const double n = (double)N_[d];
    pend(kFamPred, n * 32 + (mode == kPredCdf ? 512.0 * n : mode == kPredEnc ? 5.0 * n : 255.0 * n),
         2.0 * n * (32 * 32 + 255 * 32));
  };
  if (d == b_) {
    ensure_Fb();
    pred(0, fb_, 32);
    return;
  }
  ensure_Ft();
  if (d == t_) {
    pred(1, xt_, 64);
    return;
  }
  // deep level d = t + m: G^t = Downsampling(Y_{d-1}) (Eq. 4)
  ensure_nbr_t();
  const int m = d - t_, j = m + 1;
  if (m == 1) {
    embed(M_.G[j], t_, xt_, 64, 32);
  } else {
    embed(M_.G[j], d - 1, g_[0], 32, 0);
    const int8_t* cur = g_[0];
    for (int i = 1; i < m; i++) {
      const int k = d - 1 - i;  // V_{k+1} -> V_k
      int8_t* dst = i == m - 1 ? xt_ : g_[i & 1];
      const int ds = i == m - 1 ? 64 : 32, dc = i == m - 1 ? 32 : 0;
      pbeg(kFamDown);
      launch_down(M_.D[j][i], lv_.key[k + 1], lv_.off[k], d_N_ + k, N_[k], cur, 32, dst, ds, dc,
                  st_);
      pend(kFamDown, 32.0 * (N_[k + 1] + N_[k]), 2.0 * N_[k + 1] * 32 * 32);
      cur = dst;
    }
  }
  // H^t = ResBlock(Concat(F^t, G^t)) (Eq. 10)
  to_bf16(xt_, 64, 64, M_.RA[j].z_in, t_);
  conv(M_.RA[j], t_, nbr_t_, 1, xb16_, 64, y1_, 32, 0, nullptr, y1b16_, M_.RB[j].z_in);
  conv(M_.RB[j], t_, nbr_t_, 1, y1b16_, 32, hx_[0], 64, 0, &M_.RM[j], nullptr, 0);
  // F^{k+1} = Pruning(Upsampling(Concat(H^k, Y_k)), Y_k), k = t..d-1 (Eq. 11)
  int cur = 0;
  for (int k = t_; k < d; k++) {
    embed(M_.E[j][k - t_], k, hx_[cur], 64, 32);
    int8_t* dst = k == d - 1 ? fo_ : hx_[1 - cur];
    const int ds = k == d - 1 ? 32 : 64;
    up(M_.UP[j][k - t_], k, hx_[cur], 64, dst, ds);
    cur = 1 - cur;
  }
  pred(j, fo_, 32);
}

// --------------------------------------------------------------- encode --
int Codec::encode(const int32_t* d_xyz, int64_t n, uint8_t* out, size_t cap, size_t* out_len) {
  err.clear();
  if (!out_len || n < 0 || (n > 0 && !d_xyz) || (cap > 0 && !out))
    return fail(LPC_INVALID_ARG, "encode_frame: bad arguments");
  if (n > cfg_.max_points) return fail(LPC_CAPACITY, "encode_frame: n exceeds max_points");
  const int L = cfg_.L;
  begin_frame(L);
  const double t0 = now_us();
  if (n > 0) {
    build_octree(d_xyz, n, L);
    cudaMemcpyAsync(h_N_, d_N_, 8 * (L + 1), cudaMemcpyDeviceToHost, st_);
    cudaMemcpyAsync(h_err_, d_err_, 4, cudaMemcpyDeviceToHost, st_);
    if (cudaStreamSynchronize(st_) != cudaSuccess) return cuda_check("encode_frame: octree");
    if (int s = check_device_error()) return s;
    stats.phase_us[0] = now_us() - t0;
    for (int d = 0; d <= L; d++) N_[d] = h_N_[d];
    level_bytes(L);
    // coarse codes to the host
    size_t coff[kMaxDepth + 1], pos = 0;
    for (int d = 0; d < b_; d++) {
      coff[d] = pos;
      cudaMemcpyAsync(h_codes_ + pos, lv_.code[d], N_[d], cudaMemcpyDeviceToHost, st_);
      pos += N_[d];
    }
    cudaEventRecord(ev_[0], st_);
    // network levels: (C_s, f_s) of the true symbol of every node; each
    // level's intervals go to the host as soon as that level is done, so the
    // host codes level d while the device computes level d + 1
    int64_t eoff[kMaxDepth + 1], ep = 0;
    for (int d = b_; d < L; d++) {
      eoff[d] = ep;
      net_level(d, kPredEnc, nullptr, d_enc_ + ep, nullptr);
      cudaMemcpyAsync(h_enc_ + ep, d_enc_ + ep, 4 * N_[d], cudaMemcpyDeviceToHost, st_);
      cudaEventRecord(ev_[1 + d - b_], st_);
      ep += N_[d];
    }
    cudaMemcpyAsync(h_err_, d_err_, 4, cudaMemcpyDeviceToHost, st_);
    cudaEventRecord(ev_[1 + L - b_], st_);
    if (int s = cuda_check("encode_frame: launch")) return s;
    // substreams: coarse levels (one each), then chunks of the network levels
    tasks_.clear();
    size_t ao = 0;
    auto add_task = [&](int d, int64_t s0, int64_t cnt) {
      tasks_.push_back(SubTask{d, s0, cnt, ao, 0});
      ao += coded_bound((size_t)cnt);
    };
    for (int d = 0; d < b_; d++) add_task(d, 0, N_[d]);
    for (int d = b_; d < L; d++)
      for (int64_t s0 = 0; s0 < N_[d]; s0 += cfg_.chunk)
        add_task(d, s0, std::min<int64_t>(cfg_.chunk, N_[d] - s0));
    if (ao > arena_cap_) return fail(LPC_CAPACITY, "encode_frame: coding arena too small");
    stats.phase_us[1] = now_us() - t0;
    // coarse levels are coded while the device runs the network
    cudaEventSynchronize(ev_[0]);
    for (int d = 0; d < b_; d++)
      for (int64_t i = 0; i < N_[d]; i++) h_codes_[coff[d] + i] -= 1;
    for (int i = b_ - 1; i >= 0; i--) {  // largest level first
      pool_->submit([this, i, &coff] {
        SubTask& T = tasks_[i];
        T.len = encode_adaptive(h_codes_ + coff[T.d], (size_t)T.count, h_arena_ + T.arena,
                                coded_bound((size_t)T.count));
      });
    }
    int level_done = b_ - 1;
    for (size_t i = b_; i < tasks_.size(); i++) {
      while (level_done < tasks_[i].d) {
        level_done++;
        cudaEventSynchronize(ev_[1 + level_done - b_]);
      }
      pool_->submit([this, i, &eoff] {
        SubTask& T = tasks_[i];
        T.len = encode_packed(h_enc_ + eoff[T.d] + T.start, (size_t)T.count, h_arena_ + T.arena,
                              coded_bound((size_t)T.count));
      });
    }
    cudaEventSynchronize(ev_[1 + L - b_]);
    pool_->wait();
    stats.phase_us[2] = now_us() - t0;
    if (int s = check_device_error()) return s;
    prof_collect();
  } else {
    tasks_.clear();
  }
  // assemble straight into the caller's buffer
  uint8_t head[kHdr + 32];
  const uint8_t hdr[10] = {'L', 'P', 'C', '1', 1, (uint8_t)L, (uint8_t)b_, (uint8_t)t_,
                           (uint8_t)M_.C, (uint8_t)(n > 0 ? 0 : 1)};
  memcpy(head, hdr, 10);
  for (int i = 0; i < 8; i++) head[10 + i] = (uint8_t)(M_.hash >> (8 * i));
  std::vector<uint8_t> table;
  put_varint(table, (uint64_t)cfg_.chunk);
  put_varint(table, tasks_.size());
  size_t body = 0;
  for (const SubTask& T : tasks_) {
    put_varint(table, T.len);
    body += T.len;
  }
  const size_t total = kHdr + table.size() + body;
  *out_len = total;
  stats.L = L;
  for (int d = 0; d <= L; d++) stats.N[d] = n > 0 ? N_[d] : 0;
  if (total > cap) return fail(LPC_CAPACITY, "encode_frame: output buffer too small");
  memcpy(out, head, kHdr);
  memcpy(out + kHdr, table.data(), table.size());
  uint8_t* p = out + kHdr + table.size();
  for (const SubTask& T : tasks_) {
    memcpy(p, h_arena_ + T.arena, T.len);
    p += T.len;
  }
  stats.host_us = now_us() - t0;
  stats.phase_us[3] = stats.host_us;
  return LPC_OK;
}

// --------------------------------------------------------------- decode --
int Codec::decode(const uint8_t* in, size_t len, int32_t* d_out, int64_t cap, int64_t* n_out) {
  err.clear();
  if (!in || !n_out) return fail(LPC_INVALID_ARG, "decode_frame: bad arguments");
  *n_out = 0;
  if (len < (size_t)kHdr || memcmp(in, "LPC1", 4) != 0 || in[4] != 1)
    return fail(LPC_CORRUPT_STREAM, "decode_frame: not an LPC1 stream");
  const int L = in[5], b = in[6], t = in[7], C = in[8], flags = in[9];
  uint64_t hash = 0;
  for (int i = 0; i < 8; i++) hash |= (uint64_t)in[10 + i] << (8 * i);
  if (L < 6 || L > kMaxDepth || b != L - 5 || t != L - 4)
    return fail(LPC_CORRUPT_STREAM, "decode_frame: bad depth fields");
  if (hash != M_.hash || C != M_.C)
    return fail(LPC_WEIGHTS_MISMATCH, "decode_frame: stream was written with another weight blob");
  if (L > cfg_.L) return fail(LPC_INVALID_ARG, "decode_frame: stream depth exceeds codec L");
  size_t pos = kHdr;
  uint64_t chunk, nsub;
  if (!get_varint(in, len, pos, chunk) || !get_varint(in, len, pos, nsub) || chunk < 1 ||
      chunk > (1u << 30) || nsub > len)
    return fail(LPC_CORRUPT_STREAM, "decode_frame: bad stream table");
  if (flags & 1) {
    if (nsub != 0) return fail(LPC_CORRUPT_STREAM, "decode_frame: empty frame with substreams");
    return LPC_OK;
  }
  std::vector<uint64_t> slen(nsub);
  std::vector<size_t> soff(nsub);
  for (uint64_t i = 0; i < nsub; i++)
    if (!get_varint(in, len, pos, slen[i]))
      return fail(LPC_CORRUPT_STREAM, "decode_frame: bad stream table");
  for (uint64_t i = 0; i < nsub; i++) {
    if (slen[i] > len - pos) return fail(LPC_CORRUPT_STREAM, "decode_frame: truncated stream");
    soff[i] = pos;
    pos += slen[i];
  }
  begin_frame(L);
  const double t0 = now_us();
  const int64_t P = cfg_.max_points;
  uint64_t si = 0;
  size_t coff[kMaxDepth + 1], cp = 0;
  // coarse levels on the host, then the device expansion up to V_b
  N_[0] = 1;
  for (int d = 0; d < b; d++) {
    if (si >= nsub) return fail(LPC_CORRUPT_STREAM, "decode_frame: missing substream");
    coff[d] = cp;
    uint8_t* Y = h_codes_ + cp;
    if (!decode_adaptive((size_t)N_[d], in + soff[si], (size_t)slen[si], Y))
      return fail(LPC_CORRUPT_STREAM, "decode_frame: corrupt coarse substream");
    si++;
    int64_t nc = 0;
    for (int64_t i = 0; i < N_[d]; i++) {
      Y[i] += 1;
      nc += __builtin_popcount(Y[i]);
    }
    cp += N_[d];
    if (nc > P) return fail(LPC_CAPACITY, "decode_frame: frame exceeds max_points");
    N_[d + 1] = nc;
  }
  stats.phase_us[4] = now_us() - t0;
  for (int i = 5; i < 9; i++) stats.phase_us[i] = 0;
  // the coarse levels are tiny: expand them on the host up to V_{b-1} and
  // upload only V_{b-1} and Y_{b-1}; the device expands V_b from there
  {
    uint64_t* keys = reinterpret_cast<uint64_t*>(h_cdf_);  // pinned staging, free here
    uint64_t* tmp = keys + P;
    keys[0] = 0;
    for (int d = 0; d + 1 < b; d++) {
      const uint8_t* Y = h_codes_ + coff[d];
      int64_t r = 0;
      for (int64_t p = 0; p < N_[d]; p++)
        for (int c = 0; c < 8; c++)
          if (Y[p] >> c & 1) tmp[r++] = (keys[p] << 3) | (uint64_t)c;
      std::swap(keys, tmp);
    }
    cudaMemsetAsync(d_err_, 0, 4, st_);
    h_N_[b - 1] = N_[b - 1];
    cudaMemcpyAsync(d_N_ + b - 1, h_N_ + b - 1, 8, cudaMemcpyHostToDevice, st_);
    cudaMemcpyAsync(lv_.key[b - 1], keys, 8 * N_[b - 1], cudaMemcpyHostToDevice, st_);
    cudaMemcpyAsync(lv_.code[b - 1], h_codes_ + coff[b - 1], N_[b - 1], cudaMemcpyHostToDevice,
                    st_);
    pbeg(kFamLevels);
    launch_expand(lv_.key[b - 1], lv_.code[b - 1], d_N_ + b - 1, lv_.cap[b - 1], lv_.key[b],
                  lv_.par[b], lv_.off[b - 1], d_N_ + b, scan_, d_err_, st_);
    pend(kFamLevels, 13.0 * N_[b - 1] + 12.0 * N_[b], 0);
  }
  // network levels: full tables to the host in chunks, decoded in parallel
  for (int d = b; d < L; d++) {
    const int64_t N = N_[d];
    double tl = now_us();
    net_level(d, kPredCdf, d_cdf_, nullptr, nullptr);
    const int64_t nch = (N + (int64_t)chunk - 1) / (int64_t)chunk;
    if ((int64_t)(si + nch) > (int64_t)nsub)
      return fail(LPC_CORRUPT_STREAM, "decode_frame: missing substream");
    if (nch > (int64_t)ev_.size()) return fail(LPC_CAPACITY, "decode_frame: chunk too small");
    for (int64_t c = 0; c < nch; c++) {
      const int64_t r0 = c * (int64_t)chunk, rows = std::min<int64_t>((int64_t)chunk, N - r0);
      cudaMemcpyAsync(h_cdf_ + r0 * 256, d_cdf_ + r0 * 256, rows * 512, cudaMemcpyDeviceToHost,
                      st_);
      cudaEventRecord(ev_[c], st_);
    }
    if (int s = cuda_check("decode_frame: launch")) return s;
    coff[d] = cp;
    uint8_t* Y = h_codes_ + cp;
    stats.phase_us[5] += now_us() - tl;
    tl = now_us();
    std::atomic<bool> bad{false};
    const uint64_t s0 = si;
    for (int64_t c = 0; c < nch; c++) {  // each chunk is decoded as soon as its table lands
      cudaEventSynchronize(ev_[c]);
      pool_->submit([&, c] {
        const int64_t r0 = c * (int64_t)chunk, rows = std::min<int64_t>((int64_t)chunk, N - r0);
        if (!decode_rows(h_cdf_ + r0 * 256, (size_t)rows, in + soff[s0 + c],
                         (size_t)slen[s0 + c], Y + r0))
          bad = true;
        for (int64_t i = 0; i < rows; i++) Y[r0 + i] += 1;
      });
    }
    pool_->wait();
    si += nch;
    stats.phase_us[6] += now_us() - tl;
    tl = now_us();
    if (bad) return fail(LPC_CORRUPT_STREAM, "decode_frame: corrupt level substream");
    int64_t nc = 0;
    for (int64_t i = 0; i < N; i++) nc += __builtin_popcount(Y[i]);
    cp += N;
    if (nc > P) return fail(LPC_CAPACITY, "decode_frame: frame exceeds max_points");
    N_[d + 1] = nc;
    cudaMemcpyAsync(lv_.code[d], Y, N, cudaMemcpyHostToDevice, st_);
    pbeg(kFamLevels);
    launch_expand(lv_.key[d], lv_.code[d], d_N_ + d, lv_.cap[d], lv_.key[d + 1], lv_.par[d + 1],
                  lv_.off[d], d_N_ + d + 1, scan_, d_err_, st_);
    pend(kFamLevels, 13.0 * N + 12.0 * nc, 0);
    stats.phase_us[7] += now_us() - tl;
  }
  if (si != nsub) return fail(LPC_CORRUPT_STREAM, "decode_frame: extra substreams");
  *n_out = N_[L];
  stats.L = L;
  for (int d = 0; d <= L; d++) stats.N[d] = N_[d];
  if (N_[L] > cap) {
    cudaStreamSynchronize(st_);
    return fail(LPC_CAPACITY, "decode_frame: output capacity too small");
  }
  launch_keys_to_xyz(lv_.key[L], d_N_ + L, N_[L], L, d_out, st_);
  cudaMemcpyAsync(h_err_, d_err_, 4, cudaMemcpyDeviceToHost, st_);
  if (cudaStreamSynchronize(st_) != cudaSuccess) return cuda_check("decode_frame");
  stats.host_us = now_us() - t0;
  stats.phase_us[8] = stats.host_us;
  prof_collect();
  return check_device_error();
}

// ---------------------------------------------------------------- probs --
int Codec::probs(const int32_t* d_xyz, int64_t n, int d, uint16_t* d_cdf, int64_t cap,
                 int64_t* nn) {
  err.clear();
  const int L = cfg_.L;
  if (!nn || n < 0 || (n > 0 && (!d_xyz || !d_cdf)) || d < L - cfg_.b_off || d > L - 1)
    return fail(LPC_INVALID_ARG, "probs_level: bad arguments");
  if (n > cfg_.max_points) return fail(LPC_CAPACITY, "probs_level: n exceeds max_points");
  *nn = 0;
  if (n == 0) return LPC_OK;
  begin_frame(L);
  build_octree(d_xyz, n, L);
  cudaMemcpyAsync(h_N_, d_N_, 8 * (L + 1), cudaMemcpyDeviceToHost, st_);
  cudaMemcpyAsync(h_err_, d_err_, 4, cudaMemcpyDeviceToHost, st_);
  if (cudaStreamSynchronize(st_) != cudaSuccess) return cuda_check("probs_level");
  if (int s = check_device_error()) return s;
  for (int k = 0; k <= L; k++) N_[k] = h_N_[k];
  level_bytes(L);
  *nn = N_[d];
  if (N_[d] > cap) return fail(LPC_CAPACITY, "probs_level: output rows too few");
  net_level(d, kPredCdf, d_cdf, nullptr, nullptr);
  cudaMemcpyAsync(h_err_, d_err_, 4, cudaMemcpyDeviceToHost, st_);
  if (cudaStreamSynchronize(st_) != cudaSuccess) return cuda_check("probs_level");
  if (int s = cuda_check("probs_level")) return s;
  prof_collect();
  return check_device_error();
}

// ---------------------------------------------------------------- batch --
int Codec::encode_batch(int nf, const int32_t* const* xyz, const int64_t* n, const int* Ls,
                        uint8_t* const* out, const size_t* caps, size_t* lens) {
  if (nf < 0 || nf > cfg_.max_frames || (nf > 0 && (!xyz || !n || !Ls || !out || !caps || !lens)))
    return fail(LPC_INVALID_ARG, "encode_batch: bad arguments");
  int first = LPC_OK;
  const int Lsave = cfg_.L;
  for (int i = 0; i < nf; i++) {
    if (Ls[i] < 6 || Ls[i] > Lsave) {
      if (!first) first = fail(LPC_INVALID_ARG, "encode_batch: frame depth out of range");
      continue;
    }
    cfg_.L = Ls[i];
    int s = encode(xyz[i], n[i], out[i], caps[i], &lens[i]);
    if (s && !first) first = s;
  }
  cfg_.L = Lsave;
  return first;
}

int Codec::decode_batch(int nf, const uint8_t* const* in, const size_t* lens, int32_t* const* out,
                        const int64_t* caps, int64_t* n_out) {
  if (nf < 0 || nf > cfg_.max_frames || (nf > 0 && (!in || !lens || !out || !caps || !n_out)))
    return fail(LPC_INVALID_ARG, "decode_batch: bad arguments");
  int first = LPC_OK;
  for (int i = 0; i < nf; i++) {
    int s = decode(in[i], lens[i], out[i], caps[i], &n_out[i]);
    if (s && !first) first = s;
  }
  return first;
}

}  // namespace lpc

// ----------------------------------------------------------------- C ABI --
struct lpc_codec {
  lpc::Codec c;
};

extern "C" {

int codec_create(const lpc_config* cfg, const void* blob, size_t blob_len, codec_t** out) {
  if (!cfg || !blob || !out) return LPC_INVALID_ARG;
  *out = nullptr;
  lpc_codec* c = new lpc_codec();
  int s = c->c.create(*cfg, blob, blob_len);
  if (s) {
    delete c;
    return s;
  }
  *out = c;
  return LPC_OK;
}

void codec_destroy(codec_t* codec) { delete codec; }

const char* codec_last_error(codec_t* codec) { return codec ? codec->c.err.c_str() : "null codec"; }

int encode_frame(codec_t* codec, const int32_t* d_xyz, int64_t n, uint8_t* h_out, size_t cap,
                 size_t* out_len) {
  if (!codec) return LPC_INVALID_ARG;
  return codec->c.encode(d_xyz, n, h_out, cap, out_len);
}

int decode_frame(codec_t* codec, const uint8_t* h_in, size_t len, int32_t* d_xyz_out, int64_t cap,
                 int64_t* n_out) {
  if (!codec) return LPC_INVALID_ARG;
  return codec->c.decode(h_in, len, d_xyz_out, cap, n_out);
}

int probs_level(codec_t* codec, const int32_t* d_xyz, int64_t n, int d, uint16_t* d_cdf_out,
                int64_t cap_nodes, int64_t* n_nodes) {
  if (!codec) return LPC_INVALID_ARG;
  return codec->c.probs(d_xyz, n, d, d_cdf_out, cap_nodes, n_nodes);
}

int encode_batch(codec_t* codec, int nf, const int32_t* const* d_xyz, const int64_t* n,
                 const int* Ls, uint8_t* const* h_out, const size_t* caps, size_t* out_lens) {
  if (!codec) return LPC_INVALID_ARG;
  return codec->c.encode_batch(nf, d_xyz, n, Ls, h_out, caps, out_lens);
}

int decode_batch(codec_t* codec, int nf, const uint8_t* const* h_in, const size_t* lens,
                 int32_t* const* d_xyz_out, const int64_t* caps, int64_t* n_out) {
  if (!codec) return LPC_INVALID_ARG;
  return codec->c.decode_batch(nf, h_in, lens, d_xyz_out, caps, n_out);
}

int codec_profile(codec_t* codec, unsigned family_mask) {
  if (!codec) return LPC_INVALID_ARG;
  codec->c.profile_reset(family_mask);
  return LPC_OK;
}

int codec_profile_read(codec_t* codec, int family, double* ms, int64_t* launches, double* bytes,
                       double* ops) {
  if (!codec || family < 0 || family >= lpc::kFamCount) return LPC_INVALID_ARG;
  const lpc::Profile& p = codec->c.prof;
  if (ms) *ms = p.ms[family];
  if (launches) *launches = p.launches[family];
  if (bytes) *bytes = p.bytes[family];
  if (ops) *ops = p.ops[family];
  return LPC_OK;
}

const char* codec_profile_name(int family) {
  static const char* names[lpc::kFamCount] = {"sort", "levels", "hash_kmap", "embed",
                                              "up_prune", "down_s2", "conv333", "predictor_cdf"};
  return family >= 0 && family < lpc::kFamCount ? names[family] : "";
}

int64_t lpc_kernel_launches(void) { return lpc::launches_total(); }

int codec_last_phases(codec_t* codec, double* us, int n) {
  if (!codec || !us) return LPC_INVALID_ARG;
  for (int i = 0; i < n && i < 16; i++) us[i] = codec->c.stats.phase_us[i];
  return LPC_OK;
}

int codec_last_stats(codec_t* codec, int64_t* counts, double* gpu_us, double* host_us) {
  if (!codec) return LPC_INVALID_ARG;
  const lpc::Stats& s = codec->c.stats;
  if (counts)
    for (int d = 0; d <= s.L; d++) counts[d] = s.N[d];
  if (gpu_us) *gpu_us = s.gpu_us;
  if (host_us) *host_us = s.host_us;
  return s.L;
}

}  // extern "C"
