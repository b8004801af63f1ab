// Codec orchestration over a batch of frames: workspace, octree build, the
// per-level network schedule of Sec. 3 (GRED + XFP, or an ablation of
// Sec. 4.3), and the range coding of the network levels (on the device, or
// on host threads from the device-made tables).  Exported through the C ABI
// of lpc.h.
//
// Every level array holds all frames of a batch at once, frame-major then
// Morton order, indexed by height above the leaves: height h is depth L_f - h
// of frame f.  The network-coded levels b..L-1 of every frame are heights
// 5..1, so relative level j = d - b is height 5 - j for every frame, whatever
// its depth L_f: one launch sequence per relative level codes every frame.
// The coarse levels (depth < b) are built on the device; their codes are
// range coded on host threads with an adaptive model, in chunks of 512
// nodes that each code and decode on their own.
#include "codec.h"

#include <string.h>

#include <algorithm>
#include <chrono>

#include "coder.h"

namespace lpc {

// ------------------------------------------------------------------ pool --
Pool::Pool(int workers) {
  for (int i = 0; i < workers; i++) th_.emplace_back([this, i] { loop(i); });
}

Pool::~Pool() {
  {
    std::lock_guard<std::mutex> g(mu_);
    stop_ = true;
    spin_.store(0, std::memory_order_relaxed);
  }
  cv_.notify_all();
  for (auto& t : th_) t.join();
}

// Runs the next queued task (lock held on entry and on return).
bool Pool::run_one(std::unique_lock<std::mutex>& lk) {
  if (head_ >= q_.size()) return false;
  const int g = q_[head_].first;
  std::function<void()> f = std::move(q_[head_].second);
  head_++;
  queued_.fetch_sub(1, std::memory_order_relaxed);
  running_++;
  lk.unlock();
  f();
  lk.lock();
  running_--;
  pending_[g]--;
  if (head_ >= q_.size() && running_ == 0) {
    q_.clear();
    head_ = 0;
  }
  done_.notify_all();
  return true;
}

static inline void cpu_relax() {
#if defined(__x86_64__) || defined(__i386__)
  __builtin_ia32_pause();
#endif
}

void Pool::loop(int idx) {
  std::unique_lock<std::mutex> lk(mu_);
  auto polls = [&] { return idx < spin_.load(std::memory_order_relaxed); };
  auto queued = [&] { return queued_.load(std::memory_order_relaxed) != 0; };
  for (;;) {
    if (stop_) return;
    if (run_one(lk)) continue;
    lk.unlock();
    if (polls()) {
      for (int k = 1; polls() && !queued(); k++) {
        cpu_relax();  // leaves the core's resources to a hyper-thread sibling
        if (k % 64 == 0) std::this_thread::yield();
      }
    } else {
      // a call just ended: keep polling a few milliseconds, since the next
      // call usually follows at once and a woken worker runs its first
      // milliseconds several times slower
      const auto until = std::chrono::steady_clock::now() + std::chrono::milliseconds(3);
      for (int k = 1; !polls() && !queued(); k++) {
        cpu_relax();
        if (k % 64 == 0) {
          std::this_thread::yield();
          if (std::chrono::steady_clock::now() > until) break;
        }
      }
    }
    lk.lock();
    if (stop_ || head_ < q_.size() || polls()) continue;
    cv_.wait(lk, [&] { return stop_ || head_ < q_.size() || polls(); });
  }
}

void Pool::set_spin(int n) {
  {
    std::lock_guard<std::mutex> g(mu_);
    spin_.store(n, std::memory_order_relaxed);
  }
  if (n > 0) cv_.notify_all();
}

void Pool::submit(int group, std::function<void()> task) {
  if (th_.empty()) {
    task();
    return;
  }
  {
    std::lock_guard<std::mutex> g(mu_);
    q_.emplace_back(group, std::move(task));
    pending_[group]++;
    queued_.fetch_add(1, std::memory_order_relaxed);
  }
  // while workers poll, they take the task; a sleeping worker is not woken
  // (its first milliseconds after waking run several times slower)
  if (spin_.load(std::memory_order_relaxed) == 0) cv_.notify_one();
}

void Pool::run_indexed(int64_t n, const std::function<void(int64_t)>& fn) {
  if (n <= 0) return;
  std::atomic<int64_t> next{0};
  auto runner = [&] {
    for (int64_t i = next.fetch_add(1); i < n; i = next.fetch_add(1)) fn(i);
  };
  const int64_t helpers = std::min<int64_t>(n - 1, (int64_t)th_.size());
  for (int64_t k = 0; k < helpers; k++) submit(kIndexedGroup, runner);
  runner();
  wait(kIndexedGroup);
}

void Pool::wait(int group) {
  std::unique_lock<std::mutex> lk(mu_);
  while (pending_[group] > 0) {
    if (!run_one(lk))
      done_.wait(lk, [&] { return pending_[group] == 0 || head_ < q_.size(); });
  }
}

// ------------------------------------------------- coarse-level decoding --
// Every coarse level is coded in chunks of kc nodes, each chunk its own
// substream with a fresh adaptive model, and the stream's header carries the
// levels' sizes: every chunk of every level decodes on its own, in parallel.
// The sizes are checked afterwards against the codes (N_d is the popcount sum
// of the codes of level d - 1).
namespace {

constexpr int kMaxCoarseTasks = 512;
constexpr size_t kCopyPart = 64 << 10;  // host copies split for the pool

struct HostCopy {
  uint8_t* dst;
  const uint8_t* src;
  size_t len;
};

void coarse_alloc(Frame& F) {
  F.coarse.assign(F.b, {});
  for (int d = 0; d < F.b; d++) F.coarse[d].resize((size_t)F.cN[d]);
}

// Chunk k of coarse level d from substream `sub`.
bool coarse_chunk(Frame& F, int d, int64_t k, size_t sub) {
  const int64_t s0 = k * F.kc, n = std::min(F.kc, F.cN[d] - s0);
  uint8_t* Y = F.coarse[d].data() + s0;
  if (!decode_adaptive((size_t)n, F.in + F.soff[sub], (size_t)F.slen[sub], Y)) return false;
  for (int64_t i = 0; i < n; i++) Y[i]++;  // symbol s codes occupancy s + 1
  return true;
}

bool coarse_consistent(const Frame& F) {
  for (int d = 1; d < F.b; d++) {
    int64_t c = 0;
    for (uint8_t y : F.coarse[d - 1]) c += __builtin_popcount(y);
    if (c != F.cN[d]) return false;
  }
  return true;
}

// All coarse levels of one frame in order on this thread.
void coarse_frame(Frame& F, std::atomic<int>& status) {
  coarse_alloc(F);
  size_t sub = 0;
  for (int d = 0; d < F.b; d++)
    for (int64_t k = 0; k * F.kc < F.cN[d]; k++)
      if (!coarse_chunk(F, d, k, sub++)) {
        status = LPC_CORRUPT_STREAM;
        return;
      }
  if (!coarse_consistent(F)) status = LPC_CORRUPT_STREAM;
}

}  // namespace

// ------------------------------------------------------------ bitstream --
// "LPC1", u8 version (3), u8 L, u8 b, u8 t, u8 C, u8 flags (bit0: empty
// frame), u64 blob hash (little endian), varint chunk, varint coarse chunk,
// varint N_1 .. N_{b-1} (not for an empty frame), varint n_sub, n_sub varints
// of the zigzag-coded difference between a substream's length and the
// previous one's (0 before the first), then the substreams: coarse levels
// 0..b-1 in chunks of `coarse chunk` nodes (adaptive model, a fresh one
// each), then every network level d = b..L-1 in chunks of `chunk` nodes.
namespace {

constexpr int kHdr = 18;
constexpr int64_t kCoarseChunk = 512;
// arena bytes of a coarse level of n nodes: every chunk's coded bound
size_t coarse_level_bound(int64_t n) {
  return 2 * (size_t)n + 8 * (size_t)((n + kCoarseChunk - 1) / kCoarseChunk);
}
constexpr int kMaxL = 19;  // 3 L Morton bits stay below the frame bits

void put_varint(std::vector<uint8_t>& o, uint64_t v) {
  while (v >= 0x80) {
    o.push_back((uint8_t)(v | 0x80));
    v >>= 7;
  }
  o.push_back((uint8_t)v);
}

constexpr uint8_t kStreamVersion = 3;

// a substream length as the zigzag varint of its difference to `prev`
void put_len(std::vector<uint8_t>& o, uint64_t len, uint64_t& prev) {
  put_varint(o, len >= prev ? (len - prev) << 1 : ((prev - len) << 1) - 1);
  prev = len;
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
  for (auto& row : gexec_)
    for (auto& e : row)
      if (e) cudaGraphExecDestroy(e);
  if (genc_) cudaGraphExecDestroy(genc_);
  for (auto s : ls_)
    if (s) cudaStreamDestroy(s);
  for (auto e : lev_)
    if (e) cudaEventDestroy(e);
  for (auto e : gev_)
    if (e) cudaEventDestroy(e);
  for (auto e : tev_)
    if (e) cudaEventDestroy(e);
  if (gs_) cudaStreamDestroy(gs_);
  if (cs_) cudaStreamDestroy(cs_);
  if (up_ev_) cudaEventDestroy(up_ev_);
  for (auto e : ev_) cudaEventDestroy(e);
  for (auto e : pev_) cudaEventDestroy(e);
  if (dmem_) cudaFree(dmem_);
  if (hmem_) cudaFreeHost(hmem_);
  for (Buf* b : {&d_rcck_, &d_rclen_, &d_rcbuf_, &d_subfr_, &d_subs_, &d_nck_, &d_cck_, &d_cchk_})
    if (b->p) cudaFree(b->p);
  for (Buf* b : {&h_rcck_, &h_rclen_, &h_rcbuf_, &h_ccodes_, &h_subfr_, &h_subs_, &h_cck_, &h_cchk_})
    if (b->p) cudaFreeHost(b->p);
  model_free(M_);
}

void* Codec::dgrow(Buf& b, size_t bytes) {
  if (bytes <= b.cap) return b.p;
  cudaStreamSynchronize(st_);
  if (b.p) cudaFree(b.p);
  b.cap = std::max<size_t>(bytes + bytes / 4, 4096);
  if (cudaMalloc(&b.p, b.cap) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    b.cap = 0;
  }
  return b.p;
}

void* Codec::hgrow(Buf& b, size_t bytes) {
  if (bytes <= b.cap) return b.p;
  cudaStreamSynchronize(st_);
  if (b.p) cudaFreeHost(b.p);
  b.cap = std::max<size_t>(bytes + bytes / 4, 4096);
  if (cudaMallocHost(&b.p, b.cap) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    b.cap = 0;
  }
  return b.p;
}

int Codec::cuda_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(LPC_CUDA_ERROR, std::string(what) + ": " + cudaGetErrorString(e));
  return LPC_OK;
}

int64_t Codec::hash_slots(int64_t n) const {
  int64_t s = 1024;
  while (s < 2 * n) s <<= 1;
  return std::min<int64_t>(s, hash_.cap);
}

int Codec::create(const lpc_config& cfg, const void* blob, size_t len) {
  cfg_ = cfg;
  if (cfg.L < 6 || cfg.L > kMaxL || cfg.C != 32 || cfg.b_off != 5 ||
      (cfg.t_off != 4 && cfg.t_off != 3) ||
      cfg.max_points < 1 || cfg.max_points > (int64_t)1 << 31 || cfg.max_frames < 1 ||
      cfg.max_frames > kMaxBatch || cfg.chunk < 1 || cfg.chunk > (1 << 24) ||
      cfg.host_coding < 0 || cfg.host_coding > 1)
    return fail(LPC_INVALID_ARG,
                "config: need 6 <= L <= 19, C = 32, b_off = 5, t_off = 4 or 3, max_points >= 1, "
                "1 <= max_frames <= 64, chunk >= 1");
  st_ = reinterpret_cast<cudaStream_t>(cfg.cuda_stream);
  dev_rc_ = cfg.host_coding == 0;
  int s = model_load(blob, len, M_, err);
  if (s) return s;
  if (M_.toff != cfg.t_off)
    return fail(LPC_INVALID_ARG, "config: t_off differs from the weight blob's threshold offset");
  F_ = cfg.max_frames;
  P_ = cfg.max_batch_points > 0 ? cfg.max_batch_points : cfg.max_points * (int64_t)cfg.max_frames;
  if (P_ > ((int64_t)1 << 31) - 2) return fail(LPC_INVALID_ARG, "config: batch capacity too large");
  const int64_t P = P_;
  const int L = cfg.L;
  // ---- device workspace (one allocation, 256-byte aligned slices) ----
  struct Slice {
    void** p;
    size_t bytes;
  };
  std::vector<Slice> sl;
  auto add = [&](void** p, size_t bytes) { sl.push_back({p, bytes}); };
  for (int h = 0; h < kHeights; h++) {
    add((void**)&key_[h], 8 * P);
    add((void**)&code_[h], P + 16);
    add((void**)&off_[h], 4 * (P + 1));
    add((void**)&par_[h], 4 * P);
  }
  add((void**)&d_N_, 8 * (kHeights + 1));
  add((void**)&d_foff_, 8 * kHeights * (F_ + 1));
  add((void**)&d_cN_, 8 * (kMaxDepth + 2));
  add((void**)&d_cfoff_, 8 * (kMaxDepth + 1) * (F_ + 1));
  add((void**)&d_fr_, sizeof(DevFrame) * F_);
  add((void**)&d_L_, 4 * F_);
  add((void**)&d_err_, 16);
  add((void**)&d_pairs_, 32);
  add((void**)&d_keys0_, 8 * P);
  sort_.n_max = P;
  add((void**)&sort_.alt, 8 * P);
  add((void**)&sort_.hist, 4 * 256 * (sort_tiles(P) + 1));
  scan_.max_tiles = scan_tiles_for(P);
  add((void**)&scan_.tiles, 4 * scan_.max_tiles);
  add((void**)&d_cup_, 4 * 32 * coarse_up_blocks(P));
  hash_.cap = 1024;
  while (hash_.cap < 2 * P) hash_.cap <<= 1;
  add((void**)&hash_.slots, 16 * hash_.cap);
  // kernel maps from height 5 (level b) down to the deepest conv level:
  // t for GRED + XFP and GRED, L - 2 (height 2) for the baseline
  for (int h = 5; h >= (M_.arch == kArchBase ? 2 : M_.toff); h--) {
    add((void**)&nbr_[h], 4 * 27 * P);
    add((void**)&tmask_[h], 4 * conv_tiles(P));
    add((void**)&ranges_[h], 8 * 148);
  }
  if (M_.arch == kArchXfp && M_.toff == 3) add((void**)&fmid_, 32 * P);
  add((void**)&gk_, 32 * P);
  if (P <= kLanePoints)
    for (int l = 1; l < kLanes; l++) {
      Scratch& S = lane_[l];
      add((void**)&S.y1, 32 * P);
      add((void**)&S.g0, 32 * P);
      add((void**)&S.g1, 32 * P);
      add((void**)&S.gk, 32 * P);
      add((void**)&S.hx0, 64 * P);
      add((void**)&S.hx1, 64 * P);
      add((void**)&S.fo, 32 * P);
      add((void**)&S.xb16, 2 * 64 * P);
      add((void**)&S.y1b16, 2 * 32 * P);
    }
  add((void**)&fb_, 32 * P);
  add((void**)&xb_, 64 * P);
  add((void**)&xt_, 64 * P);
  add((void**)&y1_, 32 * P);
  add((void**)&xe_, 32 * P);
  add((void**)&xb16_, 2 * 64 * P);
  add((void**)&y1b16_, 2 * 32 * P);
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
  // Coded substreams fit in 2 bytes per symbol plus 8 per substream
  // (coded_bound); coarse levels add at most b levels of N_{b-1} symbols.  The
  // arena is pinned so that host threads write it without page faults.  The
  // table ring holds two halves of 16 chunks each (at least 2^15 rows each).
  arena_cap_ = (size_t)2 * (L + 5) * P + (size_t)16 * (L + 5 * P / cfg.chunk + 8) * F_ + 4096;
  const int64_t half_rows = std::max<int64_t>((int64_t)16 * cfg.chunk, 1 << 15);
  ring_slots_ = (int)half_rows;
  struct HSlice {
    void** p;
    size_t bytes;
  };
  std::vector<HSlice> hs = {
      {(void**)&h_N_, 8 * (kHeights + 1)},
      {(void**)&h_foff_, 8 * (size_t)kHeights * (F_ + 1)},
      {(void**)&h_cN_, 8 * (kMaxDepth + 2)},
      {(void**)&h_cfoff_, 8 * (size_t)(kMaxDepth + 1) * (F_ + 1)},
      {(void**)&h_fr_, sizeof(DevFrame) * F_},
      {(void**)&h_L_, 4 * (size_t)F_},
      {(void**)&h_err_, 16},
      {(void**)&h_keys6_, 8 * (size_t)P},
      {(void**)&h_codes_, (size_t)kHeights * P + 64},
      {(void**)&h_enc_, 4 * 5 * (size_t)P},
      {(void**)&h_ring_, (size_t)512 * 2 * half_rows},
      {(void**)&h_arena_, arena_cap_},
  };
  size_t htotal = 0;
  for (auto& x : hs) htotal += (x.bytes + 255) / 256 * 256;
  if (cudaMallocHost(&hmem_, htotal) != cudaSuccess) {
    cudaGetLastError();
    hmem_ = nullptr;
    return fail(LPC_CUDA_ERROR, "pinned host allocation failed");
  }
  size_t ho = 0;
  for (auto& x : hs) {
    *x.p = static_cast<uint8_t*>(hmem_) + ho;
    ho += (x.bytes + 255) / 256 * 256;
  }
  if (cudaEventCreate(&tev_[0]) != cudaSuccess || cudaEventCreate(&tev_[1]) != cudaSuccess)
    return fail(LPC_CUDA_ERROR, "event creation failed");
  if (cudaStreamCreateWithFlags(&gs_, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&gev_[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&gev_[1], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    gs_ = nullptr;  // no graphs: direct launches
  }
  if (cudaStreamCreateWithFlags(&cs_, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    cs_ = nullptr;
  }
  if (cudaEventCreateWithFlags(&up_ev_, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    up_ev_ = nullptr;
  }
  lane_[0] = Scratch{y1_, g_[0], g_[1], gk_, hx_[0], hx_[1], fo_, xb16_, y1b16_};
  lanes_ = gs_ != nullptr && lane_[1].y1 != nullptr;
  for (int l = 1; l < kLanes && lanes_; l++)
    lanes_ = cudaStreamCreateWithFlags(&ls_[l], cudaStreamNonBlocking) == cudaSuccess;
  for (auto& e : lev_)
    if (lanes_) lanes_ = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
  cudaGetLastError();
  ev_.resize(512);
  for (auto& e : ev_) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  // every worker polls during a call: a single frame's host work that kept
  // to half the cores, the other workers asleep, measured slower (the
  // sleepers' wake-ups) and no steadier on the shared hosts
  const int threads = cfg.host_threads > 0
                          ? cfg.host_threads
                          : std::max(1, (int)std::thread::hardware_concurrency());
  pool_ = new Pool(std::max(0, threads - 1));
  return cuda_check("codec_create");
}

// --------------------------------------------------------------- profiler --
void Codec::profile_reset(unsigned mask) {
  prof = Profile();
  prof.mask = mask;
  marks_.clear();
  pev_used_ = 0;
  if (mask && pev_.empty()) {
    pev_.resize(4096);
    for (auto& e : pev_) cudaEventCreate(&e);
  }
}

void Codec::pbeg(int f) {
  if (!(prof.mask >> f & 1) || pev_used_ + 2 > (int)pev_.size()) return;
  cudaEventRecord(pev_[pev_used_], st_);
  marks_.push_back(Mark{f, pev_used_, -1, -1, 0, 0, 0, 0});
  pev_used_ += 2;
}

void Codec::pend(int f, double bytes, double ops, int pair_slot, double ppo, double ppb,
                 double staged, double pps) {
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
  m.staged = staged < 0 ? bytes : staged;
  m.pps = pps < 0 ? ppb : pps;
}

// After the call's final synchronisation: fold the marks into the totals.
void Codec::prof_collect() {
  if (!prof.mask) return;
  uint64_t pairs[4] = {0, 0, 0, 0};
  cudaMemcpy(pairs, d_pairs_, sizeof(pairs), cudaMemcpyDeviceToHost);
  for (const Mark& m : marks_) {
    if (m.e1 < 0) continue;
    float ms = 0;
    cudaEventElapsedTime(&ms, pev_[m.e0], pev_[m.e1]);
    prof.ms[m.f] += ms;
    prof.launches[m.f] += 1;
    const double P = m.pair_slot >= 0 ? (double)pairs[m.pair_slot] : 0.0;
    prof.bytes[m.f] += m.bytes + P * m.ppb;
    prof.ops[m.f] += m.ops + P * m.ppo;
    prof.staged[m.f] += m.staged + P * m.pps;
  }
  marks_.clear();
  pev_used_ = 0;
}

// Algorithmic bytes of the level build once the sizes are known.
void Codec::level_bytes() {
  double b = 0;
  for (int h = 0; h + 1 < kHeights; h++) b += 8.0 * N_[h] + 4.0 * N_[h] + 13.0 * N_[h + 1] + 4.0;
  for (auto it = marks_.rbegin(); it != marks_.rend(); ++it)
    if (it->f == kFamLevels) {
      it->bytes = b;
      break;
    }
}

// ------------------------------------------------------------- per batch --
void Codec::begin_batch() {
  for (int h = 0; h < kHeights; h++) have_F_[h] = have_nbr_[h] = false;
  cudaMemsetAsync(d_err_, 0, 4, st_);
  if (prof.mask) cudaMemsetAsync(d_pairs_, 0, 32, st_);
}

int Codec::check_device_error() {
  if (conv_tc_error(true)) return fail(LPC_TIMEOUT, "tensor-core conv gave up on a bounded wait");
  if (pred_tc_error(true)) return fail(LPC_TIMEOUT, "tensor-core predictor gave up on a bounded wait");
  if (up_tc_error(true)) return fail(LPC_TIMEOUT, "tensor-core up-step gave up on a bounded wait");
  const int e = *h_err_;
  if (e == 0) return LPC_OK;
  if (e == kErrCoord) return fail(LPC_INVALID_ARG, "coordinate outside [0, 2^L)");
  if (e == kErrHashFull) return fail(LPC_HASH_FULL, "voxel hash probe limit reached");
  if (e == kErrCapacity) return fail(LPC_CAPACITY, "a level exceeds the codec's capacity");
  if (e == kErrTimeout) return fail(LPC_TIMEOUT, "a device range decoder gave up on a bounded wait");
  return fail(LPC_CORRUPT_STREAM, "decoded occupancy code is invalid");
}

int Codec::sync_and_check(const char* what) {
  cudaMemcpyAsync(h_err_, d_err_, 4, cudaMemcpyDeviceToHost, st_);
  if (cudaStreamSynchronize(st_) != cudaSuccess) return cuda_check(what);
  if (int s = cuda_check(what)) return s;
  return check_device_error();
}

// Levels of the batch at heights 0..6 on the device: Morton keys (frame in
// the top bits), one radix sort, duplicate removal, then six rounds of
// floor-halving with occupancy codes (supplement, "Implementation of Octree
// Operations").  Ends with N_ and every frame's offsets on the host.
int Codec::build_levels_device(int nf, const int32_t* const* xyz, const int64_t* n,
                                bool coarse) {
  int64_t total = 0;
  int maxL = 0;
  for (int f = 0; f < nf; f++) {
    h_fr_[f] = DevFrame{xyz[f], nullptr, n[f], total, fr_[f].L, 0};
    h_L_[f] = fr_[f].L;
    total += n[f];
    maxL = std::max(maxL, fr_[f].L);
  }
  h_N_[kHeights] = total;
  cudaMemcpyAsync(d_fr_, h_fr_, sizeof(DevFrame) * nf, cudaMemcpyHostToDevice, st_);
  cudaMemcpyAsync(d_L_, h_L_, 4 * nf, cudaMemcpyHostToDevice, st_);
  cudaMemcpyAsync(d_N_ + kHeights, h_N_ + kHeights, 8, cudaMemcpyHostToDevice, st_);
  pbeg(kFamSort);
  launch_morton_batch(d_fr_, nf, total, d_keys0_, d_err_, st_);
  uint64_t* sorted = radix_sort(d_keys0_, total, 3 * maxL, nf > 1, sort_, st_);
  launch_unique(sorted, d_N_ + kHeights, total, key_[0], d_N_, scan_, st_);
  const int passes = (3 * maxL + 7) / 8 + (nf > 1 ? 1 : 0);
  pend(kFamSort, 12.0 * total + 8.0 * total + 16.0 * total * passes + 16.0 * total, 0);
  pbeg(kFamLevels);
  for (int h = 0; h + 1 < kHeights; h++)
    launch_level_up(key_[h], d_N_ + h, P_, key_[h + 1], code_[h + 1], off_[h + 1], par_[h],
                    d_N_ + h + 1, scan_, st_);
  // coarse heights (encoder): the same halving up to the deepest frame's
  // root; frames with a smaller depth carry their root up unchanged
  max_h_ = kHeights - 1;
  if (coarse) {
    launch_coarse_up(key_[kHeights - 1], d_N_ + kHeights - 1, P_, maxL, coarse_codes(kHeights), P_,
                     d_cN_, nf, d_cfoff_, d_cup_, st_);
    max_h_ = std::max(maxL, kHeights - 1);
    if (max_h_ >= kHeights) {
      cudaMemcpyAsync(h_cN_ + kHeights, d_cN_ + kHeights, 8 * (max_h_ - kHeights + 1),
                      cudaMemcpyDeviceToHost, st_);
      cudaMemcpyAsync(h_cfoff_ + (size_t)kHeights * (nf + 1), d_cfoff_ + (size_t)kHeights * (nf + 1),
                      8 * (size_t)(max_h_ - kHeights + 1) * (nf + 1), cudaMemcpyDeviceToHost, st_);
    }
  }
  pend(kFamLevels, 0, 0);
  fetch_frame_offsets(nf);
  cudaMemcpyAsync(h_N_, d_N_, 8 * kHeights, cudaMemcpyDeviceToHost, st_);
  return LPC_OK;
}

void Codec::fetch_frame_offsets(int nf) {
  LevelPtrs lp;
  for (int h = 0; h < kHeights; h++) {
    lp.key[h] = key_[h];
    lp.n[h] = d_N_ + h;
  }
  launch_frame_offsets(lp, kHeights, nf, d_foff_, st_);
  cudaMemcpyAsync(h_foff_, d_foff_, 8 * kHeights * (nf + 1), cudaMemcpyDeviceToHost, st_);
}

// --------------------------------------------------------------- network --
// Launch wrappers: one kernel each, bracketed by the profiler with the
// algorithmic work of that launch.  `h` is a height of the level arrays.

void Codec::embed(const DEmb& E, int h, int8_t* out, int stride, int col) {
  pbeg(kFamEmbed);
  launch_embed(E, code_[h], d_N_ + h, gridn(h), out, stride, col, st_);
  pend(kFamEmbed, 33.0 * N_[h], 0);
}

// Pruning(Upsampling(x)) from height h to height h - 1; with oe, the output
// rows' columns [oe_col, oe_col + 32) also get E[Y] of their codes
void Codec::up(const DLayer& W, int h, const int8_t* x, int xs, int8_t* out, int os, EmbSrc oe,
               int oe_col) {
  const int ci = W.cin == 64 ? 1 : 0;
  auto go = [&](int v) {
    if (v == 1 && W.Wtc) {
      UpTcArgs a{W.cin,  W.z_in, W.prelu, W.shift, W.z_out, W.mult_hi != nullptr, W.Wtc, W.bias,
                 W.mult_hi ? W.mult_hi : W.mult, W.slope, x,
                 xs,     d_N_ + h, off_[h], code_[h], out,  os,    0,      oe,     oe_col};
      launch_up_tc(a, gridn(h), st_);
    } else {
      launch_up_prune(W, key_[h - 1], par_[h - 1], d_N_ + h - 1, gridn(h - 1), x, xs, out, os, 0,
                      st_, oe, oe_col);
    }
  };
  if (up_variant_[ci] < 0 && !cap_grid_) {
    // autotuner, as the predictor's: both variants on this launch's input
    // (same output), warm once, best of three interleaved timed rounds
    for (int v = 0; v < kUpVariants; v++) {
      go(v);
      up_tune_ms_[ci][v] = 1e30f;
    }
    for (int rd = 0; rd < 3; rd++)
      for (int v = 0; v < kUpVariants; v++) {
        cudaEventRecord(tev_[0], st_);
        go(v);
        cudaEventRecord(tev_[1], st_);
        float ms = 1e30f;
        if (cudaEventSynchronize(tev_[1]) != cudaSuccess ||
            cudaEventElapsedTime(&ms, tev_[0], tev_[1]) != cudaSuccess) {
          cudaGetLastError();
          ms = 1e30f;
        }
        up_tune_ms_[ci][v] = std::min(up_tune_ms_[ci][v], ms);
      }
    up_variant_[ci] = 0;
    for (int v = 1; v < kUpVariants; v++)
      if (W.Wtc && up_tune_ms_[ci][v] < up_tune_ms_[ci][up_variant_[ci]]) up_variant_[ci] = v;
  }
  pbeg(kFamUp);
  go(up_variant_[ci] < 0 ? 0 : up_variant_[ci]);
  pend(kFamUp, (double)W.cin * N_[h] + 32.0 * N_[h - 1] + 8.0 * N_[h - 1],
       2.0 * N_[h - 1] * W.cin * 32);
}

// int8 activations -> bf16 (q - z) rows, the tensor-core conv's input
void Codec::to_bf16(const int8_t* x, int xs, int cols, int z, int h) {
  pbeg(kFamEmbed);
  launch_to_bf16(x, xs, cols, z, d_N_ + h, gridn(h), xb16_, st_);
  pend(kFamEmbed, 3.0 * cols * N_[h], 0);
}

// 3x3x3 conv at height h: bf16 input rows xb (stride xbs elements); with res
// the residual merge reads y1_; outb (optional) gets the next conv's input.
void Codec::conv(const DLayer& W, int h, const int32_t* nbr, int slot, const void* xb, int xbs,
                 int8_t* out, int os, int oc, const DRes* res, void* outb, int outb_z,
                 EmbSrc emb, int emb_col) {
  ConvTcArgs a{};
  a.wimg = W.Wtc;
  a.bias = W.bias;
  a.mult = W.mult;
  a.mult_hi = W.mult_hi;
  a.slope = W.slope;
  a.prelu = W.prelu;
  a.shift = W.shift;
  a.z_out = W.z_out;
  a.nbr = nbr;
  a.tmask = nbr == nbr_[h] ? tmask_[h] : nullptr;
  a.ranges = a.tmask ? ranges_[h] : nullptr;
  a.d_n = d_N_ + h;
  a.xb = xb;
  a.x_stride = xbs;
  a.out = out;
  a.out_stride = os;
  a.out_col = oc;
  a.outb = outb;
  a.outb_stride = 32;
  a.outb_z = outb_z;
  a.emb = emb;
  a.emb_col = emb_col;
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
  const int ci = W.cin == 64;
  if (conv_variant_[ci] < 0 && !cap_grid_) tune_conv(a, W.cin, h);
  pbeg(kFamConv);
  launch_conv333_tc(a, W.cin, gridn(h), st_, conv_variant_[ci] < 0 ? 0 : conv_variant_[ci]);
  // algorithmic: per present neighbour pair 2 Cin C ops and Cin int8 bytes
  // gathered; per node the int8 output (+ the residual's y1 read); the int8
  // weights once.  Staged: the bf16 rows actually gathered (2 Cin a pair),
  // the map's 27 entries a node, the bf16 copy of the output for the next
  // conv, the bf16 weight image.
  const double node_b = 32.0 + (res ? 32.0 : 0.0);
  pend(kFamConv, N_[h] * node_b + 27.0 * W.cin * 32, 0, slot, 2.0 * W.cin * 32, (double)W.cin,
       N_[h] * (node_b + 27.0 * 4 + (outb ? 64.0 : 0.0)) + 27.0 * W.cin * 32 * 2,
       2.0 * W.cin);
}

// Autotuner: every variant of the conv runs on this launch's real input (all
// give the same output, so the runs are harmless), warm once and timed once
// with events; the fastest is kept for the codec's lifetime.
void Codec::tune_conv(const ConvTcArgs& a, int cin, int h) {
  const int ci = cin == 64;
  // every variant warm once, then kTuneRounds interleaved rounds of one
  // timed launch each; a variant's time is its best round (a single timing
  // picked variants up to 15 % slower than the best)
  constexpr int kTuneRounds = 3;
  for (int v = 0; v < kConvVariants; v++) {
    launch_conv333_tc(a, cin, N_[h], st_, v);
    conv_tune_ms_[ci][v] = 1e30f;
  }
  for (int rd = 0; rd < kTuneRounds; rd++)
    for (int v = 0; v < kConvVariants; v++) {
      cudaEventRecord(tev_[0], st_);
      launch_conv333_tc(a, cin, N_[h], st_, v);
      cudaEventRecord(tev_[1], st_);
      float ms = 1e30f;
      if (cudaEventSynchronize(tev_[1]) != cudaSuccess ||
          cudaEventElapsedTime(&ms, tev_[0], tev_[1]) != cudaSuccess) {
        cudaGetLastError();
        ms = 1e30f;
      }
      conv_tune_ms_[ci][v] = std::min(conv_tune_ms_[ci][v], ms);
    }
  int bv = 0;
  for (int v = 1; v < kConvVariants; v++)
    if (conv_tune_ms_[ci][v] < conv_tune_ms_[ci][bv]) bv = v;
  conv_variant_[ci] = bv;
}

void Codec::kmap(int h, int32_t* nbr, int slot) {
  pbeg(kFamHash);
  const int64_t slots = hash_slots(gridn(h));
  launch_kernel_map(key_[h], d_N_ + h, gridn(h), d_L_, h, hash_, slots, nbr, d_err_, st_,
                    prof.mask ? d_pairs_ + slot : nullptr, tmask_[h]);
  pend(kFamHash, 12.0 * slots + 20.0 * N_[h] + 27.0 * N_[h] * (4 + 8), 0);
}

// Kernel map at height h: hashed at height 5 (level b); below it from the
// parent level's map (every node is a child of a node one level up, so its
// neighbours are children of its parent's neighbours; no second hash table).
void Codec::ensure_nbr(int h) {
  if (have_nbr_[h]) return;
  if (h == 5) {
    kmap(5, nbr_[5], 0);
    launch_conv_ranges(tmask_[5], d_N_ + 5, gridn(5), ranges_[5], st_);
  } else {
    ensure_nbr(h + 1);
    pbeg(kFamHash);
    launch_kernel_map_child(key_[h], par_[h], d_N_ + h, gridn(h), nbr_[h + 1], code_[h + 1],
                            off_[h + 1], nbr_[h], st_, prof.mask ? d_pairs_ + (5 - h) : nullptr,
                            tmask_[h]);
    launch_conv_ranges(tmask_[h], d_N_ + h, gridn(h), ranges_[h], st_);
    pend(kFamHash, 120.0 * N_[h] + 113.0 * N_[h + 1], 0);
  }
  have_nbr_[h] = true;
}

// Propagated features F^d at height h = L - d: level b from Y_{b-1} alone,
// F^b = Pruning(Upsampling(E_0[Y_{b-1}]), Y_{b-1}); with GRED + XFP, for the
// levels below b down to t, S^{d-1} = ResBlock(F^{d-1}) (Eq. 8) and
// F^d = Pruning(Upsampling(Concat(S^{d-1}, Y_{d-1})), Y_{d-1}) (Eq. 9).
// F^t lands in the first half of xt_, where the deeper levels concatenate
// G^t (Eq. 10).
const int8_t* Codec::shallow_F(int h, int* stride) {
  const bool at_t = h == M_.toff && M_.arch == kArchXfp;
  int8_t* buf = h == 5 ? fb_ : at_t ? xt_ : fmid_;
  *stride = at_t ? 64 : 32;
  if (have_F_[h]) return buf;
  if (h == 5) {
    embed(M_.ESH[0], 6, xe_, 32, 0);
    up(M_.USH[0], 6, xe_, 32, buf, *stride);
  } else {
    const int j = 5 - h, hp = h + 1;
    int ps = 32;
    const int8_t* Fp = shallow_F(hp, &ps);
    ensure_nbr(hp);
    to_bf16(Fp, ps, 32, M_.RA[j].z_in, hp);
    conv(M_.RA[j], hp, nbr_[hp], 5 - hp, xb16_, 32, y1_, 32, 0, nullptr, y1b16_, M_.RB[j].z_in);
    // Concat(S, E[Y]): the ResBlock's epilogue writes both halves
    conv(M_.RB[j], hp, nbr_[hp], 5 - hp, y1b16_, 32, xb_, 64, 0, &M_.RM[j], nullptr, 0,
         emb_src(M_.ESH[j], hp), 32);
    up(M_.USH[j], hp, xb_, 64, buf, *stride);
  }
  have_F_[h] = true;
  return buf;
}

// Network of relative level j (depth b + j of every frame, height 5 - j):
// needs the levels above it and their codes.
void Codec::set_lane(int l) {
  const Scratch& S = lane_[l];
  y1_ = S.y1;
  g_[0] = S.g0;
  g_[1] = S.g1;
  gk_ = S.gk;
  hx_[0] = S.hx0;
  hx_[1] = S.hx1;
  fo_ = S.fo;
  xb16_ = S.xb16;
  y1b16_ = S.y1b16;
}

void Codec::net_level(int j, int mode, uint16_t* cdf, uint32_t* enc, int8_t* logits, int part) {
  const int h = 5 - j;
  auto pred = [&](int jj, const int8_t* F, int stride) {
    auto go = [&](int v) {
      launch_predictor(M_.P1[jj], M_.P2[jj], M_.d_lut, F, stride, d_N_ + h, gridn(h), mode,
                       code_[h], cdf, enc, logits, st_, v);
    };
    if (pred_variant_ < 0 && !cap_grid_) {
      // autotuner: both variants on this launch's input (same output), the
      // faster kept for the codec
      // as the conv's: warm once, best of three interleaved timed rounds
      for (int v = 0; v < kPredVariants; v++) {
        go(v);
        pred_tune_ms_[v] = 1e30f;
      }
      for (int rd = 0; rd < 3; rd++)
        for (int v = 0; v < kPredVariants; v++) {
          cudaEventRecord(tev_[0], st_);
          go(v);
          cudaEventRecord(tev_[1], st_);
          float ms = 1e30f;
          if (cudaEventSynchronize(tev_[1]) != cudaSuccess ||
              cudaEventElapsedTime(&ms, tev_[0], tev_[1]) != cudaSuccess) {
            cudaGetLastError();
            ms = 1e30f;
          }
          pred_tune_ms_[v] = std::min(pred_tune_ms_[v], ms);
        }
      pred_variant_ = 0;
      for (int v = 1; v < kPredVariants; v++)
        if (pred_tune_ms_[v] < pred_tune_ms_[pred_variant_]) pred_variant_ = v;
    }
    pbeg(kFamPred);
    go(pred_variant_ < 0 ? 0 : pred_variant_);
    const double n = (double)N_[h];
    pend(kFamPred,
         n * 32 + (mode == kPredCdf ? 512.0 * n : mode == kPredEnc ? 5.0 * n : 255.0 * n),
         2.0 * n * (32 * 32 + 255 * 32));
  };
  const int m = M_.span[j];
  if (m == 0) {  // level b, and with GRED + XFP the levels down to t
    int fs = 32;
    const int8_t* F = shallow_F(h, &fs);
    pred(j, F, fs);
    return;
  }
  // features extracted at level k = d - m (height hk) from Y_{d-1}; with
  // GRED + XFP fused with the propagated F^t (k = t)
  const int hk = h + m;
  const bool cat = M_.arch == kArchXfp;
  const int w = cat ? 64 : 32;  // row width of the ResBlock's input
  if (part != kNetPost) {
    // G^k = Downsampling(Y_{d-1}) (Eq. 4): embedding at height h + 1, then
    // m - 1 stride-2 steps up to height hk, into gk_ (with m = 1 the bf16
    // conversion of the ResBlock's input reads the embedding from its table)
    if (m > 1) {
      embed(M_.G[j], h + 1, g_[0], 32, 0);
      const int8_t* cur = g_[0];
      for (int i = 1; i < m; i++) {
        const int hp = h + 1 + i;  // parent height of this step
        int8_t* dst = i == m - 1 ? gk_ : g_[i & 1];
        pbeg(kFamDown);
        launch_down(M_.D[j][i], key_[hp - 1], off_[hp], d_N_ + hp, gridn(hp), cur, 32, dst, 32, 0,
                    st_);
        pend(kFamDown, 32.0 * (N_[hp - 1] + N_[hp]), 2.0 * N_[hp - 1] * 32 * 32);
        cur = dst;
      }
    }
    if (part == kNetPre) return;
  }
  int fs = 32;
  const int8_t* Ft = cat ? shallow_F(hk, &fs) : nullptr;
  ensure_nbr(hk);
  // H^k = ResBlock(Concat(F^t, G^t)) (Eq. 10), or ResBlock(G^k) (Eq. 5)
  pbeg(kFamEmbed);
  if (m == 1)  // G^k = E[Y] at height hk itself, read from the table
    launch_to_bf16_emb(cat ? Ft : nullptr, fs, cat ? 32 : 0, emb_src(M_.G[j], hk),
                       M_.RA[j].z_in, d_N_ + hk, gridn(hk), xb16_, st_);
  else if (cat)
    launch_to_bf16_cat(Ft, fs, gk_, 32, M_.RA[j].z_in, d_N_ + hk, gridn(hk), xb16_, st_);
  else
    launch_to_bf16(gk_, 32, 32, M_.RA[j].z_in, d_N_ + hk, gridn(hk), xb16_, st_);
  pend(kFamEmbed, 3.0 * w * N_[hk], 0);
  conv(M_.RA[j], hk, nbr_[hk], 5 - hk, xb16_, w, y1_, 32, 0, nullptr, y1b16_, M_.RB[j].z_in);
  // with GRED + XFP the ResBlock's epilogue writes the first up-step's
  // Concat(H^k, E[Y]) whole, and every up-step the next one's
  conv(M_.RB[j], hk, nbr_[hk], 5 - hk, y1b16_, 32, hx_[0], w, 0, &M_.RM[j], nullptr, 0,
       cat ? emb_src(M_.E[j][0], hk) : EmbSrc{}, 32);
  // F^{k+1} = Pruning(Upsampling(Concat(H^k, Y_k)), Y_k) (Eq. 11), or
  // Pruning(Upsampling(F^k), Y_k) (Eq. 6): heights hk -> h
  int cur = 0;
  for (int k = 0; k < m; k++) {
    const int hp = hk - k;
    int8_t* dst = k == m - 1 ? fo_ : hx_[1 - cur];
    const int ds = k == m - 1 ? 32 : w;
    up(M_.UP[j][k], hp, hx_[cur], w, dst, ds,
       cat && k + 1 < m ? emb_src(M_.E[j][k + 1], hp - 1) : EmbSrc{}, 32);
    cur = 1 - cur;
  }
  pred(j, fo_, 32);
}

// A relative level's network as a CUDA graph: captured once per (mode, j)
// on the codec's private stream with grids sized for the codec's capacity
// (every kernel reads its level size on the device), then replayed after the
// work already queued on the codec's stream.  The five levels of an encode
// or a decode always run in the order j = 0..4, so each graph holds exactly
// what that level issues in that order.  Falls back to direct launches while
// profiling, or if a capture fails.
void Codec::run_level(int j, int mode, uint16_t* cdf, uint32_t* enc) {
  // direct launches while profiling, and until the conv autotuner has picked
  // its variants (it times real launches, which a capture cannot)
  // (the ablation architectures have no 64-channel conv)
  if (!gs_ || (prof.mask & ~kAsyncProfiled) || conv_variant_[0] < 0 ||
      (M_.arch == kArchXfp && conv_variant_[1] < 0) || pred_variant_ < 0 || up_variant_[0] < 0 ||
      (M_.arch == kArchXfp && up_variant_[1] < 0)) {
    net_level(j, mode, cdf, enc, nullptr);
    return;
  }
  cudaGraphExec_t& ex = gexec_[mode][j];
  if (!ex && !gfail_[mode][j]) {
    cudaStream_t saved = st_;
    st_ = gs_;
    cap_grid_ = true;
    const int64_t c0 = launches_total();
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(gs_, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      net_level(j, mode, cdf, enc, nullptr);
      ok = cudaStreamEndCapture(gs_, &g) == cudaSuccess && g;
    }
    const int64_t n = launches_total() - c0;
    count_launches((int)-n);  // captured, not run
    gkern_[mode][j] = (int)n;
    if (ok && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    st_ = saved;
    cap_grid_ = false;
    if (!ex) gfail_[mode][j] = true;
  }
  if (!ex) {
    net_level(j, mode, cdf, enc, nullptr);
    return;
  }
  cudaEventRecord(gev_[0], st_);
  cudaStreamWaitEvent(gs_, gev_[0], 0);
  cudaGraphLaunch(ex, gs_);
  cudaEventRecord(gev_[1], gs_);
  cudaStreamWaitEvent(st_, gev_[1], 0);
  count_launches(gkern_[mode][j]);
}

// The encoder's five levels with levels 3 and 4 (the longest chains) on
// lanes 1 and 2: each lane starts its level's Downsampling chain at once and
// the rest once the propagated F^t and the kernel maps it reads exist; the
// main stream computes those first, then runs levels 0..2.  Inside a capture
// the lanes fork from and join the capturing stream.
void Codec::enc_network_lanes() {
  cudaStream_t main = st_;
  const int jl[kLanes] = {-1, 4, 3};
  cudaEventRecord(lev_[0], main);
  for (int l = 1; l < kLanes; l++) {
    cudaStreamWaitEvent(ls_[l], lev_[0], 0);
    st_ = ls_[l];
    set_lane(l);
    net_level(jl[l], kPredEnc, nullptr, d_enc_ + (size_t)jl[l] * P_, nullptr, kNetPre);
  }
  st_ = main;
  set_lane(0);
  for (int l = 1; l < kLanes; l++) {  // what the lanes' levels read
    const int hk = 5 - jl[l] + M_.span[jl[l]];
    int fs = 32;
    if (M_.arch == kArchXfp) shallow_F(hk, &fs);
    ensure_nbr(hk);
  }
  cudaEventRecord(lev_[1], main);
  for (int l = 1; l < kLanes; l++) {
    st_ = ls_[l];
    set_lane(l);
    cudaStreamWaitEvent(ls_[l], lev_[1], 0);
    net_level(jl[l], kPredEnc, nullptr, d_enc_ + (size_t)jl[l] * P_, nullptr, kNetPost);
    cudaEventRecord(lev_[1 + l], ls_[l]);
  }
  st_ = main;
  set_lane(0);
  for (int j = 0; j < 3; j++) net_level(j, kPredEnc, nullptr, d_enc_ + (size_t)j * P_, nullptr);
  for (int l = 1; l < kLanes; l++) cudaStreamWaitEvent(main, lev_[1 + l], 0);
}

bool Codec::enc_graphs_ready() const {
  if (lanes_) return genc_ != nullptr;
  for (int j = 0; j < 5; j++)
    if (!gexec_[kPredEnc][j]) return false;
  return true;
}

// The encoder's network: one captured graph of the laned levels when the
// codec has lanes, else level by level.
void Codec::run_enc_network() {
  const bool direct = !gs_ || (prof.mask & ~kAsyncProfiled) || conv_variant_[0] < 0 ||
                      (M_.arch == kArchXfp && conv_variant_[1] < 0) || pred_variant_ < 0 ||
                      up_variant_[0] < 0 || (M_.arch == kArchXfp && up_variant_[1] < 0);
  if (!lanes_ || direct || genc_fail_) {
    for (int j = 0; j < 5; j++) run_level(j, kPredEnc, nullptr, d_enc_ + (size_t)j * P_);
    return;
  }
  if (!genc_) {
    cudaStream_t saved = st_;
    st_ = gs_;
    cap_grid_ = true;
    const int64_t c0 = launches_total();
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(gs_, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      enc_network_lanes();
      ok = cudaStreamEndCapture(gs_, &g) == cudaSuccess && g;
    }
    const int64_t n = launches_total() - c0;
    count_launches((int)-n);  // captured, not run
    genc_kern_ = (int)n;
    if (ok && cudaGraphInstantiate(&genc_, g, 0) != cudaSuccess) genc_ = nullptr;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    st_ = saved;
    set_lane(0);
    cap_grid_ = false;
    if (!genc_) {
      // the capture's host-side marks (features and maps "made") are void
      genc_fail_ = true;
      for (int h = 0; h < kHeights; h++) have_F_[h] = have_nbr_[h] = false;
      for (int j = 0; j < 5; j++) run_level(j, kPredEnc, nullptr, d_enc_ + (size_t)j * P_);
      return;
    }
  }
  cudaEventRecord(gev_[0], st_);
  cudaStreamWaitEvent(gs_, gev_[0], 0);
  cudaGraphLaunch(genc_, gs_);
  cudaEventRecord(gev_[1], gs_);
  cudaStreamWaitEvent(st_, gev_[1], 0);
  count_launches(genc_kern_);
}

// --------------------------------------------------------------- encode --
int Codec::encode(int nf, const int32_t* const* xyz, const int64_t* n, const int* Ls,
                  uint8_t* const* out, const size_t* caps, size_t* lens) {
  err.clear();
  if (nf < 1 || nf > F_ || !xyz || !n || !Ls || !out || !caps || !lens)
    return fail(LPC_INVALID_ARG, "encode: bad arguments");
  const double t0 = now_us();
  SpinScope spin(pool_, pool_->size() - 1);
  stats = Stats{};
  // frames with points go to the device batch, empty frames get a flag stream
  std::vector<int> dev;  // device frame index -> caller index
  int64_t total = 0;
  for (int i = 0; i < nf; i++) {
    if (Ls[i] < 6 || Ls[i] > std::min(cfg_.L, kMaxL) || n[i] < 0 || (n[i] > 0 && !xyz[i]))
      return fail(LPC_INVALID_ARG, "encode: frame depth or point count out of range");
    if (n[i] > cfg_.max_points) return fail(LPC_CAPACITY, "encode: frame exceeds max_points");
    if (n[i] > 0) dev.push_back(i);
    total += n[i];
  }
  if (total > P_) return fail(LPC_CAPACITY, "encode: batch exceeds the codec's capacity");
  const int nd = (int)dev.size();
  nf_ = nd;
  fr_.assign(nd, Frame());
  std::vector<const int32_t*> dx(nd);
  std::vector<int64_t> dn(nd);
  for (int f = 0; f < nd; f++) {
    Frame& F = fr_[f];
    F.L = Ls[dev[f]];
    F.b = F.L - cfg_.b_off;
    F.t = F.L - cfg_.t_off;
    F.n = n[dev[f]];
    dx[f] = xyz[dev[f]];
    dn[f] = n[dev[f]];
  }
  if (nd > 0) {
    begin_batch();
    build_levels_device(nd, dx.data(), dn.data(), true);
    // once every level's network is a captured graph (sizes read on the
    // device), the network is queued behind the octree before the host has
    // its sizes, and the host's copies go through the copy stream
    const bool early = gs_ && cs_ && !(prof.mask & ~kAsyncProfiled) && enc_graphs_ready();
    if (early) {
      cudaMemcpyAsync(h_err_, d_err_, 4, cudaMemcpyDeviceToHost, st_);
      cudaEventRecord(ev_[8], st_);
      run_enc_network();
      if (cudaEventSynchronize(ev_[8]) != cudaSuccess) return cuda_check("encode: octree");
      if (*h_err_ != 0) {
        cudaStreamSynchronize(st_);
        if (int s = check_device_error()) return s;
      }
    } else {
      if (int s = sync_and_check("encode: octree")) return s;
    }
    stats.phase_us[0] = now_us() - t0;
    for (int h = 0; h < kHeights; h++) N_[h] = h_N_[h];
    level_bytes();
    for (int f = 0; f < nd; f++)
      for (int h = 0; h < kHeights; h++) {
        fr_[f].off[h] = h_foff_[h * (nd + 1) + f];
        fr_[f].cnt[h] = h_foff_[h * (nd + 1) + f + 1] - fr_[f].off[h];
      }
    // codes of the coarse levels (depths 0..b-1 = heights 6..L_f) to the host
    std::vector<size_t> hoff(max_h_ + 1, 0);
    size_t ctot = 0;
    for (int h = kHeights; h <= max_h_; h++) {
      hoff[h] = ctot;
      ctot += (size_t)h_cN_[h];
    }
    uint8_t* hcc = static_cast<uint8_t*>(hgrow(h_ccodes_, ctot + 16));
    if (!hcc) return fail(LPC_CUDA_ERROR, "encode: pinned allocation failed");
    cudaStream_t cst = early ? cs_ : st_;
    if (early) cudaStreamWaitEvent(cs_, ev_[8], 0);
    cudaMemcpyAsync(h_codes_ + 6 * P_, code_[6], N_[6], cudaMemcpyDeviceToHost, cst);
    for (int h = kHeights; h <= max_h_; h++)
      cudaMemcpyAsync(hcc + hoff[h], coarse_codes(h), (size_t)h_cN_[h], cudaMemcpyDeviceToHost,
                      cst);
    cudaEventRecord(ev_[0], cst);
    // network levels of all frames: (C_s, f_s) of the true symbol of every
    // node; with host coding each level's intervals then go to the host
    if (!early) run_enc_network();
    for (int j = 0; j < 5; j++) {
      const int h = 5 - j;
      if (!dev_rc_) {
        cudaMemcpyAsync(h_enc_ + (size_t)j * P_, d_enc_ + (size_t)j * P_, 4 * N_[h],
                        cudaMemcpyDeviceToHost, st_);
        cudaEventRecord(ev_[1 + j], st_);
      }
    }
    if (int s = cuda_check("encode: launch")) return s;
    // substream layout: per frame, b coarse slots in the host arena, then the
    // network chunks (host arena, or the device coder's byte buffer)
    tasks_.clear();
    size_t ao = 0, doff = 0;
    int64_t nck = 0;
    for (int f = 0; f < nd; f++) {
      Frame& F = fr_[f];
      F.sub_base = tasks_.size();
      const size_t coarse_bound = (size_t)F.b * coarse_level_bound(F.cnt[6]);
      tasks_.push_back(SubTask{f, -1, 0, 0, ao, 0});  // whole coarse region of the frame
      ao += coarse_bound;
      for (int d = 1; d < F.b; d++) tasks_.push_back(SubTask{f, -1, 0, 0, 0, 0});
      for (int j = 0; j < 5; j++) {
        const int h = 5 - j;
        for (int64_t s0 = 0; s0 < F.cnt[h]; s0 += cfg_.chunk) {
          const int64_t cnt = std::min<int64_t>(cfg_.chunk, F.cnt[h] - s0);
          if (dev_rc_) {
            tasks_.push_back(SubTask{f, F.b + j, s0, cnt, doff, 0, nck++});
            doff += coded_bound((size_t)cnt);
          } else {
            tasks_.push_back(SubTask{f, F.b + j, s0, cnt, ao, 0});
            ao += coded_bound((size_t)cnt);
          }
        }
      }
    }
    if (ao > arena_cap_) return fail(LPC_CAPACITY, "encode: coding arena too small");
    if (dev_rc_ && nck > 0) {
      // every network chunk of every frame range coded by one launch
      RcChunk* hc = static_cast<RcChunk*>(hgrow(h_rcck_, sizeof(RcChunk) * nck));
      RcChunk* dc = static_cast<RcChunk*>(dgrow(d_rcck_, sizeof(RcChunk) * nck));
      uint32_t* hl = static_cast<uint32_t*>(hgrow(h_rclen_, 4 * nck));
      uint32_t* dl = static_cast<uint32_t*>(dgrow(d_rclen_, 4 * nck));
      uint8_t* dbuf = static_cast<uint8_t*>(dgrow(d_rcbuf_, doff));
      uint8_t* hbuf = static_cast<uint8_t*>(hgrow(h_rcbuf_, doff));
      if (!hc || !dc || !hl || !dl || !dbuf || !hbuf)
        return fail(LPC_CUDA_ERROR, "encode: range coder buffer allocation failed");
      for (const SubTask& T : tasks_) {
        if (T.rc < 0) continue;
        const Frame& F = fr_[T.f];
        const int j = T.d - F.b;
        hc[T.rc] = RcChunk{(int64_t)j * P_ + F.off[5 - j] + T.start, T.count, (int64_t)T.arena,
                           (int64_t)coded_bound((size_t)T.count)};
      }
      cudaMemcpyAsync(dc, hc, sizeof(RcChunk) * nck, cudaMemcpyHostToDevice, st_);
      pbeg(kFamCoder);
      launch_rc_encode(dc, (int)nck, d_enc_, dbuf, dl, d_err_, st_);
      // intervals read, bytes written (at most the bound; 1 byte per symbol
      // is the order of the real output)
      pend(kFamCoder, 4.0 * (double)(N_[1] + N_[2] + N_[3] + N_[4] + N_[5]) + 32.0 * nck, 0);
      cudaMemcpyAsync(hl, dl, 4 * nck, cudaMemcpyDeviceToHost, st_);
      cudaMemcpyAsync(hbuf, dbuf, doff, cudaMemcpyDeviceToHost, st_);
    }
    cudaMemcpyAsync(h_err_, d_err_, 4, cudaMemcpyDeviceToHost, st_);
    cudaEventRecord(ev_[6], st_);
    if (int s = cuda_check("encode: range coder launch")) return s;
    stats.phase_us[1] = now_us() - t0;
    // coarse levels: one host task per (frame, level), each its own adaptive
    // model, while the device runs the network.  The largest (depth b - 1 of
    // the first frame) runs on this thread: it is the critical path, and a
    // thread that was just busy runs it faster than a woken worker.
    cudaEventSynchronize(ev_[0]);
    stats.phase_us[9] = now_us() - t0;
    std::function<void()> mine;
    for (int f = 0; f < nd; f++) {
      Frame& F = fr_[f];
      size_t ao = tasks_[F.sub_base].arena;
      for (int d = 0; d < F.b; d++) {
        const int h = F.L - d;
        const uint8_t* codes;
        int64_t cnt;
        if (h == kHeights - 1) {
          codes = h_codes_ + 6 * P_ + F.off[6];
          cnt = F.cnt[6];
        } else {
          const int64_t* fo = h_cfoff_ + (size_t)h * (nd + 1);
          codes = hcc + hoff[h] + fo[f];
          cnt = fo[f + 1] - fo[f];
        }
        SubTask& T = tasks_[F.sub_base + d];
        T.arena = ao;
        T.count = cnt;
        ao += coarse_level_bound(cnt);
        stats.N[d] = f == 0 ? cnt : stats.N[d];
        auto task = [this, &T, codes, cnt] {
          T.parts.clear();
          size_t used = 0;
          for (int64_t s0 = 0; s0 < cnt; s0 += kCoarseChunk) {
            const int64_t m = std::min(kCoarseChunk, cnt - s0);
            const size_t l = encode_adaptive_codes(codes + s0, (size_t)m,
                                                   h_arena_ + T.arena + used, coded_bound((size_t)m));
            T.parts.push_back((uint32_t)l);
            used += l;
          }
          T.len = used;
        };
        if (f == 0 && d == F.b - 1) mine = task;
        else pool_->submit(0, task);
      }
    }
    for (int j = 0; j < 5 && !dev_rc_; j++) {
      cudaEventSynchronize(ev_[1 + j]);
      const int h = 5 - j;
      for (int f = 0; f < nd; f++) {
        const Frame& F = fr_[f];
        for (size_t i = F.sub_base + F.b; i < (f + 1 < nd ? fr_[f + 1].sub_base : tasks_.size());
             i++) {
          if (tasks_[i].d != F.b + j) continue;
          pool_->submit(0, [this, i, j, h] {
            SubTask& T = tasks_[i];
            const Frame& F = fr_[T.f];
            T.len = encode_packed(h_enc_ + (size_t)j * P_ + F.off[h] + T.start, (size_t)T.count,
                                  h_arena_ + T.arena, coded_bound((size_t)T.count));
          });
        }
      }
    }
    if (mine) mine();
    pool_->wait(0);
    stats.phase_us[11] = now_us() - t0;
    cudaEventSynchronize(ev_[6]);
    stats.phase_us[10] = now_us() - t0;
    if (dev_rc_)
      for (SubTask& T : tasks_)
        if (T.rc >= 0) T.len = static_cast<const uint32_t*>(h_rclen_.p)[T.rc];
    stats.phase_us[2] = now_us() - t0;
    if (int s = check_device_error()) return s;
    prof_collect();
  }
  // assemble every frame's stream straight into its caller buffer.  Batches:
  // one pool task per frame (its header, substream table and bytes), the
  // first failing frame's status reported afterwards
  int first = LPC_OK;
  if (nf > 2) {
    std::vector<int> fidx(nf), fst(nf, LPC_OK);
    for (int i = 0, f = 0; i < nf; i++) fidx[i] = n[i] == 0 ? -1 : f++;
    pool_->run_indexed(nf, [&](int64_t ii) {
      const int i = (int)ii;
      const bool empty = fidx[i] < 0;
      const Frame* F = empty ? nullptr : &fr_[fidx[i]];
      const int f = fidx[i];
      const int L = Ls[i];
      uint8_t head[kHdr];
      const uint8_t hdr[10] = {'L', 'P', 'C', '1', kStreamVersion, (uint8_t)L,
                               (uint8_t)(L - cfg_.b_off),
                               (uint8_t)(L - cfg_.t_off), (uint8_t)M_.C, (uint8_t)(empty ? 1 : 0)};
      memcpy(head, hdr, 10);
      for (int k = 0; k < 8; k++) head[10 + k] = (uint8_t)(M_.hash >> (8 * k));
      std::vector<uint8_t> table;
      put_varint(table, (uint64_t)cfg_.chunk);
      put_varint(table, (uint64_t)kCoarseChunk);
      size_t b0 = 0, b1 = 0, nsub = 0;
      if (!empty) {
        b0 = F->sub_base;
        b1 = f + 1 < nd ? fr_[f + 1].sub_base : tasks_.size();
        for (int d = 1; d < F->b; d++) put_varint(table, (uint64_t)tasks_[b0 + d].count);
        for (size_t k = b0; k < b1; k++)
          nsub += k < b0 + (size_t)F->b ? tasks_[k].parts.size() : 1;
      }
      put_varint(table, nsub);
      size_t body = 0;
      uint64_t prev = 0;
      for (size_t k = b0; k < b1; k++) {
        if (k < b0 + (size_t)F->b) {
          for (uint32_t l : tasks_[k].parts) put_len(table, l, prev);
        } else {
          put_len(table, tasks_[k].len, prev);
        }
        body += tasks_[k].len;
      }
      const size_t total_len = kHdr + table.size() + body;
      lens[i] = total_len;
      if (total_len > caps[i] || !out[i]) {
        fst[i] = LPC_CAPACITY;
        return;
      }
      memcpy(out[i], head, kHdr);
      memcpy(out[i] + kHdr, table.data(), table.size());
      uint8_t* p = out[i] + kHdr + table.size();
      for (size_t k = b0; k < b1; k++) {
        const SubTask& T = tasks_[k];
        const uint8_t* src = T.rc >= 0 ? static_cast<const uint8_t*>(h_rcbuf_.p) : h_arena_;
        memcpy(p, src + T.arena, T.len);
        p += T.len;
      }
    });
    for (int i = 0; i < nf && !first; i++)
      if (fst[i]) first = fail(fst[i], "encode: output buffer too small");
  } else {
    struct Copy {
      uint8_t* dst;
      const uint8_t* src;
      size_t len;
    };
    std::vector<Copy> copies;
    size_t copy_bytes = 0;
    for (int i = 0, f = 0; i < nf; i++) {
      const bool empty = n[i] == 0;
      const Frame* F = empty ? nullptr : &fr_[f];
      const int L = Ls[i];
      uint8_t head[kHdr];
      const uint8_t hdr[10] = {'L', 'P', 'C', '1', kStreamVersion, (uint8_t)L,
                               (uint8_t)(L - cfg_.b_off),
                               (uint8_t)(L - cfg_.t_off), (uint8_t)M_.C, (uint8_t)(empty ? 1 : 0)};
      memcpy(head, hdr, 10);
      for (int k = 0; k < 8; k++) head[10 + k] = (uint8_t)(M_.hash >> (8 * k));
      std::vector<uint8_t> table;
      put_varint(table, (uint64_t)cfg_.chunk);
      put_varint(table, (uint64_t)kCoarseChunk);
      size_t b0 = 0, b1 = 0, nsub = 0;
      if (!empty) {
        b0 = F->sub_base;
        b1 = f + 1 < nd ? fr_[f + 1].sub_base : tasks_.size();
        for (int d = 1; d < F->b; d++) put_varint(table, (uint64_t)tasks_[b0 + d].count);
        for (size_t k = b0; k < b1; k++)
          nsub += k < b0 + (size_t)F->b ? tasks_[k].parts.size() : 1;
      }
      put_varint(table, nsub);
      size_t body = 0;
      uint64_t prev = 0;
      for (size_t k = b0; k < b1; k++) {
        if (k < b0 + (size_t)F->b) {
          for (uint32_t l : tasks_[k].parts) put_len(table, l, prev);
        } else {
          put_len(table, tasks_[k].len, prev);
        }
        body += tasks_[k].len;
      }
      const size_t total_len = kHdr + table.size() + body;
      lens[i] = total_len;
      if (total_len > caps[i] || !out[i]) {
        if (!first) first = fail(LPC_CAPACITY, "encode: output buffer too small");
      } else {
        memcpy(out[i], head, kHdr);
        memcpy(out[i] + kHdr, table.data(), table.size());
        uint8_t* p = out[i] + kHdr + table.size();
        for (size_t k = b0; k < b1; k++) {
          const SubTask& T = tasks_[k];
          const uint8_t* src = T.rc >= 0 ? static_cast<const uint8_t*>(h_rcbuf_.p) : h_arena_;
          copies.push_back(Copy{p, src + T.arena, T.len});
          copy_bytes += T.len;
          p += T.len;
        }
      }
      if (!empty) f++;
    }
    {
      const int parts = (int)std::min<size_t>((size_t)pool_->size(), 1 + copy_bytes / (256 << 10));
      const size_t per = (copy_bytes + parts - 1) / parts;
      size_t k = 0;
      auto run = [&copies](size_t a, size_t b) {
        for (size_t j = a; j < b; j++) memcpy(copies[j].dst, copies[j].src, copies[j].len);
      };
      std::vector<std::pair<size_t, size_t>> ranges;
      if (parts <= 1) ranges.push_back({0, copies.size()});
      while (parts > 1 && k < copies.size()) {
        size_t b = k, acc = 0;
        while (b < copies.size() && (acc < per || b == k)) acc += copies[b++].len;
        ranges.push_back({k, b});
        k = b;
      }
      for (size_t r = 1; r < ranges.size(); r++)
        pool_->submit(0, [&run, a = ranges[r].first, b = ranges[r].second] { run(a, b); });
      if (!ranges.empty()) run(ranges[0].first, ranges[0].second);
      pool_->wait(0);
    }
  }
  // statistics of the first frame
  if (nd > 0) {
    const Frame& F = fr_[0];
    stats.L = F.L;  // coarse depths were counted when their tasks were made
    for (int h = 0; h < kHeights; h++) stats.N[F.L - h] = F.cnt[h];
  }
  stats.host_us = now_us() - t0;
  stats.phase_us[3] = stats.host_us;
  return first;
}

// --------------------------------------------------------------- decode --
int Codec::decode(int nf, const uint8_t* const* in, const size_t* lens, int32_t* const* out,
                  const int64_t* caps, int64_t* n_out) {
  err.clear();
  if (nf < 1 || nf > F_ || !in || !lens || !out || !caps || !n_out)
    return fail(LPC_INVALID_ARG, "decode: bad arguments");
  const double t0 = now_us();
  SpinScope spin(pool_, pool_->size() - 1);
  stats = Stats{};
  std::vector<int> dev;
  std::vector<Frame> all(nf);
  // every stream's header and substream table: parsed by the pool, one
  // task a stream, for batches; the first failing stream's status returned
  struct PR {
    int st;
    const char* msg;
    bool dev;  // a frame with points, to decode
  };
  auto parse = [&](int i) -> PR {
    n_out[i] = 0;
    Frame& F = all[i];
    const uint8_t* p = in[i];
    const size_t len = lens[i];
    if (!p || len < (size_t)kHdr || memcmp(p, "LPC1", 4) != 0 || p[4] != kStreamVersion)
      return PR{LPC_CORRUPT_STREAM, "decode: not an LPC1 version 3 stream", false};
    const int L = p[5], b = p[6], t = p[7], C = p[8], flags = p[9];
    uint64_t hash = 0;
    for (int k = 0; k < 8; k++) hash |= (uint64_t)p[10 + k] << (8 * k);
    if (L < 6 || L > kMaxDepth || b != L - cfg_.b_off)
      return PR{LPC_CORRUPT_STREAM, "decode: bad depth fields", false};
    if (hash != M_.hash || C != M_.C)
      return PR{LPC_WEIGHTS_MISMATCH, "decode: stream was written with another weight blob", false};
    if (t != L - cfg_.t_off) return PR{LPC_CORRUPT_STREAM, "decode: bad threshold field", false};
    if (L > std::min(cfg_.L, kMaxL))
      return PR{LPC_INVALID_ARG, "decode: stream depth exceeds the codec's L", false};
    size_t pos = kHdr;
    uint64_t chunk, kc, nsub;
    if (!get_varint(p, len, pos, chunk) || !get_varint(p, len, pos, kc) || chunk < 1 ||
        chunk > (uint64_t)ring_slots_ || kc < 1 || kc > ((uint64_t)1 << 30))
      return PR{LPC_CORRUPT_STREAM, "decode: bad stream table", false};
    F.kc = (int64_t)kc;
    F.cN[0] = 1;
    F.nco = 1;
    for (int d = 1; d < b && !(flags & 1); d++) {
      uint64_t v;
      if (!get_varint(p, len, pos, v) || v < 1 || v > 8 * (uint64_t)F.cN[d - 1])
        return PR{LPC_CORRUPT_STREAM, "decode: bad coarse level size", false};
      if (v > (uint64_t)cfg_.max_points)
        return PR{LPC_CAPACITY, "decode: frame exceeds max_points", false};
      F.cN[d] = (int64_t)v;
      F.nco += (size_t)((v + kc - 1) / kc);
    }
    if (!get_varint(p, len, pos, nsub) || nsub > len)
      return PR{LPC_CORRUPT_STREAM, "decode: bad stream table", false};
    if (flags & 1) {
      if (nsub != 0) return PR{LPC_CORRUPT_STREAM, "decode: empty frame with substreams", false};
      return PR{LPC_OK, nullptr, false};
    }
    F.L = L;
    F.b = b;
    F.t = t;
    F.in = p;
    F.len = len;
    F.chunk = (int64_t)chunk;
    F.slen.resize(nsub);
    F.soff.resize(nsub);
    uint64_t prev = 0;
    for (uint64_t k = 0; k < nsub; k++) {
      uint64_t z;
      if (!get_varint(p, len, pos, z)) return PR{LPC_CORRUPT_STREAM, "decode: bad stream table", false};
      const uint64_t mag = (z + 1) >> 1;
      if ((z & 1) ? mag > prev : mag > len)
        return PR{LPC_CORRUPT_STREAM, "decode: bad stream table", false};
      F.slen[k] = prev = (z & 1) ? prev - mag : prev + mag;
    }
    for (uint64_t k = 0; k < nsub; k++) {
      if (F.slen[k] > len - pos) return PR{LPC_CORRUPT_STREAM, "decode: truncated stream", false};
      F.soff[k] = pos;
      pos += F.slen[k];
    }
  if (nsub < F.nco) return PR{LPC_CORRUPT_STREAM, "decode: missing substream", false};
  return PR{LPC_OK, nullptr, true};
  };
  std::vector<PR> pr(nf);
  if (nf > 2)
    pool_->run_indexed(nf, [&](int64_t i) { pr[i] = parse((int)i); });
  else
    for (int i = 0; i < nf; i++) pr[i] = parse(i);
  for (int i = 0; i < nf; i++) {
    if (pr[i].st != LPC_OK) return fail(pr[i].st, pr[i].msg);
    if (pr[i].dev) dev.push_back(i);
  }
  // Decodes the frames dev (caller indices) as one batch.  coarse_ready: their
  // coarse levels were decoded by earlier pool tasks (group 3, status in
  // async_stat); after_coarse runs once the group's coarse levels are done.
  std::atomic<int> async_stat{0};
  auto run_group = [&](const std::vector<int>& dev, bool coarse_ready,
                       const std::function<void()>& after_coarse) -> int {
    const int nd = (int)dev.size();
    nf_ = nd;
    if (coarse_ready) pool_->wait(3);  // the tasks write these frames: done before they move
    fr_.clear();
    for (int i : dev) fr_.push_back(std::move(all[i]));
    if (nd == 0) return LPC_OK;
    begin_batch();
    for (int f = 0; f < nd; f++) {
      h_fr_[f] = DevFrame{nullptr, out[dev[f]], 0, 0, fr_[f].L, 0};
      h_L_[f] = fr_[f].L;
    }
    cudaMemcpyAsync(d_L_, h_L_, 4 * nd, cudaMemcpyHostToDevice, st_);
    // device coding: every frame's bytes go to the device while the host
    // decodes the coarse levels
    in_base_.assign(nd, 0);
    std::vector<HostCopy> cps;
    void* up_dst = nullptr;
    const void* up_src = nullptr;
    size_t up_len = 0;
    if (dev_rc_) {
      size_t tot = 0;
      for (int f = 0; f < nd; f++) {
        in_base_[f] = (int64_t)tot;
        tot += (fr_[f].len + 15) & ~(size_t)15;
      }
      uint8_t* hb = static_cast<uint8_t*>(hgrow(h_rcbuf_, tot));
      uint8_t* db = static_cast<uint8_t*>(dgrow(d_rcbuf_, tot));
      if (!hb || !db) return fail(LPC_CUDA_ERROR, "decode: range coder buffer allocation failed");
      // the copies into the pinned staging buffer run on the pool beside the
      // coarse decoding (parts of at most 64 KiB); the upload follows it
      for (int f = 0; f < nd; f++)
        for (size_t o = 0; o < fr_[f].len; o += kCopyPart)
          cps.push_back(HostCopy{hb + in_base_[f] + o, fr_[f].in + o,
                                 std::min(kCopyPart, fr_[f].len - o)});
      up_dst = db;
      up_src = hb;
      up_len = tot;
    }
    stats.phase_us[12] = now_us() - t0;
    if (dev_rc_) {
      // device range coding: the stream goes up first and the coarse levels
      // are decoded there too (every coarse chunk of every frame at once).
      // One frame: its bytes through the coarse substreams go up first, and
      // while the device decodes the coarse levels the pool copies the rest
      // (the network levels' substreams), which goes up on the copy stream;
      // the network levels wait for it
      const Frame& F0 = fr_[0];
      const size_t pre = nd == 1 && cs_ && up_ev_ && F0.nco > 0
                             ? (size_t)(F0.soff[F0.nco - 1] + F0.slen[F0.nco - 1])
                             : up_len;
      uint8_t* const hbuf = static_cast<uint8_t*>(const_cast<void*>(up_src));
      uint8_t* const dbuf = static_cast<uint8_t*>(up_dst);
      size_t ncp = cps.size();
      if (pre < up_len) {  // one frame, at byte 0 of both buffers
        cps.clear();
        for (size_t o = 0; o < pre; o += kCopyPart)
          cps.push_back(HostCopy{hbuf + o, F0.in + o, std::min(kCopyPart, pre - o)});
        ncp = cps.size();
        for (size_t o = pre; o < F0.len; o += kCopyPart)
          cps.push_back(HostCopy{hbuf + o, F0.in + o, std::min(kCopyPart, F0.len - o)});
      }
      pool_->run_indexed((int64_t)ncp, [&](int64_t i) {
        memcpy(cps[i].dst, cps[i].src, cps[i].len);
      });
      cudaMemcpyAsync(up_dst, up_src, std::min(pre, up_len), cudaMemcpyHostToDevice, st_);
      stats.phase_us[13] = now_us() - t0;
      if (int s = expand_coarse_device(nd, true)) return s;
      if (pre < up_len) {
        pool_->run_indexed((int64_t)(cps.size() - ncp), [&](int64_t i) {
          const HostCopy& c = cps[ncp + i];
          memcpy(c.dst, c.src, c.len);
        });
        cudaMemcpyAsync(dbuf + pre, hbuf + pre, up_len - pre, cudaMemcpyHostToDevice, cs_);
        cudaEventRecord(up_ev_, cs_);
        cudaStreamWaitEvent(st_, up_ev_, 0);
      }
      stats.phase_us[14] = stats.phase_us[4] = now_us() - t0;
      for (int i = 5; i < 9; i++) stats.phase_us[i] = 0;
      if (int s = decode_net_device(nd, n_out, dev, caps)) return s;
      stats.L = fr_[0].L;
      for (int d = 0; d < fr_[0].b; d++) stats.N[d] = fr_[0].cN[d];
      for (int h = 0; h < kHeights; h++) stats.N[fr_[0].L - h] = fr_[0].cnt[h];
      stats.host_us = now_us() - t0;
      stats.phase_us[8] = stats.host_us;
      prof_collect();
      return LPC_OK;
    }
    // coarse levels (depths 0..b-1): adaptive-model decoding on the host
    std::atomic<int> cstat{0};
    if (!coarse_ready) {
    {
      int64_t jobs = 0;
      for (int f = 0; f < nd; f++) jobs += (int64_t)fr_[f].nco;
      if (nd == 1 || jobs <= kMaxCoarseTasks) {
        // few frames: every chunk of every coarse level its own task (the
        // header gave every level's size), the largest levels first; the
        // first on this thread
        struct Job {
          int f, d;
          int64_t k;
          size_t sub;
        };
        std::vector<Job> js;
        for (int f = 0; f < nd; f++) {
          coarse_alloc(fr_[f]);
          size_t sub = 0;
          for (int d = 0; d < fr_[f].b; d++)
            for (int64_t k = 0; k * fr_[f].kc < fr_[f].cN[d]; k++) js.push_back({f, d, k, sub++});
        }
        std::stable_sort(js.begin(), js.end(), [](const Job& x, const Job& y) { return x.d > y.d; });
        auto run = [&](const Job& J) {
          if (!coarse_chunk(fr_[J.f], J.d, J.k, J.sub)) cstat = LPC_CORRUPT_STREAM;
        };
        // the coarse chunks first (the critical path), then the copies
        const int64_t nj = (int64_t)js.size();
        pool_->run_indexed(nj + (int64_t)cps.size(), [&](int64_t i) {
          if (i < nj) run(js[i]);
          else memcpy(cps[i - nj].dst, cps[i - nj].src, cps[i - nj].len);
        });
        cps.clear();
        stats.phase_us[13] = now_us() - t0;
        for (int f = 0; f < nd && !cstat; f++)
          if (!coarse_consistent(fr_[f])) cstat = LPC_CORRUPT_STREAM;
      } else {
        // many frames: one task per frame, the largest coarse streams first
        // (longest-processing-time order balances the threads), the largest on
        // this thread
        std::vector<std::pair<uint64_t, int>> order(nd);
        for (int f = 0; f < nd; f++) order[f] = {fr_[f].coarse_bytes(), f};
        std::sort(order.begin(), order.end(), [](const auto& a, const auto& b) {
          return a.first != b.first ? a.first > b.first : a.second < b.second;
        });
        auto coarse = [&](int f) { coarse_frame(fr_[f], cstat); };
        for (int k = 1; k < nd; k++) pool_->submit(0, [&, f = order[k].second] { coarse(f); });
        coarse(order[0].second);
        pool_->wait(0);
      }
    }
    if (cstat == LPC_CORRUPT_STREAM) return fail(LPC_CORRUPT_STREAM, "decode: corrupt coarse substream");
    if (cstat == LPC_CAPACITY) return fail(LPC_CAPACITY, "decode: frame exceeds max_points");
    } else {
      if (async_stat == LPC_CORRUPT_STREAM)
        return fail(LPC_CORRUPT_STREAM, "decode: corrupt coarse substream");
      if (async_stat == LPC_CAPACITY) return fail(LPC_CAPACITY, "decode: frame exceeds max_points");
    }
    if (after_coarse) after_coarse();
    pool_->run_indexed((int64_t)cps.size(), [&](int64_t i) {
      memcpy(cps[i].dst, cps[i].src, cps[i].len);
    });
    if (up_len) cudaMemcpyAsync(up_dst, up_src, up_len, cudaMemcpyHostToDevice, st_);
    stats.phase_us[14] = now_us() - t0;
    if (int s = expand_coarse_device(nd, false)) return s;
    stats.phase_us[4] = now_us() - t0;
    for (int i = 5; i < 9; i++) stats.phase_us[i] = 0;
    if (dev_rc_) {
      if (int s = decode_net_device(nd, n_out, dev, caps)) return s;
    } else {
    const int64_t maxp = cfg_.max_points;
    // substream index of (frame, relative level j, chunk 0)
    std::vector<std::vector<size_t>> sidx(nd, std::vector<size_t>(6, 0));
    std::atomic<bool> bad{false};
    for (int j = 0; j < 5; j++) {
      const int h = 5 - j;
      double tl = now_us();
      // V at height h: children of height h + 1 (host knows the counts)
      int64_t nh = 0;
      for (int f = 0; f < nd; f++) {
        Frame& F = fr_[f];
        const uint8_t* Y = h_codes_ + (size_t)(h + 1) * P_ + F.off[h + 1];
        int64_t c = 0;
        for (int64_t i = 0; i < F.cnt[h + 1]; i++) c += __builtin_popcount(Y[i]);
        if (c > maxp) return fail(LPC_CAPACITY, "decode: frame exceeds max_points");
        F.off[h] = nh;
        F.cnt[h] = c;
        nh += c;
        if (j == 0) sidx[f][0] = F.nco;
      }
      if (nh > P_) return fail(LPC_CAPACITY, "decode: batch exceeds the codec's capacity");
      N_[h] = nh;
      pbeg(kFamLevels);
      launch_expand(key_[h + 1], code_[h + 1], d_N_ + h + 1, P_, key_[h], par_[h], off_[h + 1], P_,
                    d_N_ + h, scan_, d_err_, st_);
      pend(kFamLevels, 13.0 * N_[h + 1] + 12.0 * nh, 0);
      run_level(j, kPredCdf, d_cdf_, nullptr);
      if (int s = cuda_check("decode: launch")) return s;
      stats.phase_us[7] += now_us() - tl;
      tl = now_us();
      // tables to the host through the two-half ring; chunks are decoded as
      // they land, one host task per (frame, chunk)
      struct Ck {
        int f;
        int64_t r0, rows, local;
        size_t sub;
      };
      std::vector<Ck> cks;
      for (int f = 0; f < nd; f++) {
        const Frame& F = fr_[f];
        size_t s = sidx[f][j];
        for (int64_t c0 = 0; c0 < F.cnt[h]; c0 += F.chunk, s++) {
          if (s >= F.slen.size()) return fail(LPC_CORRUPT_STREAM, "decode: missing substream");
          cks.push_back(Ck{f, F.off[h] + c0, std::min<int64_t>(F.chunk, F.cnt[h] - c0), c0, s});
        }
        sidx[f][j + 1] = s;
      }
      stats.phase_us[5] += now_us() - tl;
      tl = now_us();
      size_t c = 0;
      int wave = 0;
      while (c < cks.size()) {
        const int half = wave & 1;
        pool_->wait(1 + half);  // the tasks that last read this half are done
        uint16_t* base = h_ring_ + (size_t)half * ring_slots_ * 256;
        int64_t used = 0;
        size_t c1 = c;
        int e = 0;
        while (c1 < cks.size() && used + cks[c1].rows <= ring_slots_ && e < 240) {
          cudaMemcpyAsync(base + used * 256, d_cdf_ + cks[c1].r0 * 256, 512 * cks[c1].rows,
                          cudaMemcpyDeviceToHost, st_);
          cudaEventRecord(ev_[16 + half * 240 + e], st_);
          used += cks[c1].rows;
          c1++;
          e++;
        }
        used = 0;
        for (size_t k = c; k < c1; k++) {
          cudaEventSynchronize(ev_[16 + half * 240 + (int)(k - c)]);
          const Ck ck = cks[k];
          const uint16_t* rows = base + used * 256;
          used += ck.rows;
          pool_->submit(1 + half, [this, ck, rows, h, &bad] {
            const Frame& F = fr_[ck.f];
            uint8_t* Y = h_codes_ + (size_t)h * P_ + ck.r0;
            if (!decode_rows(rows, (size_t)ck.rows, F.in + F.soff[ck.sub], (size_t)F.slen[ck.sub],
                             Y))
              bad = true;
            for (int64_t i = 0; i < ck.rows; i++) Y[i] += 1;
          });
        }
        c = c1;
        wave++;
      }
      pool_->wait(1);
      pool_->wait(2);
      stats.phase_us[6] += now_us() - tl;
      if (bad) return fail(LPC_CORRUPT_STREAM, "decode: corrupt level substream");
      cudaMemcpyAsync(code_[h], h_codes_ + (size_t)h * P_, nh, cudaMemcpyHostToDevice, st_);
    }
    for (int f = 0; f < nd; f++)
      if (sidx[f][5] != fr_[f].slen.size())
        return fail(LPC_CORRUPT_STREAM, "decode: extra substreams");
    // leaves: children of height 1
    int64_t n0 = 0;
    for (int f = 0; f < nd; f++) {
      Frame& F = fr_[f];
      const uint8_t* Y = h_codes_ + (size_t)P_ + F.off[1];
      int64_t c = 0;
      for (int64_t i = 0; i < F.cnt[1]; i++) c += __builtin_popcount(Y[i]);
      F.off[0] = n0;
      F.cnt[0] = c;
      n0 += c;
      n_out[dev[f]] = c;
      if (c > caps[dev[f]]) return fail(LPC_CAPACITY, "decode: output capacity too small");
    }
    if (n0 > P_) return fail(LPC_CAPACITY, "decode: batch exceeds the codec's capacity");
    N_[0] = n0;
    pbeg(kFamLevels);
    launch_expand(key_[1], code_[1], d_N_ + 1, P_, key_[0], par_[0], off_[1], P_, d_N_, scan_,
                  d_err_, st_);
    pend(kFamLevels, 13.0 * N_[1] + 12.0 * n0, 0);
    for (int f = 0; f < nd; f++) h_foff_[f] = fr_[f].off[0];
    cudaMemcpyAsync(d_fr_, h_fr_, sizeof(DevFrame) * nd, cudaMemcpyHostToDevice, st_);
    cudaMemcpyAsync(d_foff_, h_foff_, 8 * nd, cudaMemcpyHostToDevice, st_);
    launch_keys_to_xyz_batch(key_[0], d_N_, n0, d_fr_, d_foff_, st_);
    if (int s = sync_and_check("decode")) return s;
    }
    stats.L = fr_[0].L;
    for (int d = 0; d < fr_[0].b; d++) stats.N[d] = (int64_t)fr_[0].coarse[d].size();
    for (int h = 0; h < kHeights; h++) stats.N[fr_[0].L - h] = fr_[0].cnt[h];
    stats.host_us = now_us() - t0;
    stats.phase_us[8] = stats.host_us;
    prof_collect();
    return LPC_OK;
  };
  return run_group(dev, false, nullptr);
}

// Coarse codes of every frame to the device, arranged by height (height h is
// depth L_f - h; above a frame's root the root is carried up with code 1),
// and expanded from the roots down to V_{b-1} (height 6) on the device.
int Codec::expand_coarse_device(int nd, bool on_device) {
  int top = kHeights - 1;
  for (int f = 0; f < nd; f++) top = std::max(top, fr_[f].L);
  // rows by height (frames in order; a frame shallower than the height
  // carries its root up as one node with code 1), from the headers' sizes
  std::vector<int64_t> hcnt(top + 1, 0), hoff(top + 1, 0), fbase((size_t)(top + 1) * nd, 0);
  size_t tot = 0;
  for (int h = top; h >= kHeights - 1; h--) {
    hoff[h] = (int64_t)tot;
    for (int f = 0; f < nd; f++) {
      const Frame& F = fr_[f];
      fbase[(size_t)h * nd + f] = hcnt[h];
      hcnt[h] += h > F.L ? 1 : F.cN[F.L - h];
    }
    tot += (size_t)hcnt[h];
    if (hcnt[h] > P_) return fail(LPC_CAPACITY, "decode: batch exceeds the codec's capacity");
  }
  for (int f = 0; f < nd; f++) {
    Frame& F = fr_[f];
    F.off[6] = fbase[(size_t)(kHeights - 1) * nd + f];
    F.cnt[6] = F.cN[F.L - (kHeights - 1)];
  }
  auto dev_codes = [&](int h) { return h == kHeights - 1 ? code_[6] : coarse_codes(h); };
  if (on_device) {
    // every coarse chunk of every frame decoded by one launch straight into
    // the arrays by height; then the level sizes checked against the codes
    int64_t nck = 0, nchk = 0;
    for (int f = 0; f < nd; f++) {
      const Frame& F = fr_[f];
      nck += (int64_t)F.nco + std::max(0, top - F.L);
      nchk += F.b - 1;
    }
    auto* hc = static_cast<CoarseChunk*>(hgrow(h_cck_, sizeof(CoarseChunk) * (size_t)nck));
    auto* dc = static_cast<CoarseChunk*>(dgrow(d_cck_, sizeof(CoarseChunk) * (size_t)nck));
    auto* hk = static_cast<CoarseCheck*>(hgrow(h_cchk_, sizeof(CoarseCheck) * (size_t)nchk + 16));
    auto* dk = static_cast<CoarseCheck*>(dgrow(d_cchk_, sizeof(CoarseCheck) * (size_t)nchk + 16));
    if (!hc || !dc || !hk || !dk) return fail(LPC_CUDA_ERROR, "decode: coarse table allocation failed");
    int64_t k = 0, q = 0;
    for (int f = 0; f < nd; f++) {
      const Frame& F = fr_[f];
      for (int h = top; h > F.L; h--)
        hc[k++] = CoarseChunk{0, 0, dev_codes(h) + fbase[(size_t)h * nd + f], 1, 1};
      size_t sub = 0;
      for (int d = 0; d < F.b; d++) {
        const int h = F.L - d;
        uint8_t* row0 = dev_codes(h) + fbase[(size_t)h * nd + f];
        for (int64_t c0 = 0; c0 < F.cN[d]; c0 += F.kc, sub++) {
          if (sub >= F.slen.size()) return fail(LPC_CORRUPT_STREAM, "decode: missing substream");
          hc[k++] = CoarseChunk{in_base_[f] + (int64_t)F.soff[sub], (int64_t)F.slen[sub], row0 + c0,
                                (int32_t)std::min<int64_t>(F.kc, F.cN[d] - c0), 0};
        }
        if (d + 1 < F.b) hk[q++] = CoarseCheck{row0, F.cN[d], F.cN[d + 1]};
      }
    }
    cudaMemcpyAsync(dc, hc, sizeof(CoarseChunk) * (size_t)k, cudaMemcpyHostToDevice, st_);
    cudaMemcpyAsync(dk, hk, sizeof(CoarseCheck) * (size_t)q, cudaMemcpyHostToDevice, st_);
    pbeg(kFamCoder);
    launch_coarse_decode(dc, (int)k, static_cast<const uint8_t*>(d_rcbuf_.p), d_err_, st_);
    pend(kFamCoder, 2.0 * (double)tot, 0);
    launch_coarse_check(dk, (int)q, d_err_, st_);
  } else {
    uint8_t* hc = static_cast<uint8_t*>(hgrow(h_ccodes_, tot + 16));
    if (!hc) return fail(LPC_CUDA_ERROR, "decode: pinned allocation failed");
    for (int h = top; h >= kHeights - 1; h--) {
      uint8_t* o = hc + hoff[h];
      for (int f = 0; f < nd; f++) {
        const Frame& F = fr_[f];
        if (h > F.L) {
          *o++ = 1;
        } else {
          const std::vector<uint8_t>& Y = F.coarse[F.L - h];
          memcpy(o, Y.data(), Y.size());
          o += Y.size();
        }
      }
    }
    // height-6 codes also on the host (the host-coding path counts from them)
    memcpy(h_codes_ + 6 * P_, hc + hoff[kHeights - 1], (size_t)hcnt[kHeights - 1]);
    for (int h = top; h >= kHeights - 1; h--)
      cudaMemcpyAsync(dev_codes(h), hc + hoff[h], (size_t)hcnt[h], cudaMemcpyHostToDevice, st_);
  }
  N_[6] = hcnt[kHeights - 1];
  h_N_[6] = N_[6];
  // roots (one per frame) at the top height, then expansions down to 6
  for (int f = 0; f < nd; f++) h_keys6_[f] = (uint64_t)f << kFrameShift;
  h_cN_[top] = nd;
  uint64_t* pp[2] = {d_keys0_, sort_.alt};
  uint64_t* top_keys = top == kHeights - 1 ? key_[6] : pp[top & 1];
  cudaMemcpyAsync(top_keys, h_keys6_, 8 * (size_t)nd, cudaMemcpyHostToDevice, st_);
  if (top == kHeights - 1)
    cudaMemcpyAsync(d_N_ + 6, h_cN_ + top, 8, cudaMemcpyHostToDevice, st_);
  for (int h = kHeights; h <= top; h++) h_cN_[h] = hcnt[h];
  cudaMemcpyAsync(d_cN_ + kHeights, h_cN_ + kHeights, 8 * (size_t)(top - kHeights + 1),
                  cudaMemcpyHostToDevice, st_);
  pbeg(kFamLevels);
  launch_coarse_down(top_keys, top, coarse_codes(kHeights), P_, hcnt.data(), d_cN_, P_, pp[0],
                     pp[1], key_[6], d_N_ + 6, scan_, d_err_, st_);
  pend(kFamLevels, 21.0 * (double)tot, 0);
  return cuda_check("decode: coarse expansion");
}

// Network levels decoded on the device: per relative level, expand the
// codes of the level above, read the new level's frame offsets back (the
// host sizes the launches and the substream table from them), run the
// network to the cumulative tables, and range-decode every chunk of every
// frame in one launch straight into the level's code array.  Ends with the
// leaves written to the callers' buffers.
int Codec::decode_net_device(int nd, int64_t* n_out, const std::vector<int>& dev,
                             const int64_t* caps) {
  // once every level's network is a captured graph (sizes read on the
  // device), the levels need no host round trip
  bool graphs = gs_ && !(prof.mask & ~kAsyncProfiled);
  for (int j = 0; j < 5 && graphs; j++) graphs = gexec_[kPredCdf][j] != nullptr;
  if (graphs) return decode_net_async(nd, n_out, dev, caps);
  const int64_t maxp = cfg_.max_points;
  std::vector<size_t> sidx(nd);
  for (int f = 0; f < nd; f++) sidx[f] = fr_[f].nco;
  const uint8_t* d_in = static_cast<const uint8_t*>(d_rcbuf_.p);
  for (int j = 0; j <= 5; j++) {  // j = 5: the leaves
    const int h = 5 - j;
    double tl = now_us();
    pbeg(kFamLevels);
    launch_expand(key_[h + 1], code_[h + 1], d_N_ + h + 1, P_, key_[h], par_[h], off_[h + 1], P_,
                  d_N_ + h, scan_, d_err_, st_);
    pend(kFamLevels, 13.0 * N_[h + 1] + 12.0 * 2.0 * N_[h + 1], 0);
    int64_t* dfo = d_foff_ + (size_t)h * (nd + 1);
    int64_t* hfo = h_foff_ + (size_t)h * (nd + 1);
    if (nd == 1) {  // one frame: its offsets are 0 and the level's size
      hfo[0] = 0;
      cudaMemsetAsync(dfo, 0, 8, st_);
      cudaMemcpyAsync(dfo + 1, d_N_ + h, 8, cudaMemcpyDeviceToDevice, st_);
      cudaMemcpyAsync(hfo + 1, d_N_ + h, 8, cudaMemcpyDeviceToHost, st_);
    } else {
      LevelPtrs lp{};
      lp.key[0] = key_[h];
      lp.n[0] = d_N_ + h;
      launch_frame_offsets(lp, 1, nd, dfo, st_);
      cudaMemcpyAsync(hfo, dfo, 8 * (nd + 1), cudaMemcpyDeviceToHost, st_);
    }
    cudaMemcpyAsync(h_err_, d_err_, 4, cudaMemcpyDeviceToHost, st_);
    stats.phase_us[7] += now_us() - tl;
    tl = now_us();
    if (cudaStreamSynchronize(st_) != cudaSuccess) return cuda_check("decode: level");
    if (int s = check_device_error()) return s;
    stats.phase_us[6] += now_us() - tl;
    tl = now_us();
    int64_t nck = 0;
    for (int f = 0; f < nd; f++) {
      Frame& F = fr_[f];
      F.off[h] = hfo[f];
      F.cnt[h] = hfo[f + 1] - hfo[f];
      if (F.cnt[h] > maxp) return fail(LPC_CAPACITY, "decode: frame exceeds max_points");
      nck += (F.cnt[h] + F.chunk - 1) / F.chunk;
    }
    N_[h] = hfo[nd];
    if (h == 0) break;
    RcChunk* hc = static_cast<RcChunk*>(hgrow(h_rcck_, sizeof(RcChunk) * (size_t)nck));
    RcChunk* dc = static_cast<RcChunk*>(dgrow(d_rcck_, sizeof(RcChunk) * (size_t)nck));
    if (!hc || !dc) return fail(LPC_CUDA_ERROR, "decode: range coder buffer allocation failed");
    int64_t k = 0;
    for (int f = 0; f < nd; f++) {
      const Frame& F = fr_[f];
      for (int64_t c0 = 0; c0 < F.cnt[h]; c0 += F.chunk, k++) {
        const size_t s = sidx[f]++;
        if (s >= F.slen.size()) return fail(LPC_CORRUPT_STREAM, "decode: missing substream");
        hc[k] = RcChunk{F.off[h] + c0, std::min<int64_t>(F.chunk, F.cnt[h] - c0),
                        in_base_[f] + (int64_t)F.soff[s], (int64_t)F.slen[s]};
      }
    }
    cudaMemcpyAsync(dc, hc, sizeof(RcChunk) * (size_t)nck, cudaMemcpyHostToDevice, st_);
    run_level(j, kPredCdf, d_cdf_, nullptr);
    pbeg(kFamCoder);
    launch_rc_decode(dc, (int)nck, d_cdf_, d_in, code_[h], d_err_, st_);
    // table rows read, codes written
    pend(kFamCoder, 513.0 * N_[h] + 32.0 * nck, 0);
    if (int s = cuda_check("decode: launch")) return s;
    stats.phase_us[5] += now_us() - tl;
  }
  for (int f = 0; f < nd; f++)
    if (sidx[f] != fr_[f].slen.size()) return fail(LPC_CORRUPT_STREAM, "decode: extra substreams");
  for (int f = 0; f < nd; f++) {
    const int64_t c = fr_[f].cnt[0];
    n_out[dev[f]] = c;
    if (c > caps[dev[f]]) return fail(LPC_CAPACITY, "decode: output capacity too small");
  }
  cudaMemcpyAsync(d_fr_, h_fr_, sizeof(DevFrame) * nd, cudaMemcpyHostToDevice, st_);
  launch_keys_to_xyz_batch(key_[0], d_N_, N_[0], d_fr_, d_foff_, st_);
  return sync_and_check("decode");
}

// The network levels without host round trips: each level's sizes, frame
// offsets and substream table stay on the device (the table from every
// frame's substream list, uploaded once), the range decoder's grid is the
// table's capacity; the host reads the sizes back once, at the end.
int Codec::decode_net_async(int nd, int64_t* n_out, const std::vector<int>& dev,
                            const int64_t* caps) {
  const int64_t maxp = cfg_.max_points;
  int64_t nsub = 0, min_chunk = INT64_MAX;
  for (int f = 0; f < nd; f++) {
    nsub += (int64_t)fr_[f].slen.size();
    min_chunk = std::min(min_chunk, fr_[f].chunk);
  }
  const int64_t cap_ck = P_ / min_chunk + nd;
  auto* hsf = static_cast<DevSubFrame*>(hgrow(h_subfr_, sizeof(DevSubFrame) * nd));
  auto* dsf = static_cast<DevSubFrame*>(dgrow(d_subfr_, sizeof(DevSubFrame) * nd));
  auto* hsub = static_cast<int64_t*>(hgrow(h_subs_, 16 * (size_t)nsub + 16));
  auto* dsub = static_cast<int64_t*>(dgrow(d_subs_, 16 * (size_t)nsub + 16));
  auto* dnck = static_cast<int64_t*>(dgrow(d_nck_, 8));
  auto* dc = static_cast<RcChunk*>(dgrow(d_rcck_, sizeof(RcChunk) * (size_t)cap_ck));
  if (!hsf || !dsf || !hsub || !dsub || !dnck || !dc)
    return fail(LPC_CUDA_ERROR, "decode: substream table allocation failed");
  int64_t k = 0;
  for (int f = 0; f < nd; f++) {
    const Frame& F = fr_[f];
    hsf[f] = DevSubFrame{k, (int64_t)F.slen.size(), F.chunk, in_base_[f], (int64_t)F.nco};
    for (size_t s = 0; s < F.slen.size(); s++, k++) {
      hsub[2 * k] = (int64_t)F.soff[s];
      hsub[2 * k + 1] = (int64_t)F.slen[s];
    }
  }
  cudaMemcpyAsync(dsf, hsf, sizeof(DevSubFrame) * nd, cudaMemcpyHostToDevice, st_);
  cudaMemcpyAsync(dsub, hsub, 16 * (size_t)nsub, cudaMemcpyHostToDevice, st_);
  const uint8_t* d_in = static_cast<const uint8_t*>(d_rcbuf_.p);
  int coder_marks[kHeights];  // profiler mark of each height's decode launch
  for (int h = 0; h < kHeights; h++) coder_marks[h] = -1;
  for (int j = 0; j <= 5; j++) {  // j = 5: the leaves
    const int h = 5 - j;
    launch_expand(key_[h + 1], code_[h + 1], d_N_ + h + 1, P_, key_[h], par_[h], off_[h + 1], P_,
                  d_N_ + h, scan_, d_err_, st_);
    int64_t* dfo = d_foff_ + (size_t)h * (nd + 1);
    if (nd == 1) {
      cudaMemsetAsync(dfo, 0, 8, st_);
      cudaMemcpyAsync(dfo + 1, d_N_ + h, 8, cudaMemcpyDeviceToDevice, st_);
    } else {
      LevelPtrs lp{};
      lp.key[0] = key_[h];
      lp.n[0] = d_N_ + h;
      launch_frame_offsets(lp, 1, nd, dfo, st_);
    }
    if (h == 0) break;
    launch_rc_chunks(dfo, nd, dsf, dsub, dc, cap_ck, maxp, dnck, d_err_, st_);
    run_level(j, kPredCdf, d_cdf_, nullptr);
    pbeg(kFamCoder);
    launch_rc_decode_dev(dc, dnck, cap_ck, d_cdf_, d_in, code_[h], d_err_, st_);
    pend(kFamCoder, 0, 0);  // bytes once the level sizes are on the host
    if (!marks_.empty() && marks_.back().f == kFamCoder && marks_.back().e1 >= 0)
      coder_marks[h] = (int)marks_.size() - 1;
    if (int s = cuda_check("decode: launch")) return s;
  }
  cudaMemcpyAsync(h_foff_, d_foff_, 8 * (size_t)kHeights * (nd + 1), cudaMemcpyDeviceToHost, st_);
  cudaMemcpyAsync(hsf, dsf, sizeof(DevSubFrame) * nd, cudaMemcpyDeviceToHost, st_);
  if (int s = sync_and_check("decode: levels")) return s;
  for (int f = 0; f < nd; f++) {
    Frame& F = fr_[f];
    if (hsf[f].next != hsf[f].nsub) return fail(LPC_CORRUPT_STREAM, "decode: extra substreams");
    for (int h = 0; h < 6; h++) {
      const int64_t* hfo = h_foff_ + (size_t)h * (nd + 1);
      F.off[h] = hfo[f];
      F.cnt[h] = hfo[f + 1] - hfo[f];
    }
    n_out[dev[f]] = F.cnt[0];
    if (F.cnt[0] > caps[dev[f]]) return fail(LPC_CAPACITY, "decode: output capacity too small");
  }
  for (int h = 0; h < 6; h++) N_[h] = h_foff_[(size_t)h * (nd + 1) + nd];
  for (int h = 1; h < 6; h++)
    if (coder_marks[h] >= 0) {  // table rows read, codes written
      double nck = 0;
      for (int f = 0; f < nd; f++)
        nck += (double)((fr_[f].cnt[h] + fr_[f].chunk - 1) / fr_[f].chunk);
      marks_[(size_t)coder_marks[h]].bytes = 513.0 * N_[h] + 32.0 * nck;
    }
  cudaMemcpyAsync(d_fr_, h_fr_, sizeof(DevFrame) * nd, cudaMemcpyHostToDevice, st_);
  launch_keys_to_xyz_batch(key_[0], d_N_, N_[0], d_fr_, d_foff_, st_);
  return sync_and_check("decode");
}

// ---------------------------------------------------------------- probs --
int Codec::probs(const int32_t* d_xyz, int64_t n, int d, uint16_t* d_cdf, int64_t cap,
                 int64_t* nn) {
  err.clear();
  const int L = cfg_.L;
  if (!nn || n < 0 || (n > 0 && (!d_xyz || !d_cdf)) || d < L - cfg_.b_off || d > L - 1)
    return fail(LPC_INVALID_ARG, "probs_level: bad arguments");
  if (reinterpret_cast<uintptr_t>(d_cdf) & 15)  // rows leave by 16-byte-aligned copies
    return fail(LPC_INVALID_ARG, "probs_level: d_cdf_out must be 16-byte aligned");
  if (n > cfg_.max_points || n > P_) return fail(LPC_CAPACITY, "probs_level: n exceeds max_points");
  *nn = 0;
  if (n == 0) return LPC_OK;
  nf_ = 1;
  fr_.assign(1, Frame());
  fr_[0].L = L;
  fr_[0].b = L - cfg_.b_off;
  fr_[0].t = L - cfg_.t_off;
  fr_[0].n = n;
  begin_batch();
  const int32_t* x = d_xyz;
  build_levels_device(1, &x, &n, false);
  if (int s = sync_and_check("probs_level")) return s;
  for (int h = 0; h < kHeights; h++) N_[h] = h_N_[h];
  level_bytes();
  const int j = d - fr_[0].b;
  *nn = N_[5 - j];
  if (N_[5 - j] > cap) return fail(LPC_CAPACITY, "probs_level: output rows too few");
  net_level(j, kPredCdf, d_cdf, nullptr, nullptr);
  if (int s = sync_and_check("probs_level")) return s;
  prof_collect();
  return LPC_OK;
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
  if (!codec || !out_len) return LPC_INVALID_ARG;
  int Ls = codec->c.depth();
  return codec->c.encode(1, &d_xyz, &n, &Ls, &h_out, &cap, out_len);
}

int decode_frame(codec_t* codec, const uint8_t* h_in, size_t len, int32_t* d_xyz_out, int64_t cap,
                 int64_t* n_out) {
  if (!codec || !n_out) return LPC_INVALID_ARG;
  return codec->c.decode(1, &h_in, &len, &d_xyz_out, &cap, n_out);
}

int probs_level(codec_t* codec, const int32_t* d_xyz, int64_t n, int d, uint16_t* d_cdf_out,
                int64_t cap_nodes, int64_t* n_nodes) {
  if (!codec) return LPC_INVALID_ARG;
  return codec->c.probs(d_xyz, n, d, d_cdf_out, cap_nodes, n_nodes);
}

int encode_batch(codec_t* codec, int nf, const int32_t* const* d_xyz, const int64_t* n,
                 const int* Ls, uint8_t* const* h_out, const size_t* caps, size_t* out_lens) {
  if (!codec) return LPC_INVALID_ARG;
  return codec->c.encode(nf, d_xyz, n, Ls, h_out, caps, out_lens);
}

int decode_batch(codec_t* codec, int nf, const uint8_t* const* h_in, const size_t* lens,
                 int32_t* const* d_xyz_out, const int64_t* caps, int64_t* n_out) {
  if (!codec) return LPC_INVALID_ARG;
  return codec->c.decode(nf, h_in, lens, d_xyz_out, caps, n_out);
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

int codec_profile_staged(codec_t* codec, int family, double* bytes) {
  if (!codec || !bytes || family < 0 || family >= lpc::kFamCount) return LPC_INVALID_ARG;
  *bytes = codec->c.prof.staged[family];
  return LPC_OK;
}

const char* codec_profile_name(int family) {
  static const char* names[lpc::kFamCount] = {"sort", "levels", "hash_kmap", "embed",
                                              "up_prune", "down_s2", "conv333", "predictor_cdf",
                                              "range_coder"};
  return family >= 0 && family < lpc::kFamCount ? names[family] : "";
}

int64_t lpc_kernel_launches(void) { return lpc::launches_total(); }

int codec_set_tuning(codec_t* codec, const int* variants) {
  if (!codec || !variants) return LPC_INVALID_ARG;
  for (int c = 0; c < 2; c++)
    if (variants[c] < -1 || variants[c] >= lpc::kConvVariants) return LPC_INVALID_ARG;
  if (variants[2] < -1 || variants[2] >= lpc::kPredVariants) return LPC_INVALID_ARG;
  for (int c = 3; c < 5; c++)
    if (variants[c] < -1 || variants[c] >= lpc::kUpVariants) return LPC_INVALID_ARG;
  codec->c.set_tuning(variants);
  return LPC_OK;
}

int codec_tuning(codec_t* codec, int* variants, float* ms) {
  if (!codec) return LPC_INVALID_ARG;
  for (int c = 0; c < 2; c++) {
    if (variants) variants[c] = codec->c.conv_variant_[c];
    for (int v = 0; v < lpc::kConvVariants && ms; v++) ms[c * lpc::kConvVariants + v] =
        codec->c.conv_tune_ms_[c][v];
  }
  if (variants) variants[2] = codec->c.pred_variant_;
  for (int v = 0; v < lpc::kPredVariants && ms; v++)
    ms[2 * lpc::kConvVariants + v] = codec->c.pred_tune_ms_[v];
  for (int c = 0; c < 2; c++) {
    if (variants) variants[3 + c] = codec->c.up_variant_[c];
    for (int v = 0; v < lpc::kUpVariants && ms; v++)
      ms[2 * lpc::kConvVariants + lpc::kPredVariants + c * lpc::kUpVariants + v] =
          codec->c.up_tune_ms_[c][v];
  }
  return LPC_OK;
}

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
