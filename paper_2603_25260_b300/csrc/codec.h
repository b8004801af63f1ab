// The codec object: workspace, the per-level network schedule over a batch of
// frames, and host range coding.  A single frame is a batch of one.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lpc.h"
#include "common.cuh"
#include "kernels.h"
#include "model.h"

namespace lpc {

// Host task queue: the calling thread submits tasks as their inputs become
// ready (it alone waits on CUDA events), workers run them; wait(group) helps
// run queued tasks and returns when every task of the group has finished.
class Pool {
 public:
  explicit Pool(int workers);
  ~Pool();
  void submit(int group, std::function<void()> task);
  void wait(int group);
  // fn(0) .. fn(n - 1) on the workers and the calling thread, each index
  // once, claimed in order from a shared counter (no lock per index); returns
  // when every index is done
  void run_indexed(int64_t n, const std::function<void(int64_t)>& fn);
  // workers 0..n-1 poll the queue instead of sleeping (0: all sleep)
  void set_spin(int n);
  int size() const { return (int)th_.size() + 1; }
  static constexpr int kGroups = 5;
  static constexpr int kIndexedGroup = 4;

 private:
  void loop(int idx);
  bool run_one(std::unique_lock<std::mutex>& lk);
  std::vector<std::thread> th_;
  std::mutex mu_;
  std::condition_variable cv_, done_;
  std::vector<std::pair<int, std::function<void()>>> q_;
  size_t head_ = 0;
  int pending_[kGroups] = {};
  int running_ = 0;
  bool stop_ = false;
  std::atomic<int> queued_{0};
  std::atomic<int> spin_{0};
};

// Keeps idle workers polling the queue for the lifetime of a codec call: on
// the virtual machines this runs on, a worker woken from sleep runs its first
// milliseconds several times slower, which made the batched coarse coding
// 5-7x slower (measured on the 64-frame batch: decode's coarse levels 50 ms
// sleeping, 7.6 ms polling).
struct SpinScope {
  Pool* p;
  SpinScope(Pool* pool, int workers) : p(workers > 0 ? pool : nullptr) {
    if (p) p->set_spin(workers);
  }
  ~SpinScope() {
    if (p) p->set_spin(0);
  }
};


// Kernel families timed by the optional CUDA-event profiler.
enum Family {
  kFamSort = 0,  // Morton keys + radix sort + unique
  kFamLevels,    // level build (encoder) / code expansion (decoder)
  kFamHash,      // voxel hash + 27-neighbour map
  kFamEmbed,     // occupancy-code embedding gathers, bf16 conversions
  kFamUp,        // Upsampling + Pruning
  kFamDown,      // stride-2 down conv
  kFamConv,      // 3x3x3 sparse conv on the tensor cores (+ fused residual merge)
  kFamPred,      // predictor + integer softmax + cumulative table
  kFamCoder,     // device range coding of the network levels
  kFamCount
};

// Families whose launches the profiler can time on the graph and
// round-trip-free paths (their launches sit outside the captured graphs);
// timing any other family switches the codec to direct launches.
constexpr unsigned kAsyncProfiled = (1u << kFamSort) | (1u << kFamCoder);

// Per-family totals: summed launch durations (CUDA events on the codec's
// stream), launches, and the algorithmic bytes / integer ops the launches
// must touch (from the level sizes and the neighbour-pair counts).
struct Profile {
  unsigned mask = 0;  // families to time (0 = off)
  double ms[kFamCount] = {};
  int64_t launches[kFamCount] = {};
  double bytes[kFamCount] = {};
  double ops[kFamCount] = {};
  double staged[kFamCount] = {};  // bytes the kernels actually move (layout copies, maps)
};

struct Stats {
  int L = 0;
  int64_t N[kMaxDepth + 1] = {};
  double gpu_us = 0, host_us = 0;
  // host timeline (us since the call started): encode 0 octree ready, 1 all
  // launches issued, 2 coding done, 3 total; decode 4 coarse levels done,
  // 5 network + copy issue (sum), 6 level decoding (sum), 7 expansion issue
  // (sum), 8 total
  double phase_us[16] = {};
};

// One frame of the current batch on the host.
struct Frame {
  int L = 0, b = 0, t = 0;
  int64_t n = 0;                 // input points (encoder) / voxels (decoder)
  int64_t off[kHeights] = {};    // first row in the level arrays, by height
  int64_t cnt[kHeights] = {};    // rows of this frame, by height
  // coarse octree (depths 0..b-1) on the host: codes per depth, in order
  std::vector<std::vector<uint8_t>> coarse;
  // decoder: parsed stream
  const uint8_t* in = nullptr;
  size_t len = 0;
  int64_t chunk = 0;
  int64_t kc = 0;                   // coarse chunk: nodes per coarse substream
  int64_t cN[kMaxDepth + 1] = {};   // the coarse levels' sizes N_0 = 1, N_1 .. N_{b-1}
  size_t nco = 0;                   // coarse substreams (the network's follow them)
  std::vector<uint64_t> slen;
  std::vector<size_t> soff;
  uint64_t coarse_bytes() const {
    uint64_t s = 0;
    for (size_t k = 0; k < nco && k < slen.size(); k++) s += slen[k];
    return s;
  }
  size_t sub_base = 0;           // first substream task of this frame
  int status = 0;
};

class Codec {
 public:
  Codec() = default;
  ~Codec();
  int create(const lpc_config& cfg, const void* blob, size_t len);
  int encode(int nf, const int32_t* const* xyz, const int64_t* n, const int* Ls,
             uint8_t* const* out, const size_t* caps, size_t* lens);
  int decode(int nf, const uint8_t* const* in, const size_t* lens, int32_t* const* out,
             const int64_t* caps, int64_t* n_out);
  int probs(const int32_t* d_xyz, int64_t n, int d, uint16_t* d_cdf, int64_t cap, int64_t* nn);
  int depth() const { return cfg_.L; }

  std::string err;
  Stats stats;
  Profile prof;
  void profile_reset(unsigned mask);

 private:
  int fail(int st, const std::string& msg) {
    err = msg;
    return st;
  }
  int cuda_check(const char* what);
  int check_device_error();
  int sync_and_check(const char* what);
  // octree of the batch: heights 0..6 on the device, coarse levels on the host
  int build_levels_device(int nf, const int32_t* const* xyz, const int64_t* n, bool coarse);
  uint8_t* coarse_codes(int h) const {  // codes of coarse height h >= 7 (encoder)
    return reinterpret_cast<uint8_t*>(d_cdf_) + (size_t)(h - kHeights) * P_;
  }
  void fetch_frame_offsets(int nf);
  void begin_batch();
  void level_bytes();
  // network
  void embed(const DEmb& E, int h, int8_t* out, int stride, int col);
  void up(const DLayer& W, int h, const int8_t* x, int xs, int8_t* out, int os, EmbSrc oe = {},
          int oe_col = 0);
  // E[Y] of the height-h codes, read from the embedding table
  EmbSrc emb_src(const DEmb& E, int h) const { return EmbSrc{E.table, code_[h]}; }
  void to_bf16(const int8_t* x, int xs, int cols, int z, int h);
  void conv(const DLayer& W, int h, const int32_t* nbr, int slot, const void* xb, int xbs,
            int8_t* out, int os, int oc, const DRes* res, void* outb, int outb_z,
            EmbSrc emb = {}, int emb_col = 0);
  void kmap(int h, int32_t* nbr, int slot);
  void ensure_nbr(int h);
  const int8_t* shallow_F(int h, int* stride);
  // part: kNetAll, or a level's Downsampling chain alone (kNetPre) and the
  // rest (kNetPost)
  enum { kNetAll = 0, kNetPre = 1, kNetPost = 2 };
  void net_level(int j, int mode, uint16_t* cdf, uint32_t* enc, int8_t* logits,
                 int part = kNetAll);
  void run_level(int j, int mode, uint16_t* cdf, uint32_t* enc);
  // Scratch of a level's network.  Lane 0 is the codec's own; lanes 1 and 2
  // let the encoder run two levels beside the others (every level's input
  // is known to the encoder, and the small levels leave most SMs idle).
  struct Scratch {
    int8_t *y1 = nullptr, *g0 = nullptr, *g1 = nullptr, *gk = nullptr, *hx0 = nullptr,
           *hx1 = nullptr, *fo = nullptr;
    void *xb16 = nullptr, *y1b16 = nullptr;
  };
  static constexpr int kLanes = 3;
  static constexpr int64_t kLanePoints = (int64_t)1 << 22;  // lanes 1, 2 up to this capacity
  Scratch lane_[kLanes];
  cudaStream_t ls_[kLanes] = {};
  cudaEvent_t lev_[4] = {};
  bool lanes_ = false;
  void set_lane(int l);
  cudaGraphExec_t genc_ = nullptr;  // the encoder's five levels, lanes side by side
  bool genc_fail_ = false;
  int genc_kern_ = 0;
  void enc_network_lanes();
  void run_enc_network();
  bool enc_graphs_ready() const;
  // grid size for level height h: its size, or the capacity while a graph
  // is captured (kernels read the real size on the device)
  int64_t gridn(int h) const { return cap_grid_ ? P_ : N_[h]; }
  bool cap_grid_ = false;
  cudaStream_t gs_ = nullptr;
  cudaStream_t cs_ = nullptr;  // copies that overlap the network (encoder's coarse codes)
  cudaEvent_t up_ev_ = nullptr;  // decoder: the network levels' bytes are on the device
  cudaEvent_t gev_[2] = {};
  cudaGraphExec_t gexec_[3][5] = {};
  int gkern_[3][5] = {};
  bool gfail_[3][5] = {};
  // conv autotuner: the fastest kernel variant per input width (32, 64),
  // timed on the first direct launches of each width
 public:
  int conv_variant_[2] = {-1, -1};
  float conv_tune_ms_[2][kConvVariants] = {};
  int pred_variant_ = -1;  // predictor: CUDA cores or tensor cores
  // up-steps of 32- and 64-channel inputs: CUDA cores or tensor cores
  int up_variant_[2] = {-1, -1};
  float up_tune_ms_[2][kUpVariants] = {};
  // fix the variants (captured graphs are dropped: they hold the old ones)
  void set_tuning(const int* v) {
    conv_variant_[0] = v[0];
    conv_variant_[1] = v[1];
    pred_variant_ = v[2];
    up_variant_[0] = v[3];
    up_variant_[1] = v[4];
    for (auto& row : gexec_)
      for (auto& e : row)
        if (e) {
          cudaGraphExecDestroy(e);
          e = nullptr;
        }
    if (genc_) cudaGraphExecDestroy(genc_);
    genc_ = nullptr;
  }
  float pred_tune_ms_[kPredVariants] = {};
 private:
  cudaEvent_t tev_[2] = {};
  void tune_conv(const ConvTcArgs& a, int cin, int h);
  int64_t hash_slots(int64_t n) const;
  // profiler: bracket a launch of family f; ops/bytes are algorithmic work
  // (pair_slot >= 0: ops/bytes are per neighbour pair, scaled at collection);
  // staged / per_pair_staged (< 0: the algorithmic figures) are the bytes
  // the launch actually moves
  void pbeg(int f);
  void pend(int f, double bytes, double ops, int pair_slot = -1, double per_pair_ops = 0,
            double per_pair_bytes = 0, double staged = -1, double per_pair_staged = -1);
  void prof_collect();
  struct Mark {
    int f, e0, e1, pair_slot;
    double bytes, ops, ppo, ppb, staged, pps;
  };
  std::vector<cudaEvent_t> pev_;
  std::vector<Mark> marks_;
  int pev_used_ = 0;
  uint64_t* d_pairs_ = nullptr;  // [2]: present neighbour pairs at V_b, V_t

  lpc_config cfg_{};
  int64_t P_ = 0;  // batch capacity in points (rows per level array)
  int F_ = 0;      // batch capacity in frames
  cudaStream_t st_ = nullptr;
  Model M_;
  Pool* pool_ = nullptr;
  // per-batch state
  int nf_ = 0;
  std::vector<Frame> fr_;
  int64_t N_[kHeights] = {};  // rows per height (all frames)
  // per batch: which propagated features F (by height) and kernel maps exist
  bool have_F_[kHeights] = {}, have_nbr_[kHeights] = {};
  // device workspace: level arrays by height (0 = leaves of every frame)
  void* dmem_ = nullptr;
  uint64_t* key_[kHeights] = {};
  uint8_t* code_[kHeights] = {};   // code of each node (children mask), heights 1..6
  uint32_t* off_[kHeights] = {};   // child offsets into height h-1, heights 1..6
  uint32_t* par_[kHeights] = {};   // parent row at height h+1, heights 0..5
  int64_t* d_N_ = nullptr;         // [kHeights + 1]: rows per height, then the point count
  int64_t* d_foff_ = nullptr;      // [kHeights][F + 1] frame offsets
  // encoder's coarse heights 7..max_h_ (depths below b - 1 of every frame):
  // keys ping-pong through the sort buffers, codes in the (then unused)
  // table buffer, one P-byte slot per height
  int64_t* d_cN_ = nullptr;        // [kMaxDepth + 2] rows per coarse height
  uint32_t* d_cup_ = nullptr;      // tile counts and offsets of the coarse heights (encoder)
  int64_t* d_cfoff_ = nullptr;     // [kMaxDepth + 1][F + 1] frame offsets per coarse height
  int64_t* h_cN_ = nullptr;
  int64_t* h_cfoff_ = nullptr;
  int max_h_ = kHeights - 1;
  DevFrame* d_fr_ = nullptr;       // [F]
  int* d_L_ = nullptr;             // [F] frame depths
  int* d_err_ = nullptr;
  uint64_t* d_keys0_ = nullptr;
  SortScratch sort_;
  ScanScratch scan_;
  HashTable hash_;
  int32_t* nbr_[kHeights] = {};  // kernel maps by height, 5 down to the deepest conv level
  uint32_t* tmask_[kHeights] = {};  // their conv tiles' present-offset masks
  int2* ranges_[kHeights] = {};     // and the conv CTAs' tile runs of about equal cost
  int8_t *fb_ = nullptr, *xb_ = nullptr, *xt_ = nullptr, *y1_ = nullptr, *xe_ = nullptr;
  int8_t *fmid_ = nullptr, *gk_ = nullptr;  // F^{t-1} when t = L - 3; G^k of the ablations
  int8_t *g_[2] = {}, *hx_[2] = {}, *fo_ = nullptr;
  void *xb16_ = nullptr, *y1b16_ = nullptr;  // bf16 (q - z) inputs of the convs
  uint16_t* d_cdf_ = nullptr;
  uint32_t* d_enc_ = nullptr;      // [5][P] intervals of the true symbols, by height 5..1
  // pinned host workspace
  void* hmem_ = nullptr;
  int64_t* h_N_ = nullptr;
  int64_t* h_foff_ = nullptr;
  DevFrame* h_fr_ = nullptr;
  int* h_L_ = nullptr;
  int* h_err_ = nullptr;
  uint64_t* h_keys6_ = nullptr;    // V_{b-1} keys of every frame (height 6)
  uint8_t* h_codes_ = nullptr;     // [kHeights][P] codes by height
  uint32_t* h_enc_ = nullptr;      // [5][P]
  uint16_t* h_ring_ = nullptr;     // cumulative-table ring: 2 halves x ring_slots_ chunks
  int ring_slots_ = 0;
  uint8_t* h_arena_ = nullptr;     // pinned, pre-faulted: coded substreams
  size_t arena_cap_ = 0;
  struct SubTask {
    int f, d;  // frame, depth
    int64_t start, count;
    size_t arena, len;  // offset in the host arena, or in the device-coded bytes if rc >= 0
    int64_t rc = -1;    // index of the device-coded chunk
    std::vector<uint32_t> parts;  // a coarse level: its substreams' lengths, in order
  };
  // growable buffers for the device range coder (replaced only when a call
  // needs more; the stream is synchronised first)
  struct Buf {
    void* p = nullptr;
    size_t cap = 0;
  };
  void* dgrow(Buf& b, size_t bytes);
  void* hgrow(Buf& b, size_t bytes);
  Buf d_rcck_, d_rclen_, d_rcbuf_, h_rcck_, h_rclen_, h_rcbuf_, h_ccodes_;
  Buf d_subfr_, h_subfr_, d_subs_, h_subs_, d_nck_;  // device-built substream tables
  Buf h_cck_, d_cck_, h_cchk_, d_cchk_;  // coarse substreams decoded on the device
  bool dev_rc_ = true;
  std::vector<int64_t> in_base_;  // each decoded frame's first byte in d_rcbuf_
  int decode_net_device(int nd, int64_t* n_out, const std::vector<int>& dev, const int64_t* caps);
  int decode_net_async(int nd, int64_t* n_out, const std::vector<int>& dev, const int64_t* caps);
  // coarse codes to the device arrays (decoded on the host, or decoded there
  // from the uploaded stream when on_device) and expanded to the keys of V_{b-1}
  int expand_coarse_device(int nd, bool on_device);
  std::vector<SubTask> tasks_;
  std::vector<cudaEvent_t> ev_;
};

}  // namespace lpc
