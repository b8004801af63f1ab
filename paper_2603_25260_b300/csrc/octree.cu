// Octree construction on the device (supplement, "Implementation of Octree
// Operations"): Morton keys, an LSD radix sort, duplicate removal, the
// level-by-level floor-halving with occupancy codes, and the decoder's
// code -> child expansion.  Level sizes stay on the device, so a whole build
// is queued without host round trips.
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "kernels.h"

namespace lpc {

static std::atomic<int64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------------ block scan --
// Exclusive scan of one u32 per thread over a block of NT threads.
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total, uint32_t* sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < NT / 32 ? sm[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < NT / 32) sm[lane] = t;
  }
  __syncthreads();
  uint32_t r = (w ? sm[w - 1] : 0) + x - v;
  *total = sm[NT / 32 - 1];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------ radix sort --
constexpr int kRsThreads = 256, kRsItems = 4, kRsTile = kRsThreads * kRsItems;

int64_t sort_tiles(int64_t n) { return (n + kRsTile - 1) / kRsTile; }

__global__ void __launch_bounds__(kRsThreads)
k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, uint32_t* hist, int64_t nt) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
  for (int i = 0; i < kRsItems; i++) {
    int64_t idx = base + i * kRsThreads + threadIdx.x;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nt + blockIdx.x] = h[threadIdx.x];
}

// Per digit (one block each): exclusive scan of the digit's tile counts over
// the tiles, in place, and the digit's total into dtot[digit].
__global__ void __launch_bounds__(1024) k_rs_digit_scan(uint32_t* hist, int64_t nt,
                                                        uint32_t* dtot) {
  __shared__ uint32_t sm[32];
  uint32_t* h = hist + (int64_t)blockIdx.x * nt;
  uint32_t carry = 0;
  for (int64_t base = 0; base < nt; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const uint32_t v = i < nt ? h[i] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan<1024>(v, &tot, sm);
    if (i < nt) h[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) dtot[blockIdx.x] = carry;
}

// Stable scatter: each warp ranks its 512 keys (warp-striped, so (item, lane)
// order is the input order) with match.any, warps are ordered by a per-digit
// prefix, tiles by the per-digit scan of the histogram, digits by the
// exclusive scan of the digit totals.
__global__ void __launch_bounds__(kRsThreads)
k_rs_scatter(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, int64_t n, int shift,
             const uint32_t* __restrict__ offs, int64_t nt, const uint32_t* __restrict__ dtot) {
  __shared__ uint32_t cnt[kRsThreads / 32][256];
  __shared__ uint32_t dbase[256], sm[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < (kRsThreads / 32) * 256; i += kRsThreads) (&cnt[0][0])[i] = 0;
  {
    uint32_t tot;
    dbase[threadIdx.x] = block_excl_scan<kRsThreads>(dtot[threadIdx.x], &tot, sm);
  }
  __syncthreads();
  const int64_t seg = (int64_t)blockIdx.x * kRsTile + w * (kRsItems * 32);
  const uint32_t lt = (1u << lane) - 1u;
  uint64_t key[kRsItems];
  uint32_t rank[kRsItems];
  int dig[kRsItems];
#pragma unroll
  for (int i = 0; i < kRsItems; i++) {
    const int64_t idx = seg + i * 32 + lane;
    const bool valid = idx < n;
    key[i] = valid ? in[idx] : 0;
    const int d = valid ? (int)((key[i] >> shift) & 255) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t r = 0;
    if (valid) r = cnt[w][d] + __popc(peers & lt);
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) cnt[w][d] += __popc(peers);
    __syncwarp();
    rank[i] = r;
    dig[i] = d;
  }
  __syncthreads();
  {
    uint32_t run = 0;
    for (int ww = 0; ww < kRsThreads / 32; ww++) {
      uint32_t t = cnt[ww][threadIdx.x];
      cnt[ww][threadIdx.x] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kRsItems; i++) {
    if (dig[i] < 256)
      out[dbase[dig[i]] + offs[(int64_t)dig[i] * nt + blockIdx.x] + cnt[w][dig[i]] + rank[i]] =
          key[i];
  }
}

uint64_t* radix_sort(uint64_t* keys, int64_t n, int bits, bool frame_bits, const SortScratch& s,
                     cudaStream_t st) {
  if (n <= 1) return keys;
  const int64_t nt = sort_tiles(n);
  uint64_t* a = keys;
  uint64_t* b = s.alt;
  int shifts[9], ns = 0;
  for (int shift = 0; shift < bits && shift < 56; shift += 8) shifts[ns++] = shift;
  if (frame_bits || bits > 56) shifts[ns++] = 56;
  for (int i = 0; i < ns; i++) {
    const int shift = shifts[i];
    uint32_t* dtot = s.hist + 256 * nt;
    k_rs_hist<<<(unsigned)nt, kRsThreads, 0, st>>>(a, n, shift, s.hist, nt);
    k_rs_digit_scan<<<256, 1024, 0, st>>>(s.hist, nt, dtot);
    k_rs_scatter<<<(unsigned)nt, kRsThreads, 0, st>>>(a, b, n, shift, s.hist, nt, dtot);
    count_launches(3);
    std::swap(a, b);
  }
  return a;
}

// ---------------------------------------------------------- Morton keys --
__global__ void k_morton(const int32_t* __restrict__ xyz, int64_t n, int L, uint64_t* keys,
                         int* err) {
  const int32_t side = 1 << L;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) {
      set_error(err, kErrCoord);
      x = y = z = 0;
    }
    keys[i] = morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
  }
}

void launch_morton(const int32_t* xyz, int64_t n, int L, uint64_t* keys, int* err,
                   cudaStream_t st) {
  if (n <= 0) return;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 8);
  k_morton<<<blocks, 256, 0, st>>>(xyz, n, L, keys, err);
  count_launches(1);
}

__global__ void k_keys_to_xyz(const uint64_t* __restrict__ keys, const int64_t* d_n,
                              int32_t* xyz) {
  const int64_t n = *d_n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = keys[i];
    xyz[3 * i] = (int32_t)compact3(k >> 2);
    xyz[3 * i + 1] = (int32_t)compact3(k >> 1);
    xyz[3 * i + 2] = (int32_t)compact3(k);
  }
}

void launch_keys_to_xyz(const uint64_t* keys, const int64_t* d_n, int64_t cap, int L,
                        int32_t* xyz, cudaStream_t st) {
  (void)L;
  if (cap <= 0) return;
  int blocks = (int)std::min<int64_t>((cap + 255) / 256, 148 * 8);
  k_keys_to_xyz<<<blocks, 256, 0, st>>>(keys, d_n, xyz);
  count_launches(1);
}

// ------------------------------------------------------ frame batches --
// Key of point i of the batch: (frame << 58) | Morton(x, y, z); the frame of
// a global index is found by binary search over the frames' prefix counts.
__global__ void k_morton_batch(const DevFrame* __restrict__ fr, int nf, int64_t total,
                               uint64_t* keys, int* err) {
  __shared__ DevFrame sf[kMaxBatch];
  for (int i = threadIdx.x; i < nf; i += blockDim.x) sf[i] = fr[i];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sf[mid].pre <= i) lo = mid;
      else hi = mid - 1;
    }
    const DevFrame& f = sf[lo];
    const int64_t j = i - f.pre;
    const int32_t side = 1 << f.L;
    int32_t x = f.xyz[3 * j], y = f.xyz[3 * j + 1], z = f.xyz[3 * j + 2];
    if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) {
      set_error(err, kErrCoord);
      x = y = z = 0;
    }
    keys[i] = ((uint64_t)lo << kFrameShift) | morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
  }
}

void launch_morton_batch(const DevFrame* fr, int nf, int64_t total, uint64_t* keys, int* err,
                         cudaStream_t st) {
  if (total <= 0) return;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 8);
  k_morton_batch<<<blocks, 256, 0, st>>>(fr, nf, total, keys, err);
  count_launches(1);
}

// foff[h * (nf + 1) + f] = first row of frame f in the level array of
// height h (lower bound of f << 58); the last entry is the level size.
__global__ void k_frame_offsets(LevelPtrs lv, int nh, int nf, int64_t* foff) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nh * (nf + 1)) return;
  const int h = t / (nf + 1), f = t % (nf + 1);
  const int64_t n = *lv.n[h];
  int64_t r = n;
  if (f < nf) {
    const uint64_t target = (uint64_t)f << kFrameShift;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (lv.key[h][mid] < target) lo = mid + 1;
      else hi = mid;
    }
    r = lo;
  }
  foff[t] = r;
}

void launch_frame_offsets(const LevelPtrs& lv, int nh, int nf, int64_t* foff, cudaStream_t st) {
  const int n = nh * (nf + 1);
  k_frame_offsets<<<(n + 127) / 128, 128, 0, st>>>(lv, nh, nf, foff);
  count_launches(1);
}

// Leaf keys -> coordinates in every frame's own output buffer.
__global__ void k_keys_to_xyz_batch(const uint64_t* __restrict__ keys, const int64_t* d_n,
                                    const DevFrame* __restrict__ fr, const int64_t* foff0) {
  const int64_t n = *d_n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t kf = keys[i];
    const int f = (int)(kf >> kFrameShift);
    const uint64_t k = kf & kLowMask;
    int32_t* out = fr[f].out + 3 * (i - foff0[f]);
    out[0] = (int32_t)compact3(k >> 2);
    out[1] = (int32_t)compact3(k >> 1);
    out[2] = (int32_t)compact3(k);
  }
}

void launch_keys_to_xyz_batch(const uint64_t* keys, const int64_t* d_n, int64_t n_host,
                              const DevFrame* fr, const int64_t* foff0, cudaStream_t st) {
  if (n_host <= 0) return;
  const int blocks = (int)std::min<int64_t>((n_host + 255) / 256, 148 * 8);
  k_keys_to_xyz_batch<<<blocks, 256, 0, st>>>(keys, d_n, fr, foff0);
  count_launches(1);
}

// ------------------------------------------------- device-size scan pass --
// Three kernels: per-tile sums, one-block scan of the tile sums, per-element
// exclusive prefix handed to Op::emit.  Element count is read on the device.
constexpr int kScThreads = 256, kScItems = 2, kScTile = kScThreads * kScItems;

int64_t scan_tiles_for(int64_t cap) { return std::max<int64_t>(1, (cap + kScTile - 1) / kScTile); }

template <class Op>
__global__ void __launch_bounds__(kScThreads) k_sc_reduce(Op op, const int64_t* d_n,
                                                          uint32_t* tiles) {
  __shared__ uint32_t sm[32];
  const int64_t n = *d_n;
  const int64_t base = (int64_t)blockIdx.x * kScTile;
  if (base >= n) return;
  uint32_t s = 0;
  for (int i = 0; i < kScItems; i++) {
    int64_t idx = base + (int64_t)threadIdx.x * kScItems + i;
    if (idx < n) s += op.value(idx);
  }
  uint32_t tot;
  block_excl_scan<kScThreads>(s, &tot, sm);
  if (threadIdx.x == 0) tiles[blockIdx.x] = tot;
}

template <class Op>
__global__ void __launch_bounds__(1024) k_sc_top(Op op, const int64_t* d_n, uint32_t* tiles) {
  __shared__ uint32_t sm[32];
  const int64_t n = *d_n;
  const int64_t len = (n + kScTile - 1) / kScTile;
  const int64_t per = (len + 1023) / 1024;
  const int64_t b = threadIdx.x * per, e = std::min(len, b + per);
  uint32_t s = 0;
  for (int64_t i = b; i < e; i++) s += tiles[i];
  uint32_t tot;
  uint32_t run = block_excl_scan<1024>(s, &tot, sm);
  for (int64_t i = b; i < e; i++) {
    uint32_t v = tiles[i];
    tiles[i] = run;
    run += v;
  }
  if (threadIdx.x == 0) op.finish(tot, n);
}

template <class Op>
__global__ void __launch_bounds__(kScThreads) k_sc_emit(Op op, const int64_t* d_n,
                                                        const uint32_t* tiles) {
  __shared__ uint32_t sm[32];
  const int64_t n = *d_n;
  const int64_t base = (int64_t)blockIdx.x * kScTile;
  if (base >= n) return;
  const int64_t first = base + (int64_t)threadIdx.x * kScItems;
  uint32_t v[kScItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScItems; i++) {
    v[i] = first + i < n ? op.value(first + i) : 0;
    s += v[i];
  }
  uint32_t tot;
  uint32_t run = tiles[blockIdx.x] + block_excl_scan<kScThreads>(s, &tot, sm);
#pragma unroll
  for (int i = 0; i < kScItems; i++) {
    if (first + i < n) op.emit(first + i, run, n);
    run += v[i];
  }
}

template <class Op>
static void run_scan(const Op& op, const int64_t* d_n, int64_t cap, const ScanScratch& s,
                     cudaStream_t st) {
  const int64_t nt = scan_tiles_for(cap);
  k_sc_reduce<Op><<<(unsigned)nt, kScThreads, 0, st>>>(op, d_n, s.tiles);
  k_sc_top<Op><<<1, 1024, 0, st>>>(op, d_n, s.tiles);
  k_sc_emit<Op><<<(unsigned)nt, kScThreads, 0, st>>>(op, d_n, s.tiles);
  count_launches(3);
}

struct UniqueOp {
  const uint64_t* k;
  uint64_t* out;
  int64_t* nout;
  __device__ uint32_t value(int64_t i) const { return i == 0 || k[i] != k[i - 1]; }
  __device__ void emit(int64_t i, uint32_t ex, int64_t) const {
    if (value(i)) out[ex] = k[i];
  }
  __device__ void finish(uint32_t total, int64_t) const { *nout = total; }
};

void launch_unique(const uint64_t* keys, const int64_t* d_n, int64_t cap, uint64_t* out,
                   int64_t* d_nout, const ScanScratch& s, cudaStream_t st) {
  run_scan(UniqueOp{keys, out, d_nout}, d_n, cap, s, st);
}

// Parent = key >> 3 (floor-halving of every coordinate); consecutive
// duplicates removed; code = OR of 1 << (child key & 7) over the children.
struct LevelOp {
  const uint64_t* ck;
  uint64_t* pk;
  uint8_t* pc;
  uint32_t* poff;
  uint32_t* cpar;
  int64_t* np;
  __device__ uint32_t value(int64_t i) const {
    return i == 0 || parent_key(ck[i]) != parent_key(ck[i - 1]);
  }
  __device__ void emit(int64_t i, uint32_t ex, int64_t n) const {
    const uint32_t h = value(i);
    if (cpar) cpar[i] = ex + h - 1;
    if (h) {
      const uint64_t p = parent_key(ck[i]);
      pk[ex] = p;
      if (poff) poff[ex] = (uint32_t)i;
      uint32_t code = 0;
      for (int64_t j = i; j < n && j < i + 8 && parent_key(ck[j]) == p; j++)
        code |= 1u << (ck[j] & 7);
      pc[ex] = (uint8_t)code;
    }
  }
  __device__ void finish(uint32_t total, int64_t n) const {
    *np = total;
    if (poff) poff[total] = (uint32_t)n;
  }
};

void launch_level_up(const uint64_t* ckeys, const int64_t* d_nc, int64_t cap_c, uint64_t* pkeys,
                     uint8_t* pcodes, uint32_t* poff, uint32_t* cpar, int64_t* d_np,
                     const ScanScratch& s, cudaStream_t st) {
  run_scan(LevelOp{ckeys, pkeys, pcodes, poff, cpar, d_np}, d_nc, cap_c, s, st);
}

// --------------------------------------------------- coarse heights --
// The coarse heights (above V_{b-1}) are small.  Decoder: one block walks
// the heights under 16384 parents each (kCoarseScanMin) in a single launch.
constexpr int kCoThreads = 1024, kCoItems = 4, kCoChunk = kCoThreads * kCoItems;

// Encoder: every coarse height 7..top at once, from the sorted keys of
// height 6.  A node of height h >= 6 is the key's frame bits with its Morton
// bits shifted down by 3 (h - 6), so key j opens a node at height h exactly
// when h <= hmax_j: the top height if j opens a frame (or is the first key),
// else 6 + floor(p / 3) for p the highest Morton bit in which keys j - 1 and
// j differ (they agree above bit 3 (h - 6) - 1 exactly when p < 3 (h - 6)).
// The nodes of height h are the keys with hmax >= h, in key order, so a
// scan of [hmax_j >= h] numbers them; the node of height h - 1 that key j
// opens has the octant (key_j >> 3 (h - 7)) & 7 within its parent, the node
// of height h holding key j.  Three launches, all heights together:
//  - count: per tile of keys, the nodes each height has there (and the
//    tile's code bytes cleared at every height);
//  - scan (one block): tile offsets per height, the heights' sizes, and the
//    offsets of the frames after the last key's;
//  - emit: every opened node ORs its octant bit into its parent's code and
//    a key that opens a frame writes that frame's offset at every height.
// The keys of the coarse heights themselves are not needed and not written.
constexpr int kCuThreads = 256, kCuItems = 2, kCuTile = kCuThreads * kCuItems;
constexpr int kCuWords = 8;  // per-thread node counts of heights 7 .. 22, two 16-bit halves a word

int64_t coarse_up_blocks(int64_t cap) { return std::max<int64_t>(1, (cap + kCuTile - 1) / kCuTile); }

__device__ __forceinline__ int open_height(uint64_t prev, uint64_t cur, bool first, int top) {
  const uint64_t x = prev ^ cur;
  if (first || (x >> kFrameShift)) return top;
  const int p = 63 - __clzll((long long)(x & kLowMask));  // keys are unique: x != 0
  return min(top, 6 + p / 3);
}

// This thread's kCuItems consecutive keys from j0: their keys, hmax (0 past
// the end) and the packed counts of the nodes they open per height.
struct CuItems {
  uint64_t key[kCuItems];
  int hm[kCuItems];
  uint64_t prev;  // the key before j0
  uint32_t w[kCuWords];
};

__device__ __forceinline__ void cu_items(const uint64_t* __restrict__ key6, int64_t n6, int64_t j0,
                                         int top, CuItems& it) {
  uint64_t prev = j0 > 0 && j0 - 1 < n6 ? key6[j0 - 1] : 0ull;
  it.prev = prev;
#pragma unroll
  for (int k = 0; k < kCuWords; k++) it.w[k] = 0;
#pragma unroll
  for (int i = 0; i < kCuItems; i++) {
    const int64_t j = j0 + i;
    const uint64_t cur = j < n6 ? key6[j] : 0ull;
    it.key[i] = cur;
    const int hm = j < n6 ? open_height(prev, cur, j == 0, top) : 0;
    it.hm[i] = hm;
    prev = cur;
#pragma unroll
    for (int k = 0; k < kCuWords; k++)
      it.w[k] += (uint32_t)(hm >= 7 + 2 * k) | ((uint32_t)(hm >= 8 + 2 * k) << 16);
  }
}

__global__ void __launch_bounds__(kCuThreads)
k_cu_count(const uint64_t* __restrict__ key6, const int64_t* d_n6, int top, uint8_t* codes,
           int64_t stride, uint32_t* bt, int64_t nbmax) {
  __shared__ uint32_t ws[kCuThreads / 32][kCuWords];
  const int64_t n6 = *d_n6;
  const int64_t b = blockIdx.x, t0 = b * kCuTile;
  if (t0 >= n6) return;  // the scan reads only the tiles below n6
  // a height has at most n6 nodes: clear this tile's share of every
  // height's code bytes before the emit pass ORs bits into them
  const int64_t e = min(n6, t0 + (int64_t)kCuTile);
  for (int h = 7; h <= top; h++)
    for (int64_t i = t0 + threadIdx.x; i < e; i += kCuThreads) codes[(int64_t)(h - 7) * stride + i] = 0;
  CuItems it;
  cu_items(key6, n6, t0 + (int64_t)threadIdx.x * kCuItems, top, it);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kCuWords; k++) {
    const uint32_t v = __reduce_add_sync(0xffffffffu, it.w[k]);  // halves stay below 2^16
    if (lane == 0) ws[w][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kCuWords) {
    uint32_t v = 0;
#pragma unroll
    for (int q = 0; q < kCuThreads / 32; q++) v += ws[q][threadIdx.x];
    bt[(int64_t)(2 * threadIdx.x) * nbmax + b] = v & 0xFFFFu;
    bt[(int64_t)(2 * threadIdx.x + 1) * nbmax + b] = v >> 16;
  }
}

// One warp per height: the tiles' node counts scanned 32 at a time.
__global__ void __launch_bounds__(32 * 2 * kCuWords)
k_cu_scan(const uint64_t* __restrict__ key6, const int64_t* d_n6, int top, const uint32_t* bt,
          uint32_t* bo, int64_t nbmax, int64_t* cN, int nf, int64_t* foff) {
  const int lane = threadIdx.x & 31, h = 7 + (threadIdx.x >> 5);
  if (h > top) return;
  const int64_t n6 = *d_n6;
  const int64_t nb = (n6 + kCuTile - 1) / kCuTile;
  const uint32_t* src = bt + (int64_t)(h - 7) * nbmax;
  uint32_t* dst = bo + (int64_t)(h - 7) * nbmax;
  uint32_t run = 0;
  for (int64_t base = 0; base < nb; base += 32) {
    const int64_t i = base + lane;
    const uint32_t v = i < nb ? src[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (i < nb) dst[i] = run + x - v;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) cN[h] = run;
  // frames after the last key's have no node: they start at the end
  const int lastf = n6 > 0 ? (int)(key6[n6 - 1] >> kFrameShift) : -1;
  for (int f = lastf + 1 + lane; f <= nf; f += 32) foff[(int64_t)h * (nf + 1) + f] = run;
}

// OR v into the byte at p through its aligned 32-bit word.
__device__ __forceinline__ void or_byte(uint8_t* p, uint32_t v) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  atomicOr(reinterpret_cast<unsigned int*>(a & ~(uintptr_t)3), v << (8 * (a & 3)));
}

__global__ void __launch_bounds__(kCuThreads)
k_cu_emit(const uint64_t* __restrict__ key6, const int64_t* d_n6, int top, uint8_t* codes,
          int64_t stride, const uint32_t* __restrict__ bo, int64_t nbmax, int nf, int64_t* foff) {
  __shared__ uint32_t ws[kCuThreads / 32][kCuWords];
  const int64_t n6 = *d_n6;
  const int64_t b = blockIdx.x, t0 = b * kCuTile;
  if (t0 >= n6) return;
  const int64_t j0 = t0 + (int64_t)threadIdx.x * kCuItems;
  CuItems it;
  cu_items(key6, n6, j0, top, it);
  // block-exclusive scan of the packed counts: warp scans, then the warps'
  // totals in front
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t ex[kCuWords];
#pragma unroll
  for (int k = 0; k < kCuWords; k++) {
    uint32_t x = it.w[k];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    ex[k] = x - it.w[k];
    if (lane == 31) ws[w][k] = x;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kCuWords; k++)
    for (int q = 0; q < w; q++) ex[k] += ws[q][k];
  // pos[hi]: nodes of height 7 + hi before this thread's next key
  uint32_t pos[2 * kCuWords];
#pragma unroll
  for (int hi = 0; hi < 2 * kCuWords; hi++)
    pos[hi] = hi + 7 <= top ? bo[(int64_t)hi * nbmax + b] + ((ex[hi >> 1] >> (16 * (hi & 1))) & 0xFFFFu)
                            : 0u;
  uint64_t prev = it.prev;
#pragma unroll
  for (int i = 0; i < kCuItems; i++) {
    const int64_t j = j0 + i;
    if (j >= n6) break;
    const uint64_t key = it.key[i];
    const int hm = it.hm[i];
    const int fj = (int)(key >> kFrameShift);
    const int fp = j == 0 ? -1 : (int)(prev >> kFrameShift);
    if (fj != fp) {  // key j opens frame fj (and the empty frames before it) at every height
#pragma unroll
      for (int hi = 0; hi < 2 * kCuWords; hi++) {
        if (hi + 7 > top) break;
        for (int f = fp + 1; f <= fj; f++) foff[(int64_t)(hi + 7) * (nf + 1) + f] = pos[hi];
      }
    }
    // the node of height h - 1 that key j opens (h - 1 <= hm): its octant
    // bit into the code of its parent, node pos - 1 (or pos when key j opens
    // the parent too) of height h
#pragma unroll
    for (int hi = 0; hi < 2 * kCuWords; hi++) {
      const int h = hi + 7;
      if (h > top || h - 1 > hm) break;
      const uint32_t P = pos[hi] + (hm >= h ? 1u : 0u) - 1u;
      or_byte(codes + (int64_t)hi * stride + P, 1u << ((key >> (3 * hi)) & 7));
    }
#pragma unroll
    for (int hi = 0; hi < 2 * kCuWords; hi++)
      if (hi + 7 <= hm) pos[hi]++;
    prev = key;
  }
}

void launch_coarse_up(const uint64_t* key6, const int64_t* d_n6, int64_t cap6, int top,
                      uint8_t* codes, int64_t stride, int64_t* cN, int nf, int64_t* foff,
                      uint32_t* scratch, cudaStream_t st) {
  if (top < 7) return;
  top = std::min(top, 6 + 2 * kCuWords);
  const int64_t nbmax = coarse_up_blocks(cap6);
  uint32_t* bt = scratch;
  uint32_t* bo = scratch + (int64_t)2 * kCuWords * nbmax;
  k_cu_count<<<(unsigned)nbmax, kCuThreads, 0, st>>>(key6, d_n6, top, codes, stride, bt, nbmax);
  k_cu_scan<<<1, 32 * 2 * kCuWords, 0, st>>>(key6, d_n6, top, bt, bo, nbmax, cN, nf, foff);
  k_cu_emit<<<(unsigned)nbmax, kCuThreads, 0, st>>>(key6, d_n6, top, codes, stride, bo, nbmax, nf,
                                                      foff);
  count_launches(3);
}

// Decoder: from nf roots (frame f's root at the top height) down to height
// 6 through the codes of heights top..7 (codes + (h - 7) * stride, counts
// from the host in cnt[h]); children of every set bit in ascending order;
// keys ping-pong through k0 / k1, height 6 into key6, its count into n6.
// At most cap children per height are written (kErrCapacity beyond).
struct CoarseCounts {
  int64_t n[kMaxDepth + 1];
};
__global__ void __launch_bounds__(kCoThreads)
k_coarse_down(const uint64_t* __restrict__ roots, int top, int bottom,
              const uint8_t* __restrict__ codes, int64_t stride, CoarseCounts cnt, int64_t cap,
              uint64_t* k0, uint64_t* k1, uint64_t* key6, int64_t* n6, int* err) {
  __shared__ uint32_t sm[32];
  const uint64_t* src = roots;
  for (int h = top; h >= bottom; h--) {
    const int64_t n = cnt.n[h];
    const uint8_t* code = codes + (int64_t)(h - 7) * stride;
    uint64_t* dst = h == 7 ? key6 : ((h - 1) & 1 ? k1 : k0);
    int64_t run = 0;
    for (int64_t base = 0; base < n; base += kCoChunk) {
      const int64_t first = base + (int64_t)threadIdx.x * kCoItems;
      uint32_t pc[kCoItems], c = 0;
      uint64_t pk[kCoItems];  // the parents' keys, loaded beside their codes
#pragma unroll
      for (int i = 0; i < kCoItems; i++) {
        const bool in = first + i < n;
        pc[i] = in ? (uint32_t)code[first + i] : 0u;
        pk[i] = in ? src[first + i] : 0ull;
        c += __popc(pc[i]);
      }
      uint32_t tot;
      int64_t at = run + block_excl_scan<kCoThreads>(c, &tot, sm);
#pragma unroll
      for (int i = 0; i < kCoItems; i++) {
        if (!pc[i]) continue;
        // the children of the set bits, lowest first; the capacity is
        // checked once per parent
        const uint64_t k = pk[i];
        uint32_t m = pc[i];
        if (at + __popc(m) > cap) {
          set_error(err, kErrCapacity);
          for (; m && at < cap; m &= m - 1) dst[at++] = child_key(k, (uint32_t)(__ffs(m) - 1));
          continue;
        }
        for (; m; m &= m - 1) dst[at++] = child_key(k, (uint32_t)(__ffs(m) - 1));
      }
      run += tot;
    }
    if (h == 7 && threadIdx.x == 0) *n6 = run < cap ? run : cap;
    src = dst;
    __syncthreads();
  }
}

constexpr int64_t kCoarseScanMin = 16384;  // parents per height worth a multi-block scan

void launch_coarse_down(const uint64_t* roots, int top, const uint8_t* codes, int64_t stride,
                        const int64_t* counts, const int64_t* d_counts, int64_t cap, uint64_t* k0,
                        uint64_t* k1, uint64_t* key6, int64_t* n6, const ScanScratch& s, int* err,
                        cudaStream_t st) {
  if (top < 7) return;
  CoarseCounts c{};
  for (int h = 7; h <= top && h <= kMaxDepth; h++) c.n[h] = counts[h];
  // levels grow downward: parent heights bottom - 1 .. 7 are large enough for
  // the multi-block expansion, the ones above go through the single block
  int bottom = 7;
  while (bottom <= top && counts[bottom] >= kCoarseScanMin) bottom++;
  if (bottom <= top) {
    k_coarse_down<<<1, kCoThreads, 0, st>>>(roots, top, bottom, codes, stride, c, cap, k0, k1,
                                            key6, n6, err);
    count_launches(1);
  }
  for (int h = std::min(bottom - 1, top); h >= 7; h--) {
    const uint64_t* pk = h == top ? roots : ((h & 1) ? k1 : k0);
    uint64_t* ck = h == 7 ? key6 : (((h - 1) & 1) ? k1 : k0);
    // d_counts[h - 1] holds the child count already; the expansion rewrites it
    launch_expand(pk, codes + (int64_t)(h - 7) * stride, d_counts + h, counts[h], ck, nullptr,
                  nullptr, cap, h == 7 ? n6 : const_cast<int64_t*>(d_counts) + h - 1, s, err, st);
  }
}

// Children (parent << 3 | c) for every set bit c in ascending order: parents
// are Morton-sorted, so the children are too (no reordering).
// Codes decoded on the device may be corrupt: children past the capacity of
// the child arrays are not written, the count is clamped and err is set.
struct ExpandOp {
  const uint64_t* pk;
  const uint8_t* pc;
  uint64_t* ck;
  uint32_t* cpar;
  uint32_t* poff;
  int64_t* nc;
  int* err;
  int64_t cap_c;
  __device__ uint32_t value(int64_t p) const { return __popc((uint32_t)pc[p]); }
  __device__ void emit(int64_t p, uint32_t ex, int64_t) const {
    const uint32_t code = pc[p];
    if (code == 0) set_error(err, kErrExpand);
    int64_t r = ex;
    if (poff) poff[p] = (uint32_t)(r < cap_c ? r : cap_c);
    for (int c = 0; c < 8; c++)
      if (code >> c & 1) {
        if (r >= cap_c) {
          set_error(err, kErrCapacity);
          break;
        }
        ck[r] = child_key(pk[p], (uint32_t)c);
        if (cpar) cpar[r] = (uint32_t)p;
        r++;
      }
  }
  __device__ void finish(uint32_t total, int64_t n) const {
    const int64_t t = (int64_t)total < cap_c ? (int64_t)total : cap_c;
    *nc = t;
    if (poff) poff[n] = (uint32_t)t;
  }
};

void launch_expand(const uint64_t* pkeys, const uint8_t* pcodes, const int64_t* d_np,
                   int64_t cap_p, uint64_t* ckeys, uint32_t* cpar, uint32_t* poff, int64_t cap_c,
                   int64_t* d_nc, const ScanScratch& s, int* err, cudaStream_t st) {
  run_scan(ExpandOp{pkeys, pcodes, ckeys, cpar, poff, d_nc, err, cap_c}, d_np, cap_p, s, st);
}

}  // namespace lpc
