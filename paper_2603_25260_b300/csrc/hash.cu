// Voxel hash table and 3x3x3 kernel map.  Sparse convolution is computed as
// indexed linear transforms over neighbour pairs (Sec. 3.3, following the
// MinkowskiEngine decomposition); the map holds, for every node and each of
// the 27 offsets, the row of the neighbour or -1.
//
// Table: open addressing with linear probing over 2^k slots (k chosen so the
// load factor is at most 1/2).  A slot is 16 bytes, the u64 key (frame bits
// and Morton key) and the u32 row side by side, so a probe is one 16-byte
// load.  The home slot is the top k bits of key * 2^64 / phi (Fibonacci
// hashing: one 64-bit multiply; consecutive Morton keys land far apart).
// Probe sequences are bounded; a miss on the bound sets the HASH_FULL error.
//
// Neighbour keys are formed in Morton space: the x bits of a key are the
// bits 3i + 2, and x + 1 is the carry chain of ((key | ~xmask) + 1) & xmask
// (the bits outside the x field are set so the carry runs through them),
// x - 1 is ((key & xmask) - 1) & xmask; the field being all ones (or zero)
// means the neighbour falls outside the cube.
//
// A second builder derives the map of a level from its parents' map (the
// octree neighbour rule): the neighbour of child slot (bx, by, bz) at
// offset (dx, dy, dz) lies in the parent's neighbour at offset
// floor((b + d) / 2) per axis, as its child ((b + d) & 1); its row is that
// parent's first child row plus the number of occupied slots below it.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace lpc {

constexpr uint64_t kEmpty = ~0ull;
constexpr int kMaxProbe = 128;
constexpr uint64_t kFib = 0x9E3779B97F4A7C15ull;  // 2^64 / golden ratio
constexpr uint64_t kXBits = 0x4924924924924924ull;  // bit 3i + 2 for i < 21

__device__ __forceinline__ uint64_t home_slot(uint64_t k, int shift) { return (k * kFib) >> shift; }

__global__ void k_hash_clear(ulonglong2* tab, int64_t slots) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < slots;
       i += (int64_t)gridDim.x * blockDim.x)
    tab[i] = make_ulonglong2(kEmpty, 0);
}

__global__ void k_hash_insert(const uint64_t* __restrict__ keys, const int64_t* d_n,
                              ulonglong2* tab, uint64_t mask, int shift, int* err) {
  const int64_t n = *d_n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    uint64_t s = home_slot(k, shift);
    int p = 0;
    for (; p < kMaxProbe; p++) {
      unsigned long long prev = atomicCAS(&tab[s].x, (unsigned long long)kEmpty,
                                          (unsigned long long)k);
      if (prev == kEmpty || prev == k) {
        tab[s].y = (unsigned long long)(uint32_t)i;
        break;
      }
      s = (s + 1) & mask;
    }
    if (p == kMaxProbe) set_error(err, kErrHashFull);
  }
}

// Morton-space step of one axis field: d in {-1, 0, 1}; false if the
// neighbour coordinate leaves [0, 2^depth).
__device__ __forceinline__ bool step_axis(uint64_t k, uint64_t m, int d, uint64_t& out) {
  const uint64_t f = k & m;
  if (d > 0) {
    if (f == m) return false;
    out = ((k | ~m) + 1) & m;
  } else if (d < 0) {
    if (f == 0) return false;
    out = (f - 1) & m;
  } else {
    out = f;
  }
  return true;
}

// Add the present (node, neighbour) pairs a warp counted (each thread over
// its grid-stride loop) to the launch's count: one atomic per warp, called
// by every thread of the warp after its loop.
__device__ __forceinline__ void count_pairs(unsigned long long* pairs, uint32_t mine) {
  const uint32_t w = __reduce_add_sync(0xffffffffu, mine);
  if ((threadIdx.x & 31) == 0 && w) atomicAdd(pairs, (unsigned long long)w);
}

// OR bit 1 << o of a present (node i, offset o) pair into the present-offset
// mask of i's tile of kConvTile nodes.  A warp's 32 consecutive pairs span
// at most three nodes, so nearly always one tile (one OR reduction and one
// atomic), at a tile boundary two (one reduction and atomic each).
__device__ __forceinline__ void tile_mask_or(uint32_t* tmask, int64_t i, int o, bool present) {
  const unsigned am = __activemask();
  const int leader = __ffs(am) - 1;
  const uint32_t tile = (uint32_t)(i / kConvTile);
  const uint32_t t0 = __shfl_sync(am, tile, leader);  // the lowest tile: pairs ascend by lane
  const uint32_t bit = present ? 1u << o : 0u;
  if (__all_sync(am, tile == t0)) {
    const uint32_t a = __reduce_or_sync(am, bit);
    if ((int)(threadIdx.x & 31) == leader && a) atomicOr(tmask + t0, a);
  } else {
    const uint32_t a = __reduce_or_sync(am, tile == t0 ? bit : 0u);
    const uint32_t b = __reduce_or_sync(am, tile != t0 ? bit : 0u);
    if ((int)(threadIdx.x & 31) == leader) {
      if (a) atomicOr(tmask + t0, a);
      if (b) atomicOr(tmask + t0 + 1, b);
    }
  }
}

// One thread per (node, offset); offset o = 9(dx+1) + 3(dy+1) + (dz+1).
// The depth of a node is Lf[frame] - h for a frame batch (Lf != nullptr),
// else h itself; neighbours keep the node's frame bits.  IdxT is 32-bit
// when N * 27 fits (cheap division by 27).
template <typename IdxT>
__global__ void k_kernel_map(const uint64_t* __restrict__ keys, const int64_t* d_n,
                             const int* __restrict__ Lf, int h,
                             const ulonglong2* __restrict__ tab, uint64_t mask, int shift,
                             int32_t* nbr, int* err, unsigned long long* pairs, uint32_t* tmask) {
  const IdxT total = (IdxT)(*d_n * 27);
  uint32_t npair = 0;
  for (IdxT t = blockIdx.x * (IdxT)blockDim.x + threadIdx.x; t < total;
       t += (IdxT)gridDim.x * blockDim.x) {
    const IdxT i = t / 27;
    const int o = (int)(t - i * 27);
    const uint64_t kf = keys[i];
    int32_t r = -1;
    if (o == 13) {
      r = (int32_t)i;
    } else {
      const int depth = Lf ? Lf[kf >> kFrameShift] - h : h;
      const uint64_t xm = kXBits & ((1ull << (3 * depth)) - 1);
      uint64_t nx, ny, nz;
      if (step_axis(kf, xm, o / 9 - 1, nx) && step_axis(kf, xm >> 1, (o / 3) % 3 - 1, ny) &&
          step_axis(kf, xm >> 2, o % 3 - 1, nz)) {
        const uint64_t q = (Lf ? kf & ~kLowMask : 0ull) | nx | ny | nz;
        uint64_t s = home_slot(q, shift);
        int p = 0;
        for (; p < kMaxProbe; p++) {
          const ulonglong2 c = tab[s];
          if (c.x == q) {
            r = (int32_t)c.y;
            break;
          }
          if (c.x == kEmpty) break;
          s = (s + 1) & mask;
        }
        if (p == kMaxProbe) set_error(err, kErrHashFull);
      }
    }
    nbr[t] = r;
    npair += r >= 0;
    if (tmask) tile_mask_or(tmask, (int64_t)i, o, r >= 0);
  }
  if (pairs) count_pairs(pairs, npair);
}

// Child map from the parent map: children at one height, their parent rows
// cpar, the parents' 27-neighbour map pnbr, occupancy codes pcode and first
// child rows poff.  One thread per (child, offset).
template <typename IdxT>
__global__ void k_kernel_map_child(const uint64_t* __restrict__ ckeys,
                                   const uint32_t* __restrict__ cpar, const int64_t* d_n,
                                   const int32_t* __restrict__ pnbr,
                                   const uint8_t* __restrict__ pcode,
                                   const uint32_t* __restrict__ poff, int32_t* nbr,
                                   unsigned long long* pairs, uint32_t* tmask) {
  const IdxT total = (IdxT)(*d_n * 27);
  uint32_t npair = 0;
  for (IdxT t = blockIdx.x * (IdxT)blockDim.x + threadIdx.x; t < total;
       t += (IdxT)gridDim.x * blockDim.x) {
    const IdxT i = t / 27;
    const int o = (int)(t - i * 27);
    int32_t r = (int32_t)i;
    if (o != 13) {
      const int b = (int)(ckeys[i] & 7);
      const int vx = (b >> 2) + o / 9 - 1;  // -1 .. 2 per axis
      const int vy = ((b >> 1) & 1) + (o / 3) % 3 - 1;
      const int vz = (b & 1) + o % 3 - 1;
      const int po = 9 * ((vx >> 1) + 1) + 3 * ((vy >> 1) + 1) + ((vz >> 1) + 1);
      const int32_t q = __ldg(pnbr + (int64_t)__ldg(cpar + i) * 27 + po);
      r = -1;
      if (q >= 0) {
        const uint32_t m = __ldg(pcode + q);
        const int cs = ((vx & 1) << 2) | ((vy & 1) << 1) | (vz & 1);
        if (m >> cs & 1) r = (int32_t)(__ldg(poff + q) + __popc(m & ((1u << cs) - 1)));
      }
    }
    nbr[t] = r;
    npair += r >= 0;
    if (tmask) tile_mask_or(tmask, (int64_t)i, o, r >= 0);
  }
  if (pairs) count_pairs(pairs, npair);
}

namespace {
// per_sm: blocks of 256 threads a SM; 8 is one resident wave (2048 threads)
int grid_for(int64_t work, int per_sm) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 148 * per_sm));
}
// kernel maps: one resident wave while a thread has at most 16 items (one
// frame: ~5), two waves beyond (the 64-frame batch, ~250 items a thread,
// measured 5 % faster with them)
int map_blocks_per_sm(int64_t items) { return items <= (int64_t)148 * 2048 * 16 ? 8 : 16; }
}  // namespace

void launch_kernel_map(const uint64_t* keys, const int64_t* d_n, int64_t n_host, const int* Lf,
                       int depth, const HashTable& h, int64_t slots, int32_t* nbr, int* err,
                       cudaStream_t st, uint64_t* pairs, uint32_t* tmask) {
  if (n_host <= 0) return;
  if (tmask) cudaMemsetAsync(tmask, 0, 4 * (size_t)conv_tiles(n_host), st);
  const uint64_t mask = (uint64_t)slots - 1;
  int lg = 0;
  while (((int64_t)1 << lg) < slots) lg++;
  const int shift = 64 - lg;
  auto pc = reinterpret_cast<unsigned long long*>(pairs);
  k_hash_clear<<<grid_for(slots, 8), 256, 0, st>>>(h.slots, slots);
  k_hash_insert<<<grid_for(n_host, 8), 256, 0, st>>>(keys, d_n, h.slots, mask, shift, err);
  if (n_host * 27 < ((int64_t)1 << 31))
    k_kernel_map<uint32_t><<<grid_for(n_host * 27, map_blocks_per_sm(n_host * 27)), 256, 0, st>>>(
        keys, d_n, Lf, depth, h.slots, mask, shift, nbr, err, pc, tmask);
  else
    k_kernel_map<int64_t><<<grid_for(n_host * 27, map_blocks_per_sm(n_host * 27)), 256, 0, st>>>(
        keys, d_n, Lf, depth, h.slots, mask, shift, nbr, err, pc, tmask);
  count_launches(3);
}

void launch_kernel_map_child(const uint64_t* ckeys, const uint32_t* cpar, const int64_t* d_n,
                             int64_t n_host, const int32_t* pnbr, const uint8_t* pcode,
                             const uint32_t* poff, int32_t* nbr, cudaStream_t st,
                             uint64_t* pairs, uint32_t* tmask) {
  if (n_host <= 0) return;
  if (tmask) cudaMemsetAsync(tmask, 0, 4 * (size_t)conv_tiles(n_host), st);
  auto pc = reinterpret_cast<unsigned long long*>(pairs);
  if (n_host * 27 < ((int64_t)1 << 31))
    k_kernel_map_child<uint32_t><<<grid_for(n_host * 27, map_blocks_per_sm(n_host * 27)), 256, 0, st>>>(
        ckeys, cpar, d_n, pnbr, pcode, poff, nbr, pc, tmask);
  else
    k_kernel_map_child<int64_t><<<grid_for(n_host * 27, map_blocks_per_sm(n_host * 27)), 256, 0, st>>>(
        ckeys, cpar, d_n, pnbr, pcode, poff, nbr, pc, tmask);
  count_launches(1);
}

}  // namespace lpc
