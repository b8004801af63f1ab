// Voxel hash table and 3x3x3 kernel map.  Sparse convolution is computed as
// indexed linear transforms over neighbour pairs (Sec. 3.3, following the
// MinkowskiEngine decomposition); the map holds, for every node and each of
// the 27 offsets, the row of the neighbour or -1.
//
// Table: open addressing with linear probing over 2^k slots (k chosen so the
// load factor is at most 1/2), u64 Morton key -> u32 row.  Probe sequences
// are bounded; a miss on the bound sets the HASH_FULL error word.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace lpc {

constexpr uint64_t kEmpty = ~0ull;
constexpr int kMaxProbe = 128;

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

__global__ void k_hash_clear(uint64_t* tk, int64_t slots) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < slots;
       i += (int64_t)gridDim.x * blockDim.x)
    tk[i] = kEmpty;
}

__global__ void k_hash_insert(const uint64_t* __restrict__ keys, const int64_t* d_n, uint64_t* tk,
                              uint32_t* tv, uint64_t mask, int* err) {
  const int64_t n = *d_n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    uint64_t s = mix64(k) & mask;
    int p = 0;
    for (; p < kMaxProbe; p++) {
      unsigned long long prev =
          atomicCAS((unsigned long long*)&tk[s], (unsigned long long)kEmpty,
                    (unsigned long long)k);
      if (prev == kEmpty || prev == k) {
        tv[s] = (uint32_t)i;
        break;
      }
      s = (s + 1) & mask;
    }
    if (p == kMaxProbe) set_error(err, kErrHashFull);
  }
}

// One thread per (node, offset); offset o = 9(dx+1) + 3(dy+1) + (dz+1).
// The depth of a node is Lf[frame] - h for a frame batch (Lf != nullptr),
// else h itself; neighbours keep the node's frame bits.
__global__ void k_kernel_map(const uint64_t* __restrict__ keys, const int64_t* d_n,
                             const int* __restrict__ Lf, int h,
                             const uint64_t* __restrict__ tk, const uint32_t* __restrict__ tv,
                             uint64_t mask, int32_t* nbr, int* err,
                             unsigned long long* pairs) {
  const int64_t n = *d_n;
  const int64_t total = n * 27;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / 27;
    const int o = (int)(t - i * 27);
    const uint64_t kf = keys[i];
    const uint64_t fbits = kf & ~kLowMask;
    const uint64_t k = kf & kLowMask;
    const int depth = Lf ? Lf[kf >> kFrameShift] - h : h;
    const int32_t side = 1 << depth;
    const int32_t x = (int32_t)compact3(k >> 2) + o / 9 - 1;
    const int32_t y = (int32_t)compact3(k >> 1) + (o / 3) % 3 - 1;
    const int32_t z = (int32_t)compact3(k) + o % 3 - 1;
    int32_t r = -1;
    if (o == 13) {
      r = (int32_t)i;
    } else if (x >= 0 && y >= 0 && z >= 0 && x < side && y < side && z < side) {
      const uint64_t q = fbits | morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
      uint64_t s = mix64(q) & mask;
      int p = 0;
      for (; p < kMaxProbe; p++) {
        const uint64_t c = tk[s];
        if (c == q) {
          r = (int32_t)tv[s];
          break;
        }
        if (c == kEmpty) break;
        s = (s + 1) & mask;
      }
      if (p == kMaxProbe) set_error(err, kErrHashFull);
    }
    nbr[t] = r;
    if (pairs) {
      const unsigned am = __activemask();
      const unsigned bm = __ballot_sync(am, r >= 0);
      if ((threadIdx.x & 31) == __ffs(am) - 1) atomicAdd(pairs, (unsigned long long)__popc(bm));
    }
  }
}

void launch_kernel_map(const uint64_t* keys, const int64_t* d_n, int64_t n_host, const int* Lf,
                       int depth, const HashTable& h, int64_t slots, int32_t* nbr, int* err,
                       cudaStream_t st, uint64_t* pairs) {
  if (n_host <= 0) return;
  const uint64_t mask = (uint64_t)slots - 1;
  k_hash_clear<<<(int)std::min<int64_t>((slots + 255) / 256, 148 * 8), 256, 0, st>>>(h.keys,
                                                                                     slots);
  k_hash_insert<<<(int)std::min<int64_t>((n_host + 255) / 256, 148 * 8), 256, 0, st>>>(
      keys, d_n, h.keys, h.vals, mask, err);
  k_kernel_map<<<(int)std::min<int64_t>((n_host * 27 + 255) / 256, 148 * 16), 256, 0, st>>>(
      keys, d_n, Lf, depth, h.keys, h.vals, mask, nbr, err,
      reinterpret_cast<unsigned long long*>(pairs));
  count_launches(3);
}

}  // namespace lpc
