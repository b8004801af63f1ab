// Allocation-free variant of the 3x3x3 kernel-map builder.
//
// Some callers cannot allocate device memory at the point where they need a
// kernel map: a real-time perception loop whose memory budget is fixed at
// start-up (cudaMalloc may synchronise the whole device and has no latency
// bound), code that runs while another component owns the CUDA allocator, or
// a runtime that forbids allocation after initialisation.  For them this
// entry point keeps its voxel hash table in one file-scope device array that
// exists for as long as the library is loaded, instead of allocating it per
// call like lpc_kernel_map does.
//
// The array is a fixed 2^19-slot table (8 MiB of 16-byte key and row slots,
// plus two control words), enough for 262,144 nodes at a load factor of at
// most 1/2.  This file is its own device module, and CUDA loads modules
// lazily by default: the array's 8 MiB is committed on a device when the
// first call there looks up its address, and that load may synchronise the
// device.  A caller that must not allocate later makes one call per device
// at start-up; from then on the device holds the array until the process
// exits, and no call allocates.  The address is cached per device index; a
// cudaDeviceReset (or anything else that replaces the device's primary
// context) makes the cached address stale, so this entry point must not be
// used across such a reset.  All calls share the one table: concurrent calls
// whose work overlaps on a GPU (different streams, or different host
// threads) race and must be serialised by the caller.  The table keeps the
// previous call's contents; each call clears the slots it uses and its
// control words before inserting.
#include <mutex>

#include "../../include/lpc_ops.h"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int64_t kSlots = int64_t(1) << 19;
constexpr int64_t kMaxNodes = kSlots / 2;
constexpr size_t kSlotBytes = 16 * kSlots;
constexpr size_t kCtlBytes = 256;  // node count (int64) and error word (int)

__device__ __align__(256) unsigned char g_static_table[kSlotBytes + kCtlBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of the table on the current device, looked up once per
// device (host code cannot use the symbol itself as a device pointer).
int table_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LPC_CUDA_ERROR;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_table) != cudaSuccess || !p) {
      cudaGetLastError();
      return LPC_CUDA_ERROR;
    }
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return LPC_OK;
}

}  // namespace

extern "C" int lpc_kernel_map_noalloc(const uint64_t* d_keys, int64_t N, int depth,
                                      int32_t* d_nbr, uint64_t stream) {
  if (N < 0 || depth < 0 || depth > lpc::kMaxDepth || (N > 0 && (!d_keys || !d_nbr)))
    return LPC_INVALID_ARG;
  if (N > kMaxNodes) return LPC_CAPACITY;
  if (N == 0) return LPC_OK;
  unsigned char* base = nullptr;
  if (int s = table_address(&base)) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  lpc::HashTable h;
  h.slots = reinterpret_cast<ulonglong2*>(base);
  h.cap = kSlots;
  int64_t* d_n = reinterpret_cast<int64_t*>(base + kSlotBytes);
  int* d_err = reinterpret_cast<int*>(base + kSlotBytes + 8);
  int64_t slots = 1024;
  while (slots < 2 * N) slots <<= 1;
  const int64_t n_host = N;
  cudaMemcpyAsync(d_n, &n_host, sizeof(n_host), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(d_err, 0, sizeof(int), st);
  lpc::launch_kernel_map(d_keys, d_n, N, nullptr, depth, h, slots, d_nbr, d_err, st);
  int e = 0;
  cudaMemcpyAsync(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return LPC_CUDA_ERROR;
  if (e == lpc::kErrHashFull) return LPC_HASH_FULL;
  return e ? LPC_CUDA_ERROR : LPC_OK;
}
