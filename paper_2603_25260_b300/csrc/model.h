// Weight blob of the integer network: parsed, validated and uploaded once
// into the device layouts the kernels read (kernels.h).
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "kernels.h"

namespace lpc {

constexpr int kRelLevels = 5;  // network-coded levels b .. L-1 (b = L-5)

struct BlobRecord {
  int kind, S, cin, cout, z_in, z_in2, z_out, shift, prelu;
  const int8_t* W = nullptr;
  const int32_t* bias = nullptr;
  const int32_t* mult = nullptr;
  const int16_t* slope = nullptr;
};

struct Model {
  int C = 0;
  uint32_t lut[256];
  uint64_t hash = 0;
  std::vector<uint8_t> blob;          // owned copy (records point into it)
  std::vector<BlobRecord> recs;
  void* d_mem = nullptr;              // one device allocation for everything below
  const uint32_t* d_lut = nullptr;
  // Slots by relative level j = d - b (see the record order in the blob):
  DEmb E0{}, E1{}, G[kRelLevels]{}, E[kRelLevels][3]{};
  DLayer UP0{}, UP1{}, UP[kRelLevels][3]{}, D[kRelLevels][3]{}, RA[kRelLevels]{},
      RB[kRelLevels]{}, P1[kRelLevels]{};
  DRes RM[kRelLevels]{};
  DPred2 P2[kRelLevels]{};
};

// 64-bit FNV-1a of a byte string.
uint64_t fnv1a64(const void* data, size_t len);

// Parse + validate + upload.  Returns an LPC_* status; err gets a message.
int model_load(const void* blob, size_t len, Model& M, std::string& err);
void model_free(Model& M);

// Upload one kind-1 or kind-4 record (cout = 32) into its own device
// allocation *dmem (freed by the caller); used by the op-level entry points.
int upload_layer(const BlobRecord& r, DLayer& out, void** dmem);

}  // namespace lpc
