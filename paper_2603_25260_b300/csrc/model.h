// Weight blob of the integer network: parsed, validated and uploaded once
// into the device layouts the kernels read (kernels.h).
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "kernels.h"

namespace lpc {

constexpr int kRelLevels = 5;  // network-coded levels b .. L-1 (b = L-5)

// Network architectures: the paper's model and its two ablations (Sec. 4.3).
enum Arch { kArchXfp = 0, kArchGred = 1, kArchBase = 2 };

struct BlobRecord {
  int kind, S, cin, cout, z_in, z_in2, z_out, shift, prelu;
  const int8_t* W = nullptr;
  const int32_t* bias = nullptr;
  const int32_t* mult = nullptr;
  const int16_t* slope = nullptr;
};

struct Model {
  int C = 0;
  int arch = kArchXfp;  // Arch
  int toff = 4;         // t = L - toff (4 or 3)
  // span[j]: m = d - k for a level whose features are extracted at level k
  // from X^{d-1} (re-densified when m > 1); 0 for levels that take the
  // propagated features of the level above (GRED + XFP down to t, and level b)
  int span[kRelLevels] = {};
  uint32_t lut[256];
  uint64_t hash = 0;
  std::vector<uint8_t> blob;          // owned copy (records point into it)
  std::vector<BlobRecord> recs;
  void* d_mem = nullptr;              // one device allocation for everything below
  const uint32_t* d_lut = nullptr;
  // Slots by relative level j = d - b (see the record order in the blob);
  // ESH/USH: level b's embedding and up-sampling, and those of the levels
  // b < d <= t that take propagated features
  DEmb ESH[kRelLevels]{}, G[kRelLevels]{}, E[kRelLevels][3]{};
  DLayer USH[kRelLevels]{}, UP[kRelLevels][3]{}, D[kRelLevels][3]{}, RA[kRelLevels]{},
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
