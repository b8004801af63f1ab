// Weight blob parsing and upload.  Record order (per relative level j):
//   j=0: E_0, UP_0, P1_0, P2_0
//   j=1: RA_1, RB_1, RM_1, E_1, UP_1, P1_1, P2_1
//   j=2..4 (m = j-1): G_j, D_{j,1..m-1}, RA_j, RB_j, RM_j, (E_{j,k}, UP_{j,k}) k=0..m-1, P1_j, P2_j
#include "model.h"

#include <cuda_runtime.h>
#include <string.h>

#include "../../include/lpc.h"
#include "common.cuh"

namespace lpc {

enum { kSum = 1, kEmb = 2, kRes = 3, kSel = 4 };

uint64_t fnv1a64(const void* data, size_t len) {
  const uint8_t* p = static_cast<const uint8_t*>(data);
  uint64_t h = 0xcbf29ce484222325ull;
  for (size_t i = 0; i < len; i++) h = (h ^ p[i]) * 0x100000001b3ull;
  return h;
}

namespace {

int32_t le32(const uint8_t* p) {
  uint32_t v;
  memcpy(&v, p, 4);
  return (int32_t)v;
}
size_t up16(size_t n) { return (n + 15) / 16 * 16; }

// Device image builder: appends 256-byte aligned arrays to a host staging
// buffer and remembers the offsets for the pointer fix-up after upload.
struct Image {
  std::vector<uint8_t> host;
  size_t add(const void* src, size_t bytes) {
    size_t off = (host.size() + 255) / 256 * 256;
    host.resize(off + bytes);
    if (src) memcpy(host.data() + off, src, bytes);
    return off;
  }
};

struct LayerOffs {
  size_t W, wsum, bias, mult, slope, tc, mhi;
};

LayerOffs pack_layer(Image& img, const BlobRecord& r) {
  const int S = r.S, cin = r.cin, cout = r.cout, K4 = cin / 4;
  std::vector<int32_t> W((size_t)S * K4 * cout), ws((size_t)S * cout);
  for (int s = 0; s < S; s++)
    for (int co = 0; co < cout; co++) {
      const int8_t* w = r.W + ((size_t)s * cout + co) * cin;
      int32_t sum = 0;
      for (int ci = 0; ci < cin; ci++) sum += w[ci];
      ws[(size_t)s * cout + co] = sum;
      for (int k = 0; k < K4; k++) {
        uint32_t v = (uint32_t)(uint8_t)w[4 * k] | ((uint32_t)(uint8_t)w[4 * k + 1] << 8) |
                     ((uint32_t)(uint8_t)w[4 * k + 2] << 16) |
                     ((uint32_t)(uint8_t)w[4 * k + 3] << 24);
        W[((size_t)s * K4 + k) * cout + co] = (int32_t)v;
      }
    }
  const int P = r.kind == kSel ? S : 1;
  LayerOffs o;
  o.W = img.add(W.data(), W.size() * 4);
  o.wsum = img.add(ws.data(), ws.size() * 4);
  o.bias = img.add(r.bias, (size_t)P * cout * 4);
  o.mult = img.add(r.mult, (size_t)P * cout * 4);
  o.slope = img.add(r.slope, (size_t)P * cout * 2);
  o.tc = 0;
  // the multipliers in the high-word form of the requantisation, when every
  // one of the layer admits it (the kernels then take requant_hi)
  o.mhi = 0;
  bool all_hi = true;
  for (int i = 0; i < P * cout; i++) all_hi = all_hi && hi_ok(r.mult[i], r.shift);
  if (all_hi) {
    std::vector<int32_t> mh((size_t)P * cout);
    for (int i = 0; i < P * cout; i++) mh[i] = hi_scale(r.mult[i], r.shift);
    o.mhi = img.add(mh.data(), mh.size() * 4);
  }
  if (r.S == 27 && r.kind == kSum && cout == 32 && (cin == 32 || cin == 64)) {
    std::vector<uint16_t> tcimg(conv_tc_weight_bytes(cin) / 2);
    pack_conv_tc_weights(r.W, cin, tcimg.data());
    o.tc = img.add(tcimg.data(), tcimg.size() * 2);
  }
  if (r.S == 8 && r.kind == kSel && cout == 32 && (cin == 32 || cin == 64)) {  // up-steps
    std::vector<uint16_t> tcimg(up_tc_weight_bytes() / 2);
    pack_up_tc_weights(r.W, cin, tcimg.data());
    o.tc = img.add(tcimg.data(), tcimg.size() * 2);
  }
  if (r.S == 1 && r.kind == kSum && cout == 32 && cin == 32) {  // predictor layer 1
    std::vector<uint16_t> tcimg(32 * 32);
    pack_pred_tc_weights(r.W, 32, 32, tcimg.data());
    o.tc = img.add(tcimg.data(), tcimg.size() * 2);
  }
  return o;
}

}  // namespace

int model_load(const void* blob, size_t len, Model& M, std::string& err) {
  M = Model();
  const uint8_t* b = static_cast<const uint8_t*>(blob);
  if (!blob || len < 32 + 1024 || memcmp(b, "LPCW", 4) != 0 || le32(b + 4) != 1) {
    err = "weight blob: bad header";
    return LPC_INVALID_ARG;
  }
  M.blob.assign(b, b + len);
  b = M.blob.data();
  M.C = le32(b + 8);
  const int nrec = le32(b + 12);
  M.arch = le32(b + 20);
  M.toff = le32(b + 24) == 0 ? 4 : le32(b + 24);
  if (M.arch < kArchXfp || M.arch > kArchBase || (M.toff != 3 && M.toff != 4)) {
    err = "weight blob: unknown architecture or threshold offset";
    return LPC_INVALID_ARG;
  }
  if (M.C != 32) {
    err = "weight blob: this build supports C = 32 only";
    return LPC_INVALID_ARG;
  }
  if (le32(b + 16) != 256 || nrec < 1 || nrec > 64) {
    err = "weight blob: bad record count or table length";
    return LPC_INVALID_ARG;
  }
  for (int i = 0; i < 256; i++) M.lut[i] = (uint32_t)le32(b + 32 + 4 * i);
  if (M.lut[0] != (uint32_t)kFreqTotal) {
    err = "weight blob: exp table must start at 2^16";
    return LPC_INVALID_ARG;
  }
  for (int i = 1; i < 256; i++)
    if (M.lut[i] > M.lut[i - 1]) {
      err = "weight blob: exp table must be non-increasing";
      return LPC_INVALID_ARG;
    }
  size_t off = 32 + 1024;
  for (int i = 0; i < nrec; i++) {
    if (off + 48 > len) {
      err = "weight blob: truncated record header";
      return LPC_INVALID_ARG;
    }
    const uint8_t* h = b + off;
    BlobRecord r;
    r.kind = le32(h);
    r.S = le32(h + 4);
    r.cin = le32(h + 8);
    r.cout = le32(h + 12);
    r.z_in = le32(h + 16);
    r.z_in2 = le32(h + 20);
    r.z_out = le32(h + 24);
    r.shift = le32(h + 28);
    r.prelu = le32(h + 32) & 1;
    off += 48;
    auto zbad = [](int z) { return z < -128 || z > 127; };
    if (r.S < 1 || r.S > 27 || r.cin < 1 || r.cin > 256 || r.cout < 1 || r.cout > 256 ||
        zbad(r.z_in) || zbad(r.z_in2) || zbad(r.z_out)) {
      err = "weight blob: record field out of range";
      return LPC_INVALID_ARG;
    }
    if (r.kind == kSum || r.kind == kSel) {
      const size_t nw = (size_t)r.S * r.cout * r.cin;
      const size_t np = (size_t)(r.kind == kSel ? r.S : 1) * r.cout;
      if (off + up16(nw) + 2 * up16(4 * np) + up16(2 * np) > len) {
        err = "weight blob: truncated layer";
        return LPC_INVALID_ARG;
      }
      r.W = reinterpret_cast<const int8_t*>(b + off);
      off += up16(nw);
      r.bias = reinterpret_cast<const int32_t*>(b + off);
      off += up16(4 * np);
      r.mult = reinterpret_cast<const int32_t*>(b + off);
      off += up16(4 * np);
      r.slope = reinterpret_cast<const int16_t*>(b + off);
      off += up16(2 * np);
      if (r.shift < 1 || r.shift > 62) {
        err = "weight blob: shift out of range";
        return LPC_INVALID_ARG;
      }
      for (size_t k = 0; k < nw; k++)
        if (r.W[k] == -128) {
          err = "weight blob: weight -128 (weights must be symmetric)";
          return LPC_INVALID_ARG;
        }
      for (size_t k = 0; k < np; k++)
        if (r.bias[k] >= (1 << 30) || r.bias[k] <= -(1 << 30) || r.mult[k] < 0) {
          err = "weight blob: bias or multiplier out of range";
          return LPC_INVALID_ARG;
        }
    } else if (r.kind == kEmb) {
      if (r.S != 1 || r.cin != 256 || off + up16((size_t)256 * r.cout) > len) {
        err = "weight blob: bad embedding";
        return LPC_INVALID_ARG;
      }
      r.W = reinterpret_cast<const int8_t*>(b + off);
      off += up16((size_t)256 * r.cout);
    } else if (r.kind == kRes) {
      if (r.S != 2 || r.cin != r.cout ||
          off + up16((size_t)8 * r.cout) + up16((size_t)2 * r.cout) > len) {
        err = "weight blob: bad residual record";
        return LPC_INVALID_ARG;
      }
      r.mult = reinterpret_cast<const int32_t*>(b + off);
      off += up16((size_t)8 * r.cout);
      r.slope = reinterpret_cast<const int16_t*>(b + off);
      off += up16((size_t)2 * r.cout);
      if (r.shift < 1 || r.shift > 30) {
        err = "weight blob: residual shift out of range";
        return LPC_INVALID_ARG;
      }
      for (int k = 0; k < 2 * r.cout; k++)
        if (r.mult[k] < 0 || r.mult[k] >= (1 << 16)) {
          err = "weight blob: residual multiplier out of range";
          return LPC_INVALID_ARG;
        }
    } else {
      err = "weight blob: unknown record kind";
      return LPC_INVALID_ARG;
    }
    M.recs.push_back(r);
  }
  if (off != len) {
    err = "weight blob: trailing bytes";
    return LPC_INVALID_ARG;
  }
  M.hash = fnv1a64(b, len);

  // ---- bind records to network slots and build the device image ----
  const int C = M.C;
  Image img;
  size_t lut_off = img.add(M.lut, sizeof(M.lut));
  struct Fix {
    void* slot;
    int what;  // 0 emb, 1 layer, 2 res, 3 pred2
    size_t o[7];
  };
  std::vector<Fix> fixes;
  size_t ri = 0;
  bool ok = true;
  auto next = [&](int kind, int S, int cin, int cout, int prelu) -> const BlobRecord* {
    if (ri >= M.recs.size()) {
      ok = false;
      return nullptr;
    }
    const BlobRecord& r = M.recs[ri++];
    if (r.kind != kind || r.S != S || r.cin != cin || r.cout != cout || r.prelu != prelu) ok = false;
    return ok ? &r : nullptr;
  };
  auto emb = [&](DEmb& d) {
    const BlobRecord* r = next(kEmb, 1, 256, C, 0);
    if (!r) return;
    d.cout = C;
    d.z_out = r->z_out;
    fixes.push_back({&d, 0, {img.add(r->W, (size_t)256 * C), 0, 0, 0, 0}});
  };
  auto layer = [&](DLayer& d, int kind, int S, int cin, int prelu) {
    const BlobRecord* r = next(kind, S, cin, C, prelu);
    if (!r) return;
    d.S = S;
    d.cin = cin;
    d.cout = C;
    d.z_in = r->z_in;
    d.z_out = r->z_out;
    d.shift = r->shift;
    d.prelu = r->prelu;
    d.per_slice = kind == kSel;
    LayerOffs o = pack_layer(img, *r);
    fixes.push_back({&d, 1, {o.W, o.wsum, o.bias, o.mult, o.slope, o.tc, o.mhi}});
  };
  auto resm = [&](DRes& d) {
    const BlobRecord* r = next(kRes, 2, C, C, 1);
    if (!r) return;
    d.z1 = r->z_in;
    d.z2 = r->z_in2;
    d.z_out = r->z_out;
    d.shift = r->shift;
    fixes.push_back({&d, 2, {img.add(r->mult, (size_t)8 * C), img.add(r->slope, (size_t)2 * C), 0,
                             0, 0}});
  };
  auto pred2 = [&](DPred2& d) {
    const BlobRecord* r = next(kSum, 1, C, kNsym, 0);
    if (!r) return;
    d.z_in = r->z_in;
    d.z_out = r->z_out;
    d.shift = r->shift;
    const int K4 = C / 4;
    std::vector<int32_t> W((size_t)8 * K4 * 32, 0), ws(256, 0), bi(256, 0), mu(256, 0);
    for (int s = 0; s < kNsym; s++) {
      const int lane = s / 8, i = s % 8;
      const int8_t* w = r->W + (size_t)s * C;
      int32_t sum = 0;
      for (int ci = 0; ci < C; ci++) sum += w[ci];
      ws[s] = sum;
      bi[s] = r->bias[s];
      mu[s] = r->mult[s];
      for (int k = 0; k < K4; k++) {
        uint32_t v = (uint32_t)(uint8_t)w[4 * k] | ((uint32_t)(uint8_t)w[4 * k + 1] << 8) |
                     ((uint32_t)(uint8_t)w[4 * k + 2] << 16) |
                     ((uint32_t)(uint8_t)w[4 * k + 3] << 24);
        W[((size_t)i * K4 + k) * 32 + lane] = (int32_t)v;
      }
    }
    std::vector<uint16_t> tcimg(256 * 32);
    pack_pred_tc_weights(r->W, kNsym, 256, tcimg.data());
    fixes.push_back({&d, 3, {img.add(W.data(), W.size() * 4), img.add(ws.data(), 1024),
                             img.add(bi.data(), 1024), img.add(mu.data(), 1024),
                             img.add(tcimg.data(), tcimg.size() * 2)}});
  };

  // level b: features from Y_{b-1} alone, every architecture
  emb(M.ESH[0]);
  layer(M.USH[0], kSel, 8, C, 1);
  layer(M.P1[0], kSum, 1, C, 1);
  pred2(M.P2[0]);
  const int nsh = 5 - M.toff;  // relative levels 1..nsh lie at or above t
  for (int j = 1; j < kRelLevels; j++) {
    if (M.arch == kArchXfp && j <= nsh) {
      // S^{d-1} = ResBlock(F^{d-1}); F^d = Up(Concat(S^{d-1}, Y_{d-1})) (Eq. 8-9)
      M.span[j] = 0;
      layer(M.RA[j], kSum, 27, C, 1);
      layer(M.RB[j], kSum, 27, C, 0);
      resm(M.RM[j]);
      emb(M.ESH[j]);
      layer(M.USH[j], kSel, 8, 2 * C, 1);
    } else {
      // GRED + XFP below t: re-densified to t and fused with F^t (Eq. 10-11);
      // the ablations: features of Y_{d-1} alone, extracted at k = t for
      // GRED's levels below t (Eq. 4-6), at k = d - 1 otherwise
      const int below = j - nsh;
      const int m = (M.arch == kArchXfp || (M.arch == kArchGred && below > 0)) ? below : 1;
      const int cat = M.arch == kArchXfp ? 2 : 1;
      M.span[j] = m;
      emb(M.G[j]);
      for (int k = 1; k < m; k++) layer(M.D[j][k], kSum, 8, C, 1);
      layer(M.RA[j], kSum, 27, cat * C, 1);
      layer(M.RB[j], kSum, 27, C, 0);
      resm(M.RM[j]);
      for (int k = 0; k < m; k++) {
        if (cat == 2) emb(M.E[j][k]);
        layer(M.UP[j][k], kSel, 8, cat * C, 1);
      }
    }
    layer(M.P1[j], kSum, 1, C, 1);
    pred2(M.P2[j]);
  }
  if (!ok || ri != M.recs.size()) {
    err = "weight blob: records do not match the network structure";
    return LPC_INVALID_ARG;
  }
  if (cudaMalloc(&M.d_mem, img.host.size()) != cudaSuccess ||
      cudaMemcpy(M.d_mem, img.host.data(), img.host.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    err = "weight blob: device upload failed";
    if (M.d_mem) cudaFree(M.d_mem);
    M.d_mem = nullptr;
    return LPC_CUDA_ERROR;
  }
  uint8_t* base = static_cast<uint8_t*>(M.d_mem);
  M.d_lut = reinterpret_cast<const uint32_t*>(base + lut_off);
  for (const Fix& f : fixes) {
    if (f.what == 0) {
      static_cast<DEmb*>(f.slot)->table = reinterpret_cast<const int8_t*>(base + f.o[0]);
    } else if (f.what == 1) {
      DLayer* d = static_cast<DLayer*>(f.slot);
      d->Wp = reinterpret_cast<const int32_t*>(base + f.o[0]);
      d->wsum = reinterpret_cast<const int32_t*>(base + f.o[1]);
      d->bias = reinterpret_cast<const int32_t*>(base + f.o[2]);
      d->mult = reinterpret_cast<const int32_t*>(base + f.o[3]);
      d->slope = reinterpret_cast<const int16_t*>(base + f.o[4]);
      d->Wtc = f.o[5] ? reinterpret_cast<const uint16_t*>(base + f.o[5]) : nullptr;
      d->mult_hi = f.o[6] ? reinterpret_cast<const int32_t*>(base + f.o[6]) : nullptr;
    } else if (f.what == 2) {
      DRes* d = static_cast<DRes*>(f.slot);
      d->mab = reinterpret_cast<const int32_t*>(base + f.o[0]);
      d->slope = reinterpret_cast<const int16_t*>(base + f.o[1]);
    } else {
      DPred2* d = static_cast<DPred2*>(f.slot);
      d->Wp = reinterpret_cast<const int32_t*>(base + f.o[0]);
      d->wsum = reinterpret_cast<const int32_t*>(base + f.o[1]);
      d->bias = reinterpret_cast<const int32_t*>(base + f.o[2]);
      d->mult = reinterpret_cast<const int32_t*>(base + f.o[3]);
      d->Wtc = reinterpret_cast<const uint16_t*>(base + f.o[4]);
    }
  }
  return LPC_OK;
}

int upload_layer(const BlobRecord& r, DLayer& d, void** dmem) {
  Image img;
  LayerOffs o = pack_layer(img, r);
  *dmem = nullptr;
  if (cudaMalloc(dmem, img.host.size()) != cudaSuccess ||
      cudaMemcpy(*dmem, img.host.data(), img.host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return LPC_CUDA_ERROR;
  uint8_t* base = static_cast<uint8_t*>(*dmem);
  d.S = r.S;
  d.cin = r.cin;
  d.cout = r.cout;
  d.z_in = r.z_in;
  d.z_out = r.z_out;
  d.shift = r.shift;
  d.prelu = r.prelu;
  d.per_slice = r.kind == kSel;
  d.Wp = reinterpret_cast<const int32_t*>(base + o.W);
  d.wsum = reinterpret_cast<const int32_t*>(base + o.wsum);
  d.bias = reinterpret_cast<const int32_t*>(base + o.bias);
  d.mult = reinterpret_cast<const int32_t*>(base + o.mult);
  d.slope = reinterpret_cast<const int16_t*>(base + o.slope);
  d.Wtc = o.tc ? reinterpret_cast<const uint16_t*>(base + o.tc) : nullptr;
  d.mult_hi = o.mhi ? reinterpret_cast<const int32_t*>(base + o.mhi) : nullptr;
  return LPC_OK;
}

void model_free(Model& M) {
  if (M.d_mem) cudaFree(M.d_mem);
  M.d_mem = nullptr;
}

}  // namespace lpc
