/*
 * CPU oracle of the integer-only LiDAR geometry codec (arXiv 2603.25260).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.  Plain loops,
 * 64-bit integer arithmetic, binary search for every coordinate lookup, no
 * blocking or fusion.  Shares no source with the CUDA path.
 *
 * Where the paper is silent the oracle takes these readings (all integer):
 *  - depth d in [0, L]; Y_d (the paper's X^d) is the 8-bit child mask of each
 *    depth-d node; child index c = 4*xbit + 2*ybit + zbit (x-major Morton);
 *  - coded alphabet: symbol = code - 1 in 0..254 (Sec. 3.1, 255 classes);
 *  - base level b = L-5 (levels below are coded with adaptive symbol
 *    frequencies, supplement "Detailed Model Structure"), threshold t = L-4
 *    or L-3 (supplement, "Ablation on the Choice of t"), dense level k = t;
 *  - ablations (Sec. 4.3): without XFP a level d > b takes no feature from
 *    the level above, only G^k = Downsampling(X^{d-1}) with Eq. 5-6 as
 *    printed, k = t below t (GRED) and k = d-1 otherwise (and for every
 *    level in the baseline); level b is the same in all architectures;
 *  - requantisation: round half up, floor shift, clip to [-128, 127] (Eq. 14);
 *  - PReLU on the INT32 accumulator before requantisation, Q15 slope;
 *  - absent neighbours / children contribute zero (zero padding, Sec. 3.1);
 *  - ResBlock: y1 = rq(prelu(conv_a x)), y2 = rq(conv_b y1),
 *    out = rq'(prelu((y1-z1) ma + (y2-z2) mb)) with rq' a pure shift;
 *  - Downsampling(X^{l-1}) = embedding of the codes, then stride-2 convs;
 *  - H^k for k > t in Eq. 11 is the previous up-step's output;
 *  - softmax: exp table over the non-positive domain, 16-bit frequencies with
 *    floor 1, remainder to the lowest-index maximum (Eq. 15);
 *  - range coder with 32-bit range and byte-wise carry propagation.
 */
#include "lpc_oracle.h"

#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;
void or_set_threads(int n) { g_threads = n < 1 ? 1 : n; }

/* Wall time of the last or_encode / or_decode on the calling thread, split
 * into the network with its softmax tables and the range coding (for the
 * CPU baseline's breakdown; no effect on any result). */
static _Thread_local double g_t_net, g_t_code;
static double now_s(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}
void or_last_phase_times(double* network_s, double* coding_s) {
  *network_s = g_t_net;
  *coding_s = g_t_code;
}
int or_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------------ */
/* Integer primitives (Eq. 13, Eq. 14)                                       */
/* ------------------------------------------------------------------------ */

/* floor(v / 2^r) for r in [0, 62] */
static int64_t floor_shift(int64_t v, int r) {
  int64_t d = (int64_t)1 << r;
  if (v >= 0) return v / d;
  return -((-v + d - 1) / d);
}

int or_requant(int64_t acc, int32_t m, int r, int z) {
  int64_t p = acc * (int64_t)m;
  int64_t q = floor_shift(p + ((int64_t)1 << (r - 1)), r) + z;
  if (q < -128) q = -128;
  if (q > 127) q = 127;
  return (int)q;
}

int64_t or_prelu(int64_t acc, int a) {
  if (acc >= 0) return acc;
  return floor_shift(acc * (int64_t)a + (1 << 14), 15);
}

/* ------------------------------------------------------------------------ */
/* Morton keys and the octree (supplement, Implementation of Octree Ops)     */
/* ------------------------------------------------------------------------ */

uint64_t or_morton(uint32_t x, uint32_t y, uint32_t z, int bits) {
  uint64_t k = 0;
  for (int i = 0; i < bits; i++) {
    k |= (uint64_t)((x >> i) & 1) << (3 * i + 2);
    k |= (uint64_t)((y >> i) & 1) << (3 * i + 1);
    k |= (uint64_t)((z >> i) & 1) << (3 * i);
  }
  return k;
}

static void morton_decode(uint64_t k, int bits, int64_t* x, int64_t* y, int64_t* z) {
  *x = *y = *z = 0;
  for (int i = 0; i < bits; i++) {
    *x |= (int64_t)((k >> (3 * i + 2)) & 1) << i;
    *y |= (int64_t)((k >> (3 * i + 1)) & 1) << i;
    *z |= (int64_t)((k >> (3 * i)) & 1) << i;
  }
}

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* index of key in sorted keys[0..n), or -1 */
static int64_t find_key(const uint64_t* keys, int64_t n, uint64_t key) {
  int64_t lo = 0, hi = n - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (keys[mid] == key) return mid;
    if (keys[mid] < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

int or_leaf_keys(const int32_t* xyz, int64_t n, int L, uint64_t* keys_out, int64_t* n_out) {
  if (L < 1 || L > 21 || n < 0) return OR_INVALID_ARG;
  for (int64_t i = 0; i < n; i++) {
    for (int a = 0; a < 3; a++)
      if (xyz[3 * i + a] < 0 || xyz[3 * i + a] >= (1 << L)) return OR_INVALID_ARG;
    keys_out[i] = or_morton((uint32_t)xyz[3 * i], (uint32_t)xyz[3 * i + 1],
                            (uint32_t)xyz[3 * i + 2], L);
  }
  qsort(keys_out, (size_t)n, sizeof(uint64_t), cmp_u64);
  int64_t u = 0;
  for (int64_t i = 0; i < n; i++)
    if (u == 0 || keys_out[u - 1] != keys_out[i]) keys_out[u++] = keys_out[i];
  *n_out = u;
  return OR_OK;
}

#define OR_MAXL 21
typedef struct {
  int L;
  int64_t N[OR_MAXL + 1];
  uint64_t* key[OR_MAXL + 1]; /* V_d, sorted */
  uint8_t* code[OR_MAXL + 1]; /* Y_d, d < L */
} octree;

static void octree_free(octree* T) {
  for (int d = 0; d <= OR_MAXL; d++) {
    free(T->key[d]);
    free(T->code[d]);
  }
  memset(T, 0, sizeof(*T));
}

/* Shallower levels by repeated floor-halving (>> 3 on the key) and removal
 * of consecutive duplicates; the code of a parent ORs 1 << (child & 7). */
static int octree_from_points(const int32_t* xyz, int64_t n, int L, octree* T) {
  memset(T, 0, sizeof(*T));
  T->L = L;
  uint64_t* leaf = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
  int64_t nl = 0;
  int st = or_leaf_keys(xyz, n, L, leaf, &nl);
  if (st) { free(leaf); return st; }
  T->key[L] = leaf;
  T->N[L] = nl;
  for (int d = L - 1; d >= 0; d--) {
    const uint64_t* ck = T->key[d + 1];
    int64_t nc = T->N[d + 1];
    uint64_t* pk = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nc > 0 ? nc : 1));
    uint8_t* cd = (uint8_t*)calloc((size_t)(nc > 0 ? nc : 1), 1);
    int64_t np = 0;
    for (int64_t i = 0; i < nc; i++) {
      uint64_t p = ck[i] >> 3;
      if (np == 0 || pk[np - 1] != p) pk[np++] = p;
      cd[np - 1] |= (uint8_t)(1u << (ck[i] & 7));
    }
    T->key[d] = pk;
    T->code[d] = cd;
    T->N[d] = np;
  }
  return OR_OK;
}

int or_build_levels(const int32_t* xyz, int64_t n, int L, int64_t* counts, uint64_t* keys_out,
                    uint8_t* codes_out, int64_t cap) {
  octree T;
  int st = octree_from_points(xyz, n, L, &T);
  if (st) return st;
  int64_t kp = 0, cp = 0;
  for (int d = 0; d <= L; d++) {
    counts[d] = T.N[d];
    if (kp + T.N[d] > cap) { octree_free(&T); return OR_CAPACITY; }
    memcpy(keys_out + kp, T.key[d], sizeof(uint64_t) * (size_t)T.N[d]);
    kp += T.N[d];
    if (d < L) {
      memcpy(codes_out + cp, T.code[d], (size_t)T.N[d]);
      cp += T.N[d];
    }
  }
  octree_free(&T);
  return OR_OK;
}

/* children of V_d in Morton order: (key << 3) | c for each set bit c,
 * ascending (the supplement's offset-matrix upsampling with masking) */
static int octree_expand(octree* T, int d) {
  int64_t np = T->N[d];
  int64_t nc = 0;
  for (int64_t p = 0; p < np; p++) nc += __builtin_popcount(T->code[d][p]);
  uint64_t* ck = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nc > 0 ? nc : 1));
  int64_t r = 0;
  for (int64_t p = 0; p < np; p++)
    for (int c = 0; c < 8; c++)
      if (T->code[d][p] & (1u << c)) ck[r++] = (T->key[d][p] << 3) | (uint64_t)c;
  for (int64_t i = 1; i < nc; i++)
    if (ck[i - 1] >= ck[i]) { free(ck); return OR_CORRUPT_STREAM; }
  free(T->key[d + 1]);
  T->key[d + 1] = ck;
  T->N[d + 1] = nc;
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Sparse layers                                                             */
/* ------------------------------------------------------------------------ */

static int8_t out_q(int64_t acc, int32_t m, int shift, const int16_t* slope, int c, int z_out) {
  if (slope) acc = or_prelu(acc, slope[c]);
  return (int8_t)or_requant(acc, m, shift, z_out);
}

int or_conv333(const uint64_t* keys, int64_t N, int depth, const int8_t* x, int cin, int z_in,
               const int8_t* W, const int32_t* bias, const int32_t* mult, int shift,
               const int16_t* slope, int z_out, int cout, int8_t* out) {
  const int64_t side = (int64_t)1 << depth;
#pragma omp parallel for schedule(dynamic, 256) num_threads(g_threads)
  for (int64_t n = 0; n < N; n++) {
    int64_t acc[256];
    int64_t px, py, pz;
    morton_decode(keys[n], depth, &px, &py, &pz);
    for (int co = 0; co < cout; co++) acc[co] = bias[co];
    for (int o = 0; o < 27; o++) {
      int64_t qx = px + (o / 9) - 1, qy = py + (o / 3) % 3 - 1, qz = pz + o % 3 - 1;
      if (qx < 0 || qy < 0 || qz < 0 || qx >= side || qy >= side || qz >= side) continue;
      int64_t nb = find_key(keys, N, or_morton((uint32_t)qx, (uint32_t)qy, (uint32_t)qz, depth));
      if (nb < 0) continue;
      for (int co = 0; co < cout; co++) {
        const int8_t* w = W + ((int64_t)o * cout + co) * cin;
        int64_t s = 0;
        for (int ci = 0; ci < cin; ci++) s += (int64_t)(x[nb * cin + ci] - z_in) * w[ci];
        acc[co] += s;
      }
    }
    for (int co = 0; co < cout; co++)
      out[n * cout + co] = out_q(acc[co], mult[co], shift, slope, co, z_out);
  }
  return OR_OK;
}

int or_down_s2(const uint64_t* ckeys, int64_t Nc, const uint64_t* pkeys, int64_t Np,
               const int8_t* x, int cin, int z_in, const int8_t* W, const int32_t* bias,
               const int32_t* mult, int shift, const int16_t* slope, int z_out, int cout,
               int8_t* out) {
#pragma omp parallel for schedule(dynamic, 256) num_threads(g_threads)
  for (int64_t p = 0; p < Np; p++) {
    int64_t acc[256];
    for (int co = 0; co < cout; co++) acc[co] = bias[co];
    for (int c = 0; c < 8; c++) {
      int64_t r = find_key(ckeys, Nc, (pkeys[p] << 3) | (uint64_t)c);
      if (r < 0) continue;
      for (int co = 0; co < cout; co++) {
        const int8_t* w = W + ((int64_t)c * cout + co) * cin;
        int64_t s = 0;
        for (int ci = 0; ci < cin; ci++) s += (int64_t)(x[r * cin + ci] - z_in) * w[ci];
        acc[co] += s;
      }
    }
    for (int co = 0; co < cout; co++)
      out[p * cout + co] = out_q(acc[co], mult[co], shift, slope, co, z_out);
  }
  return OR_OK;
}

int or_up_prune(const uint64_t* pkeys, const uint8_t* codes, int64_t Np, const uint64_t* ckeys,
                int64_t Nc, const int8_t* x, int cin, int z_in, const int8_t* W,
                const int32_t* bias, const int32_t* mult, int shift, const int16_t* slope,
                int z_out, int cout, int8_t* out) {
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 256) num_threads(g_threads) reduction(| : bad)
  for (int64_t p = 0; p < Np; p++) {
    for (int c = 0; c < 8; c++) {
      if (!(codes[p] & (1u << c))) continue;
      int64_t r = find_key(ckeys, Nc, (pkeys[p] << 3) | (uint64_t)c);
      if (r < 0) { bad = 1; continue; }
      for (int co = 0; co < cout; co++) {
        const int8_t* w = W + ((int64_t)c * cout + co) * cin;
        int64_t acc = bias[c * cout + co];
        for (int ci = 0; ci < cin; ci++) acc += (int64_t)(x[p * cin + ci] - z_in) * w[ci];
        out[r * cout + co] =
            out_q(acc, mult[c * cout + co], shift, slope ? slope + c * cout : NULL, co, z_out);
      }
    }
  }
  return bad ? OR_INVALID_ARG : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Integer softmax -> frequencies -> cumulative table (Eq. 15)               */
/* ------------------------------------------------------------------------ */

#define NSYM 255
#define FREQ_BITS 16
#define FREQ_TOTAL (1 << FREQ_BITS)

/* freq[255] of one logit row: e_i = lut[max - l_i]; S = sum e_i;
 * f_i = 1 + floor(e_i (2^16 - 255) / S); remainder to the first argmax. */
static void softmax_freq(const int8_t* l, const uint32_t* lut, uint32_t* f) {
  int mx = -129, am = 0;
  for (int i = 0; i < NSYM; i++)
    if (l[i] > mx) { mx = l[i]; am = i; }
  uint64_t S = 0;
  uint32_t e[NSYM];
  for (int i = 0; i < NSYM; i++) {
    e[i] = lut[mx - l[i]];
    S += e[i];
  }
  uint64_t tot = 0;
  for (int i = 0; i < NSYM; i++) {
    f[i] = 1 + (uint32_t)(((uint64_t)e[i] * (FREQ_TOTAL - NSYM)) / S);
    tot += f[i];
  }
  f[am] += (uint32_t)(FREQ_TOTAL - tot);
}

static void freq_to_row(const uint32_t* f, uint16_t* row) {
  uint32_t c = 0;
  for (int s = 0; s < 254; s++) {
    c += f[s];
    row[s] = (uint16_t)c; /* C_{s+1} <= 65535 since every f >= 1 */
  }
  row[254] = 0xFFFF;
  row[255] = 0xFFFF;
}

int or_softmax_cdf(const int8_t* logits, int64_t N, const uint32_t* lut, uint16_t* cdf) {
#pragma omp parallel for schedule(static) num_threads(g_threads)
  for (int64_t n = 0; n < N; n++) {
    uint32_t f[NSYM];
    softmax_freq(logits + n * NSYM, lut, f);
    freq_to_row(f, cdf + n * 256);
  }
  return OR_OK;
}

/* (C_s, f_s) of symbol s from a table row */
static void row_interval(const uint16_t* row, int s, uint32_t* lo, uint32_t* f) {
  uint32_t a = s == 0 ? 0 : row[s - 1];
  uint32_t b = s == 254 ? FREQ_TOTAL : row[s];
  *lo = a;
  *f = b - a;
}

/* ------------------------------------------------------------------------ */
/* Range coder: 32-bit range, low kept to 33 bits, carry propagated through  */
/* one cached byte and a run of pending 0xFF bytes (Martin 1979 range coding */
/* with the usual cache-byte carry scheme).                                  */
/* ------------------------------------------------------------------------ */

/* Stream version 3 (the paper leaves the entropy coder open): the byte the cache holds before the first
 * output is never written (it is always 0: every coded interval lies inside
 * the initial [0, 2^32), so no carry reaches it), the decoder starts from
 * the first four bytes, and the flush writes the value with the most
 * trailing zero bits inside the final interval, whose trailing zero bytes
 * (up to four) are left out: the decoder reads up to four bytes past a
 * substream's end as zero. */
#define RC_PAD 4

typedef struct {
  uint8_t* buf;
  size_t cap, len;
  int overflow;
  int skip; /* the leading cache byte is still to be dropped */
  uint64_t low;
  uint32_t range;
  uint8_t cache;
  uint64_t cache_size;
} rc_enc;

static void enc_put(rc_enc* e, uint8_t b) {
  if (e->skip) { e->skip = 0; return; }
  if (e->len < e->cap) e->buf[e->len] = b; else e->overflow = 1;
  e->len++;
}

static void enc_init(rc_enc* e, uint8_t* buf, size_t cap) {
  e->buf = buf; e->cap = cap; e->len = 0; e->overflow = 0; e->skip = 1;
  e->low = 0; e->range = 0xFFFFFFFFu; e->cache = 0; e->cache_size = 1;
}

static void enc_shift_low(rc_enc* e) {
  if ((uint32_t)e->low < 0xFF000000u || (e->low >> 32) != 0) {
    uint8_t carry = (uint8_t)(e->low >> 32);
    uint8_t b = e->cache;
    do {
      enc_put(e, (uint8_t)(b + carry));
      b = 0xFF;
    } while (--e->cache_size != 0);
    e->cache = (uint8_t)((e->low >> 24) & 0xFF);
  }
  e->cache_size++;
  e->low = (e->low & 0x00FFFFFFu) << 8;
}

static void enc_code(rc_enc* e, uint32_t r, uint32_t lo, uint32_t f) {
  e->low += (uint64_t)r * lo;
  e->range = r * f;
  while (e->range < (1u << 24)) {
    e->range <<= 8;
    enc_shift_low(e);
  }
}

static void enc_flush(rc_enc* e) {
  /* any value in [low, low + range) identifies the coded symbols: take the
   * multiple of 2^k in it with k largest (k >= 24 since range >= 2^24) */
  const uint64_t end = e->low + e->range;
  for (int k = 32; k > 0; k--) {
    const uint64_t v = ((e->low + (((uint64_t)1 << k) - 1)) >> k) << k;
    if (v < end) {
      e->low = v;
      break;
    }
  }
  for (int i = 0; i < 5; i++) enc_shift_low(e);
  for (int i = 0; i < RC_PAD && !e->overflow && e->len > 0 && e->buf[e->len - 1] == 0; i++)
    e->len--;
}

typedef struct {
  const uint8_t* buf;
  size_t len, pos;
  int bad;
  uint32_t range, code;
} rc_dec;

static uint8_t dec_get(rc_dec* d) {
  if (d->pos < d->len) return d->buf[d->pos++];
  /* past the end: the flush's dropped zero bytes, at most RC_PAD of them */
  if (++d->pos > d->len + RC_PAD) d->bad = 1;
  return 0;
}

static void dec_init(rc_dec* d, const uint8_t* buf, size_t len) {
  d->buf = buf; d->len = len; d->pos = 0; d->bad = 0;
  d->range = 0xFFFFFFFFu; d->code = 0;
  for (int i = 0; i < 4; i++) d->code = (d->code << 8) | dec_get(d);
}

static void dec_update(rc_dec* d, uint32_t r, uint32_t lo, uint32_t f) {
  d->code -= r * lo;
  d->range = r * f;
  if (d->code >= d->range) d->bad = 1;
  while (d->range < (1u << 24)) {
    d->code = (d->code << 8) | dec_get(d);
    d->range <<= 8;
  }
}

static void enc_symbol_row(rc_enc* e, const uint16_t* row, int s) {
  uint32_t lo, f;
  row_interval(row, s, &lo, &f);
  enc_code(e, e->range >> FREQ_BITS, lo, f);
}

static int dec_symbol_row(rc_dec* d, const uint16_t* row) {
  uint32_t r = d->range >> FREQ_BITS;
  uint32_t v = d->code / r;
  if (v > FREQ_TOTAL - 1) v = FREQ_TOTAL - 1;
  int s = 0; /* number of C_{i+1} <= v, i.e. the s with C_s <= v < C_{s+1} */
  while (s < 254 && row[s] <= v) s++;
  uint32_t lo, f;
  row_interval(row, s, &lo, &f);
  dec_update(d, r, lo, f);
  return s;
}

int or_rc_encode_cdf(const uint16_t* cdf, const uint8_t* syms, int64_t n, uint8_t* out,
                     size_t cap, size_t* out_len) {
  rc_enc e;
  enc_init(&e, out, cap);
  for (int64_t i = 0; i < n; i++) {
    if (syms[i] > 254) return OR_INVALID_ARG;
    enc_symbol_row(&e, cdf + i * 256, syms[i]);
  }
  enc_flush(&e);
  *out_len = e.len;
  return e.overflow ? OR_CAPACITY : OR_OK;
}

int or_rc_decode_cdf(const uint16_t* cdf, int64_t n, const uint8_t* in, size_t len,
                     uint8_t* syms) {
  rc_dec d;
  dec_init(&d, in, len);
  for (int64_t i = 0; i < n; i++) syms[i] = (uint8_t)dec_symbol_row(&d, cdf + i * 256);
  return d.bad ? OR_CORRUPT_STREAM : OR_OK;
}

/* Adaptive model of the coarse levels: 255 counts starting at 1, +32 per
 * coded symbol, all counts halved (rounding up) once the total exceeds 2^16. */
typedef struct {
  uint32_t f[NSYM];
  uint32_t total;
} amodel;

static void am_init(amodel* m) {
  for (int i = 0; i < NSYM; i++) m->f[i] = 1;
  m->total = NSYM;
}

static void am_update(amodel* m, int s) {
  m->f[s] += 32;
  m->total += 32;
  if (m->total > FREQ_TOTAL) {
    m->total = 0;
    for (int i = 0; i < NSYM; i++) {
      m->f[i] = (m->f[i] + 1) >> 1;
      m->total += m->f[i];
    }
  }
}

static void am_encode(rc_enc* e, amodel* m, int s) {
  uint32_t lo = 0;
  for (int i = 0; i < s; i++) lo += m->f[i];
  enc_code(e, e->range / m->total, lo, m->f[s]);
  am_update(m, s);
}

static int am_decode(rc_dec* d, amodel* m) {
  uint32_t r = d->range / m->total;
  uint32_t v = d->code / r;
  if (v > m->total - 1) v = m->total - 1;
  uint32_t lo = 0;
  int s = 0;
  while (s < NSYM - 1 && lo + m->f[s] <= v) lo += m->f[s++];
  dec_update(d, r, lo, m->f[s]);
  am_update(m, s);
  return s;
}

int or_rc_encode_adaptive(const uint8_t* syms, int64_t n, uint8_t* out, size_t cap,
                          size_t* out_len) {
  rc_enc e;
  amodel m;
  enc_init(&e, out, cap);
  am_init(&m);
  for (int64_t i = 0; i < n; i++) {
    if (syms[i] > 254) return OR_INVALID_ARG;
    am_encode(&e, &m, syms[i]);
  }
  enc_flush(&e);
  *out_len = e.len;
  return e.overflow ? OR_CAPACITY : OR_OK;
}

int or_rc_decode_adaptive(int64_t n, const uint8_t* in, size_t len, uint8_t* syms) {
  rc_dec d;
  amodel m;
  dec_init(&d, in, len);
  am_init(&m);
  for (int64_t i = 0; i < n; i++) syms[i] = (uint8_t)am_decode(&d, &m);
  return d.bad ? OR_CORRUPT_STREAM : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Weight blob                                                               */
/* ------------------------------------------------------------------------ */

uint64_t or_fnv1a64(const void* data, size_t len) {
  const uint8_t* p = (const uint8_t*)data;
  uint64_t h = 14695981039346656037ull;
  for (size_t i = 0; i < len; i++) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

enum { K_SUM = 1, K_EMB = 2, K_RES = 3, K_SEL = 4 };

typedef struct {
  int kind, S, cin, cout, z_in, z_in2, z_out, shift, prelu;
  const int8_t* W;
  const int32_t* bias;
  const int32_t* mult;
  const int16_t* slope;
} rec;

#define MAXREC 64
/* Architectures (Sec. 4.3, Table 4): the paper's model and its two ablations */
enum { ARCH_XFP = 0, ARCH_GRED = 1, ARCH_BASE = 2 };

typedef struct {
  int C;
  int arch; /* ARCH_* */
  int toff; /* t = L - toff (Sec. 3.2; supplement, choice of t): 4 or 3 */
  uint32_t lut[256];
  uint64_t hash;
  int nrec;
  rec r[MAXREC];
  /* named slots, by relative level j = d - b */
  rec *ESH[5], *USH[5]; /* level b, and the propagated levels down to t */
  rec *RA[5], *RB[5], *RM[5], *P1[5], *P2[5], *G[5];
  rec *D[5][3], *E[5][3], *UP[5][3];
  int span[5]; /* m = d - k of a level extracted at level k (0: propagated) */
} model;

static size_t pad16(size_t n) { return (n + 15) & ~(size_t)15; }

static int rd_u32(const uint8_t* p) {
  return (int)((uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) |
               ((uint32_t)p[3] << 24));
}

static int parse_blob(const void* blob, size_t len, model* M) {
  const uint8_t* b = (const uint8_t*)blob;
  memset(M, 0, sizeof(*M));
  if (len < 32 + 1024 || memcmp(b, "LPCW", 4) != 0) return OR_INVALID_ARG;
  if (rd_u32(b + 4) != 1) return OR_INVALID_ARG;
  M->C = rd_u32(b + 8);
  M->nrec = rd_u32(b + 12);
  M->arch = rd_u32(b + 20);
  M->toff = rd_u32(b + 24) == 0 ? 4 : rd_u32(b + 24);
  if (M->arch < ARCH_XFP || M->arch > ARCH_BASE || (M->toff != 3 && M->toff != 4))
    return OR_INVALID_ARG;
  if (M->C < 8 || M->C > 128 || M->C % 8 || rd_u32(b + 16) != 256) return OR_INVALID_ARG;
  if (M->nrec < 1 || M->nrec > MAXREC) return OR_INVALID_ARG;
  for (int i = 0; i < 256; i++) M->lut[i] = (uint32_t)rd_u32(b + 32 + 4 * i);
  if (M->lut[0] != FREQ_TOTAL) return OR_INVALID_ARG;
  for (int i = 1; i < 256; i++)
    if (M->lut[i] > M->lut[i - 1]) return OR_INVALID_ARG;
  size_t off = 32 + 1024;
  for (int i = 0; i < M->nrec; i++) {
    rec* r = &M->r[i];
    if (off + 48 > len) return OR_INVALID_ARG;
    const uint8_t* h = b + off;
    r->kind = rd_u32(h); r->S = rd_u32(h + 4); r->cin = rd_u32(h + 8); r->cout = rd_u32(h + 12);
    r->z_in = rd_u32(h + 16); r->z_in2 = rd_u32(h + 20); r->z_out = rd_u32(h + 24);
    r->shift = rd_u32(h + 28); r->prelu = rd_u32(h + 32) & 1;
    off += 48;
    if (r->S < 1 || r->S > 27 || r->cin < 1 || r->cin > 256 || r->cout < 1 || r->cout > 256)
      return OR_INVALID_ARG;
    if (r->z_in < -128 || r->z_in > 127 || r->z_in2 < -128 || r->z_in2 > 127 ||
        r->z_out < -128 || r->z_out > 127)
      return OR_INVALID_ARG;
    size_t nw = (size_t)r->S * r->cout * r->cin;
    size_t np = (r->kind == K_SEL) ? (size_t)r->S * r->cout : (size_t)r->cout;
    if (r->kind == K_SUM || r->kind == K_SEL) {
      size_t need = pad16(nw) + pad16(4 * np) * 2 + pad16(2 * np);
      if (off + need > len) return OR_INVALID_ARG;
      r->W = (const int8_t*)(b + off); off += pad16(nw);
      r->bias = (const int32_t*)(b + off); off += pad16(4 * np);
      r->mult = (const int32_t*)(b + off); off += pad16(4 * np);
      r->slope = (const int16_t*)(b + off); off += pad16(2 * np);
      if (r->shift < 1 || r->shift > 62) return OR_INVALID_ARG;
      for (size_t k = 0; k < nw; k++)
        if (r->W[k] == -128) return OR_INVALID_ARG;
      for (size_t k = 0; k < np; k++) {
        if (r->bias[k] >= (1 << 30) || r->bias[k] <= -(1 << 30)) return OR_INVALID_ARG;
        if (r->mult[k] < 0) return OR_INVALID_ARG;
      }
    } else if (r->kind == K_EMB) {
      if (r->S != 1 || r->cin != 256) return OR_INVALID_ARG;
      size_t need = pad16((size_t)256 * r->cout);
      if (off + need > len) return OR_INVALID_ARG;
      r->W = (const int8_t*)(b + off); off += need;
    } else if (r->kind == K_RES) {
      if (r->S != 2 || r->cin != r->cout) return OR_INVALID_ARG;
      size_t need = pad16((size_t)8 * r->cout) + pad16((size_t)2 * r->cout);
      if (off + need > len) return OR_INVALID_ARG;
      r->mult = (const int32_t*)(b + off); off += pad16((size_t)8 * r->cout);
      r->slope = (const int16_t*)(b + off); off += pad16((size_t)2 * r->cout);
      if (r->shift < 1 || r->shift > 30) return OR_INVALID_ARG;
      for (int k = 0; k < 2 * r->cout; k++)
        if (r->mult[k] < 0 || r->mult[k] >= (1 << 16)) return OR_INVALID_ARG;
    } else {
      return OR_INVALID_ARG;
    }
  }
  if (off != len) return OR_INVALID_ARG;
  M->hash = or_fnv1a64(blob, len);
  return OR_OK;
}

/* Walk the records in network order and check every shape. */
static int bind_model(model* M) {
  const int C = M->C;
  int i = 0;
#define TAKE(slot, K, S_, CIN, COUT, PR)                                                   \
  do {                                                                                     \
    if (i >= M->nrec) return OR_INVALID_ARG;                                               \
    rec* r_ = &M->r[i++];                                                                  \
    if (r_->kind != (K) || r_->S != (S_) || r_->cin != (CIN) || r_->cout != (COUT) ||      \
        r_->prelu != (PR))                                                                 \
      return OR_INVALID_ARG;                                                               \
    (slot) = r_;                                                                           \
  } while (0)
  /* level b: F^b = Up(E_0[Y_{b-1}]) with no earlier features, every architecture */
  TAKE(M->ESH[0], K_EMB, 1, 256, C, 0);
  TAKE(M->USH[0], K_SEL, 8, C, C, 1);
  TAKE(M->P1[0], K_SUM, 1, C, C, 1);
  TAKE(M->P2[0], K_SUM, 1, C, NSYM, 0);
  const int nsh = 5 - M->toff; /* relative levels 1..nsh lie at or above t */
  for (int j = 1; j < 5; j++) {
    if (M->arch == ARCH_XFP && j <= nsh) { /* propagated shallow level (Eq. 8-9) */
      M->span[j] = 0;
      TAKE(M->RA[j], K_SUM, 27, C, C, 1);
      TAKE(M->RB[j], K_SUM, 27, C, C, 0);
      TAKE(M->RM[j], K_RES, 2, C, C, 1);
      TAKE(M->ESH[j], K_EMB, 1, 256, C, 0);
      TAKE(M->USH[j], K_SEL, 8, 2 * C, C, 1);
    } else {
      /* XFP deep level: re-densified to t and fused with F^t (Eq. 10-11);
       * otherwise features of X^{d-1} alone, extracted at k = t for GRED's
       * deep levels (Eq. 4-6) and at k = d - 1 elsewhere */
      const int deep = j - nsh;
      const int m = M->arch == ARCH_XFP ? deep
                    : (M->arch == ARCH_GRED && deep > 0) ? deep : 1;
      const int cat = M->arch == ARCH_XFP ? 2 : 1;
      M->span[j] = m;
      TAKE(M->G[j], K_EMB, 1, 256, C, 0);
      for (int k = 1; k < m; k++) TAKE(M->D[j][k], K_SUM, 8, C, C, 1);
      TAKE(M->RA[j], K_SUM, 27, cat * C, C, 1);
      TAKE(M->RB[j], K_SUM, 27, C, C, 0);
      TAKE(M->RM[j], K_RES, 2, C, C, 1);
      for (int k = 0; k < m; k++) {
        if (cat == 2) TAKE(M->E[j][k], K_EMB, 1, 256, C, 0);
        TAKE(M->UP[j][k], K_SEL, 8, cat * C, C, 1);
      }
    }
    TAKE(M->P1[j], K_SUM, 1, C, C, 1);
    TAKE(M->P2[j], K_SUM, 1, C, NSYM, 0);
  }
#undef TAKE
  return i == M->nrec ? OR_OK : OR_INVALID_ARG;
}

static int load_model(const void* blob, size_t len, model* M) {
  int st = parse_blob(blob, len, M);
  if (st) return st;
  return bind_model(M);
}

int or_check_blob(const void* blob, size_t len) {
  model* M = (model*)malloc(sizeof(model));
  int st = load_model(blob, len, M);
  free(M);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Network (Sec. 3.1 GRED, Sec. 3.2 XFP: Eq. 4-11)                            */
/* ------------------------------------------------------------------------ */

static const int8_t* emb_row(const rec* E, uint8_t code) { return E->W + (size_t)code * E->cout; }

/* rows of E[Y] for every node of a level, written into channels
 * [col, col + C) of a row-major [N][width] buffer */
static void embed(const rec* E, const uint8_t* codes, int64_t N, int8_t* dst, int width, int col) {
  for (int64_t n = 0; n < N; n++)
    memcpy(dst + n * width + col, emb_row(E, codes[n]), (size_t)E->cout);
}

static void copy_cols(const int8_t* src, int64_t N, int C, int8_t* dst, int width, int col) {
  for (int64_t n = 0; n < N; n++) memcpy(dst + n * width + col, src + n * C, (size_t)C);
}

static void conv_rec(const octree* T, int depth, const rec* R, const int8_t* x, int8_t* out) {
  or_conv333(T->key[depth], T->N[depth], depth, x, R->cin, R->z_in, R->W, R->bias, R->mult,
             R->shift, R->prelu ? R->slope : NULL, R->z_out, R->cout, out);
}

/* ResBlock (Eq. 5, Eq. 8, Eq. 10) on V_depth */
static void resblock(const model* M, int j, const octree* T, int depth, const int8_t* x,
                     int8_t* out) {
  const int C = M->C;
  int64_t N = T->N[depth];
  int8_t* y1 = (int8_t*)malloc((size_t)(N > 0 ? N : 1) * C);
  int8_t* y2 = (int8_t*)malloc((size_t)(N > 0 ? N : 1) * C);
  conv_rec(T, depth, M->RA[j], x, y1);
  conv_rec(T, depth, M->RB[j], y1, y2);
  const rec* R = M->RM[j];
  for (int64_t n = 0; n < N; n++)
    for (int c = 0; c < C; c++) {
      int64_t acc = (int64_t)(y1[n * C + c] - R->z_in) * R->mult[c] +
                    (int64_t)(y2[n * C + c] - R->z_in2) * R->mult[C + c];
      acc = or_prelu(acc, R->slope[c]);
      out[n * C + c] = (int8_t)or_requant(acc, 1, R->shift, R->z_out);
    }
  free(y1);
  free(y2);
}

/* Pruning(Upsampling(x), Y_d): V_d -> V_{d+1} (Eq. 6, Eq. 9, Eq. 11) */
static void up_rec(const octree* T, int d, const rec* R, const int8_t* x, int8_t* out) {
  or_up_prune(T->key[d], T->code[d], T->N[d], T->key[d + 1], T->N[d + 1], x, R->cin, R->z_in,
              R->W, R->bias, R->mult, R->shift, R->prelu ? R->slope : NULL, R->z_out, R->cout,
              out);
}

/* stride-2 conv V_{k+1} -> V_k (the sparse-conv part of Downsampling, Eq. 4) */
static void down_rec(const octree* T, int k, const rec* R, const int8_t* x, int8_t* out) {
  or_down_s2(T->key[k + 1], T->N[k + 1], T->key[k], T->N[k], x, R->cin, R->z_in, R->W, R->bias,
             R->mult, R->shift, R->prelu ? R->slope : NULL, R->z_out, R->cout, out);
}

/* Predictor (Eq. 7): C -> C (PReLU) -> 255 logits */
static void predictor(const model* M, int j, const int8_t* F, int64_t N, int8_t* logits) {
  const int C = M->C;
  const rec* A = M->P1[j];
  const rec* B = M->P2[j];
#pragma omp parallel for schedule(static) num_threads(g_threads)
  for (int64_t n = 0; n < N; n++) {
    int8_t h[256];
    for (int co = 0; co < C; co++) {
      int64_t acc = A->bias[co];
      for (int ci = 0; ci < C; ci++) acc += (int64_t)(F[n * C + ci] - A->z_in) * A->W[co * C + ci];
      h[co] = out_q(acc, A->mult[co], A->shift, A->prelu ? A->slope : NULL, co, A->z_out);
    }
    for (int s = 0; s < NSYM; s++) {
      int64_t acc = B->bias[s];
      for (int ci = 0; ci < C; ci++) acc += (int64_t)(h[ci] - B->z_in) * B->W[s * C + ci];
      logits[n * NSYM + s] = (int8_t)or_requant(acc, B->mult[s], B->shift, B->z_out);
    }
  }
}

typedef struct {
  const model* M;
  octree* T;
  int L, b, t;
  int8_t* F[22]; /* F^d on V_d of the propagated levels d = b..t (XFP), F^b otherwise */
} net;

static void net_free(net* S) {
  for (int d = 0; d < 22; d++) {
    free(S->F[d]);
    S->F[d] = NULL;
  }
}

/* F^b = Pruning(Upsampling(E_0[Y_{b-1}]), Y_{b-1}); with XFP, for b < d <= t:
 * S^{d-1} = ResBlock(F^{d-1}) (Eq. 8),
 * F^d = Pruning(Upsampling(Concat(S^{d-1}, Y_{d-1})), Y_{d-1}) (Eq. 9) */
static const int8_t* shallow_F(net* S, int d) {
  if (S->F[d]) return S->F[d];
  const model* M = S->M;
  const octree* T = S->T;
  const int C = M->C, b = S->b, j = d - b;
  int64_t Np = T->N[d - 1], Nc = T->N[d];
  int8_t* x;
  if (d == b) {
    x = (int8_t*)malloc((size_t)(Np > 0 ? Np : 1) * C);
    embed(M->ESH[0], T->code[b - 1], Np, x, C, 0);
  } else {
    const int8_t* Fp = shallow_F(S, d - 1);
    int8_t* Sp = (int8_t*)malloc((size_t)(Np > 0 ? Np : 1) * C);
    resblock(M, j, T, d - 1, Fp, Sp);
    x = (int8_t*)malloc((size_t)(Np > 0 ? Np : 1) * 2 * C);
    copy_cols(Sp, Np, C, x, 2 * C, 0);
    embed(M->ESH[j], T->code[d - 1], Np, x, 2 * C, C);
    free(Sp);
  }
  S->F[d] = (int8_t*)malloc((size_t)(Nc > 0 ? Nc : 1) * C);
  up_rec(T, d - 1, M->USH[j], x, S->F[d]);
  free(x);
  return S->F[d];
}

/* Logits of every node of V_d (b <= d <= L-1); needs V_0..V_d, Y_0..Y_{d-1}. */
static void net_level_logits(net* S, int d, int8_t* logits) {
  const model* M = S->M;
  const octree* T = S->T;
  const int C = M->C, b = S->b, t = S->t, j = d - b;
  if (d == b || (M->arch == ARCH_XFP && d <= t)) {
    predictor(M, j, shallow_F(S, d), T->N[d], logits);
    return;
  }
  /* G^k = Downsampling(Y_{d-1}) (Eq. 4): embedding on V_{d-1}, then m-1
   * stride-2 convs down to V_k; k = t for XFP's deep levels */
  const int m = M->span[j], k0 = d - m, cat = M->arch == ARCH_XFP ? 2 : 1;
  int64_t Ng = T->N[d - 1];
  int8_t* g = (int8_t*)malloc((size_t)(Ng > 0 ? Ng : 1) * C);
  embed(M->G[j], T->code[d - 1], Ng, g, C, 0);
  for (int i = 1; i < m; i++) {
    int k = d - 1 - i; /* V_{k+1} -> V_k */
    int8_t* g2 = (int8_t*)malloc((size_t)(T->N[k] > 0 ? T->N[k] : 1) * C);
    down_rec(T, k, M->D[j][i], g, g2);
    free(g);
    g = g2;
  }
  /* XFP: H^t = ResBlock(Concat(F^t, G^t)) (Eq. 10); otherwise
   * F^k = ResBlock(G^k) (Eq. 5) */
  int64_t Nk0 = T->N[k0];
  int8_t* x = g;
  if (cat == 2) {
    x = (int8_t*)malloc((size_t)(Nk0 > 0 ? Nk0 : 1) * 2 * C);
    copy_cols(shallow_F(S, t), Nk0, C, x, 2 * C, 0);
    copy_cols(g, Nk0, C, x, 2 * C, C);
    free(g);
  }
  int8_t* h = (int8_t*)malloc((size_t)(Nk0 > 0 ? Nk0 : 1) * C);
  resblock(M, j, T, k0, x, h);
  free(x);
  /* XFP: F^{k+1} = Pruning(Upsampling(Concat(H^k, Y_k)), Y_k) (Eq. 11);
   * otherwise F^{k+1} = Pruning(Upsampling(F^k), Y_k) (Eq. 6); k = k0..d-1 */
  for (int k = k0; k < d; k++) {
    int64_t Nk = T->N[k], Nn = T->N[k + 1];
    int8_t* xc = h;
    if (cat == 2) {
      xc = (int8_t*)malloc((size_t)(Nk > 0 ? Nk : 1) * 2 * C);
      copy_cols(h, Nk, C, xc, 2 * C, 0);
      embed(M->E[j][k - k0], T->code[k], Nk, xc, 2 * C, C);
      free(h);
    }
    h = (int8_t*)malloc((size_t)(Nn > 0 ? Nn : 1) * C);
    up_rec(T, k, M->UP[j][k - k0], xc, h);
    free(xc);
  }
  predictor(M, j, h, T->N[d], logits);
  free(h);
}

static int check_L(int L) { return (L >= 6 && L <= 21) ? OR_OK : OR_INVALID_ARG; }

static int level_logits(const void* blob, size_t blob_len, const int32_t* xyz, int64_t n, int L,
                        int d, int8_t** logits_out, int64_t* n_nodes, model** Mo, octree* T) {
  if (check_L(L) || d < L - 5 || d > L - 1) return OR_INVALID_ARG;
  model* M = (model*)malloc(sizeof(model));
  int st = load_model(blob, blob_len, M);
  if (st) { free(M); return st; }
  st = octree_from_points(xyz, n, L, T);
  if (st) { free(M); return st; }
  net S = {M, T, L, L - 5, L - M->toff, {NULL}};
  int64_t N = T->N[d];
  int8_t* lg = (int8_t*)malloc((size_t)(N > 0 ? N : 1) * NSYM);
  if (n > 0) net_level_logits(&S, d, lg);
  net_free(&S);
  *logits_out = lg;
  *n_nodes = N;
  *Mo = M;
  return OR_OK;
}

int or_logits_level(const void* blob, size_t blob_len, const int32_t* xyz, int64_t n, int L,
                    int d, int8_t* logits, int64_t cap_nodes, int64_t* n_nodes) {
  int8_t* lg;
  model* M;
  octree T;
  int st = level_logits(blob, blob_len, xyz, n, L, d, &lg, n_nodes, &M, &T);
  if (st) return st;
  if (*n_nodes > cap_nodes) st = OR_CAPACITY;
  else memcpy(logits, lg, (size_t)*n_nodes * NSYM);
  free(lg);
  free(M);
  octree_free(&T);
  return st;
}

int or_probs_level(const void* blob, size_t blob_len, const int32_t* xyz, int64_t n, int L,
                   int d, uint16_t* cdf, int64_t cap_nodes, int64_t* n_nodes) {
  int8_t* lg;
  model* M;
  octree T;
  int st = level_logits(blob, blob_len, xyz, n, L, d, &lg, n_nodes, &M, &T);
  if (st) return st;
  if (*n_nodes > cap_nodes) st = OR_CAPACITY;
  else or_softmax_cdf(lg, *n_nodes, M->lut, cdf);
  free(lg);
  free(M);
  octree_free(&T);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Bitstream                                                                 */
/* ------------------------------------------------------------------------ */
/* "LPC1", u8 version (3), u8 L, u8 b, u8 t, u8 C, u8 flags (bit0 = empty),
 * u64 blob hash (LE), varint chunk, varint coarse chunk, varint N_1 ..
 * N_{b-1} (the coarse levels' sizes; absent for an empty frame), varint
 * n_sub, n_sub x varint of the zigzag-coded difference between a substream's
 * length and the previous one's (0 before the first), then the substreams:
 * coarse levels 0..b-1 in
 * chunks of `coarse chunk` nodes (adaptive, a fresh model each), then for
 * d = b..L-1 the level's Morton-ordered nodes in chunks of `chunk`.  With
 * the sizes in the header every coarse chunk decodes on its own. */
#define COARSE_CHUNK 512

typedef struct {
  uint8_t* p;
  size_t len, cap;
} bytes;

static void by_put(bytes* B, const uint8_t* src, size_t n) {
  if (B->len + n > B->cap) {
    size_t nc = B->cap ? B->cap * 2 : 1024;
    while (nc < B->len + n) nc *= 2;
    B->p = (uint8_t*)realloc(B->p, nc);
    B->cap = nc;
  }
  memcpy(B->p + B->len, src, n);
  B->len += n;
}

static void by_varint(bytes* B, uint64_t v) {
  do {
    uint8_t c = (uint8_t)(v & 0x7F);
    v >>= 7;
    if (v) c |= 0x80;
    by_put(B, &c, 1);
  } while (v);
}

/* substream lengths: zigzag varints of the difference to the previous length */
static void by_len(bytes* B, size_t len, size_t* prev) {
  const int64_t d = (int64_t)len - (int64_t)*prev;
  by_varint(B, d >= 0 ? (uint64_t)d << 1 : (((uint64_t)(-d)) << 1) - 1);
  *prev = len;
}

static int rd_varint(const uint8_t* in, size_t len, size_t* pos, uint64_t* v) {
  *v = 0;
  for (int sh = 0; sh < 64; sh += 7) {
    if (*pos >= len) return OR_CORRUPT_STREAM;
    uint8_t c = in[(*pos)++];
    *v |= (uint64_t)(c & 0x7F) << sh;
    if (!(c & 0x80)) return OR_OK;
  }
  return OR_CORRUPT_STREAM;
}

/* one substream into B (and its length appended to lens) */
static void sub_begin(rc_enc* e, uint8_t** tmp, size_t n_sym) {
  size_t cap = n_sym * 4 + 64;
  *tmp = (uint8_t*)malloc(cap);
  enc_init(e, *tmp, cap);
}

int or_encode(const void* blob, size_t blob_len, const int32_t* xyz, int64_t n, int L,
              int chunk, uint8_t* out, size_t cap, size_t* out_len) {
  if (check_L(L) || chunk < 1 || n < 0) return OR_INVALID_ARG;
  model* M = (model*)malloc(sizeof(model));
  int st = load_model(blob, blob_len, M);
  if (st) { free(M); return st; }
  const int b = L - 5, t = L - M->toff;
  octree T;
  memset(&T, 0, sizeof(T));
  if (n > 0) {
    st = octree_from_points(xyz, n, L, &T);
    if (st) { free(M); return st; }
  }
  bytes subs = {0}, lens = {0};
  uint64_t n_sub = 0;
  size_t prev_len = 0;
  g_t_net = g_t_code = 0;
  if (n > 0) {
    /* coarse levels: adaptive symbol frequencies, every COARSE_CHUNK
     * symbols a substream with a fresh model */
    double t0 = now_s();
    for (int d = 0; d < b; d++) {
      for (int64_t s0 = 0; s0 < T.N[d]; s0 += COARSE_CHUNK) {
        const int64_t s1 = s0 + COARSE_CHUNK < T.N[d] ? s0 + COARSE_CHUNK : T.N[d];
        rc_enc e;
        amodel am;
        uint8_t* tmp;
        sub_begin(&e, &tmp, (size_t)(s1 - s0));
        am_init(&am);
        for (int64_t i = s0; i < s1; i++) am_encode(&e, &am, T.code[d][i] - 1);
        enc_flush(&e);
        by_put(&subs, tmp, e.len);
        by_len(&lens, e.len, &prev_len);
        n_sub++;
        free(tmp);
      }
    }
    g_t_code += now_s() - t0;
    /* network levels */
    net S = {M, &T, L, b, t, {NULL}};
    for (int d = b; d < L; d++) {
      int64_t N = T.N[d];
      int8_t* lg = (int8_t*)malloc((size_t)N * NSYM);
      uint16_t* cdf = (uint16_t*)malloc((size_t)N * 256 * sizeof(uint16_t));
      t0 = now_s();
      net_level_logits(&S, d, lg);
      or_softmax_cdf(lg, N, M->lut, cdf);
      const double t1 = now_s();
      g_t_net += t1 - t0;
      for (int64_t s0 = 0; s0 < N; s0 += chunk) {
        int64_t s1 = s0 + chunk < N ? s0 + chunk : N;
        rc_enc e;
        uint8_t* tmp;
        sub_begin(&e, &tmp, (size_t)(s1 - s0));
        for (int64_t i = s0; i < s1; i++) enc_symbol_row(&e, cdf + i * 256, T.code[d][i] - 1);
        enc_flush(&e);
        by_put(&subs, tmp, e.len);
        by_len(&lens, e.len, &prev_len);
        n_sub++;
        free(tmp);
      }
      g_t_code += now_s() - t1;
      free(lg);
      free(cdf);
    }
    net_free(&S);
  }
  bytes H = {0};
  uint8_t hdr[18];
  memcpy(hdr, "LPC1", 4);
  hdr[4] = 3;
  hdr[5] = (uint8_t)L;
  hdr[6] = (uint8_t)b;
  hdr[7] = (uint8_t)t;
  hdr[8] = (uint8_t)M->C;
  hdr[9] = n > 0 ? 0 : 1;
  for (int i = 0; i < 8; i++) hdr[10 + i] = (uint8_t)(M->hash >> (8 * i));
  by_put(&H, hdr, 18);
  by_varint(&H, (uint64_t)chunk);
  by_varint(&H, (uint64_t)COARSE_CHUNK);
  if (n > 0)
    for (int d = 1; d < b; d++) by_varint(&H, (uint64_t)T.N[d]);
  by_varint(&H, n_sub);
  if (lens.len) by_put(&H, lens.p, lens.len);
  if (subs.len) by_put(&H, subs.p, subs.len);
  *out_len = H.len;
  st = H.len > cap ? OR_CAPACITY : OR_OK;
  if (!st) memcpy(out, H.p, H.len);
  free(H.p);
  free(subs.p);
  free(lens.p);
  octree_free(&T);
  free(M);
  return st;
}

int or_decode(const void* blob, size_t blob_len, const uint8_t* in, size_t len,
              int32_t* xyz_out, int64_t cap, int64_t* n_out) {
  model* M = (model*)malloc(sizeof(model));
  int st = load_model(blob, blob_len, M);
  if (st) { free(M); return st; }
  *n_out = 0;
  if (len < 18 || memcmp(in, "LPC1", 4) != 0 || in[4] != 3) { free(M); return OR_CORRUPT_STREAM; }
  const int L = in[5], b = in[6], t = in[7], C = in[8], flags = in[9];
  uint64_t hash = 0;
  for (int i = 0; i < 8; i++) hash |= (uint64_t)in[10 + i] << (8 * i);
  if (check_L(L) || b != L - 5) { free(M); return OR_CORRUPT_STREAM; }
  if (hash != M->hash || C != M->C) { free(M); return OR_WEIGHTS_MISMATCH; }
  if (t != L - M->toff) { free(M); return OR_CORRUPT_STREAM; }
  size_t pos = 18;
  uint64_t chunk, cchunk, n_sub;
  uint64_t cN[22] = {1}; /* coarse level sizes N_0 = 1, N_1 .. N_{b-1} from the header */
  if (rd_varint(in, len, &pos, &chunk) || rd_varint(in, len, &pos, &cchunk) || chunk < 1 ||
      chunk > (1u << 30) || cchunk < 1 || cchunk > (1u << 30)) {
    free(M);
    return OR_CORRUPT_STREAM;
  }
  for (int d = 1; d < b && !(flags & 1); d++)
    if (rd_varint(in, len, &pos, &cN[d]) || cN[d] < 1 || cN[d] > 8 * cN[d - 1]) {
      free(M);
      return OR_CORRUPT_STREAM;
    }
  if (rd_varint(in, len, &pos, &n_sub) || n_sub > len) {
    free(M);
    return OR_CORRUPT_STREAM;
  }
  if (flags & 1) {
    free(M);
    return n_sub == 0 ? OR_OK : OR_CORRUPT_STREAM;
  }
  uint64_t* sl = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n_sub + 1));
  size_t* so = (size_t*)malloc(sizeof(size_t) * (size_t)(n_sub + 1));
  uint64_t prev = 0;
  for (uint64_t i = 0; i < n_sub; i++) {
    uint64_t z;
    if (rd_varint(in, len, &pos, &z)) { st = OR_CORRUPT_STREAM; break; }
    const uint64_t mag = (z + 1) >> 1;
    if ((z & 1) ? mag > prev : mag > len) { st = OR_CORRUPT_STREAM; break; }
    sl[i] = prev = (z & 1) ? prev - mag : prev + mag;
  }
  size_t p = pos;
  for (uint64_t i = 0; !st && i < n_sub; i++) {
    so[i] = p;
    if (sl[i] > len - p) st = OR_CORRUPT_STREAM;
    else p += sl[i];
  }
  octree T;
  memset(&T, 0, sizeof(T));
  T.L = L;
  uint64_t si = 0;
  g_t_net = g_t_code = 0;
  if (!st) {
    T.N[0] = 1;
    T.key[0] = (uint64_t*)calloc(1, sizeof(uint64_t));
    for (int d = 0; d < b && !st; d++) {
      /* the header's N_d must be what the level above expands to */
      if ((uint64_t)T.N[d] != cN[d]) { st = OR_CORRUPT_STREAM; break; }
      T.code[d] = (uint8_t*)malloc((size_t)T.N[d]);
      const double t0 = now_s();
      for (int64_t s0 = 0; s0 < T.N[d] && !st; s0 += (int64_t)cchunk) {
        const int64_t s1 = s0 + (int64_t)cchunk < T.N[d] ? s0 + (int64_t)cchunk : T.N[d];
        if (si >= n_sub) { st = OR_CORRUPT_STREAM; break; }
        st = or_rc_decode_adaptive(s1 - s0, in + so[si], (size_t)sl[si], T.code[d] + s0);
        si++;
      }
      g_t_code += now_s() - t0;
      for (int64_t i = 0; !st && i < T.N[d]; i++) T.code[d][i] += 1;
      if (!st) st = octree_expand(&T, d);
    }
    net S = {M, &T, L, b, t, {NULL}};
    for (int d = b; d < L && !st; d++) {
      int64_t N = T.N[d];
      int8_t* lg = (int8_t*)malloc((size_t)N * NSYM);
      uint16_t* cdf = (uint16_t*)malloc((size_t)N * 256 * sizeof(uint16_t));
      const double t0 = now_s();
      net_level_logits(&S, d, lg);
      or_softmax_cdf(lg, N, M->lut, cdf);
      const double t1 = now_s();
      g_t_net += t1 - t0;
      T.code[d] = (uint8_t*)malloc((size_t)N);
      for (int64_t s0 = 0; s0 < N && !st; s0 += (int64_t)chunk) {
        int64_t s1 = s0 + (int64_t)chunk < N ? s0 + (int64_t)chunk : N;
        if (si >= n_sub) { st = OR_CORRUPT_STREAM; break; }
        st = or_rc_decode_cdf(cdf + s0 * 256, s1 - s0, in + so[si], (size_t)sl[si],
                              T.code[d] + s0);
        si++;
      }
      g_t_code += now_s() - t1;
      for (int64_t i = 0; !st && i < N; i++) T.code[d][i] += 1;
      free(lg);
      free(cdf);
      if (!st) st = octree_expand(&T, d);
    }
    net_free(&S);
  }
  if (!st && si != n_sub) st = OR_CORRUPT_STREAM;
  if (!st) {
    int64_t N = T.N[L];
    *n_out = N;
    if (N > cap) st = OR_CAPACITY;
    else
      for (int64_t i = 0; i < N; i++) {
        int64_t x, y, z;
        morton_decode(T.key[L][i], L, &x, &y, &z);
        xyz_out[3 * i] = (int32_t)x;
        xyz_out[3 * i + 1] = (int32_t)y;
        xyz_out[3 * i + 2] = (int32_t)z;
      }
  }
  octree_free(&T);
  free(sl);
  free(so);
  free(M);
  return st;
}
