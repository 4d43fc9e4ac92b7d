// GB300 (sm_103a) per-shot sampling kernels.
//
// One thread evaluates one shot end to end (Sec. "Complexity", paragraph
// "Sampling"):
//   1. error mechanisms: one Philox4x32-10 word per reduced channel, outcome by
//      integer threshold compare, f ^= column signature (Eq. detector_sampling);
//   2. outputs in autoregressive order: deterministic outputs are GF(2)
//      parities of X = (f, random outputs) by AND + popcount; random outputs
//      follow Algorithm 1, with every marginal P = sum_t c^t prod_k h(...)
//      evaluated exactly: each factor's parities (Eq. parities) select one of
//      four packed (zero, sqrt2-exponent, w-exponent) increments, a term is
//      w^J sqrt2^S or 0, and the sum is accumulated in four integer
//      coefficients of Z[w] (no floating point anywhere);
//   3. the Bernoulli draw compares U * P_prev with 2^32 * P_1 exactly;
//   4. bit-packed records.
// The program tables are read-only and identical for every thread: all
// threads of a warp read the same table word at the same time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "device.h"
#include "zx.h"

namespace tsim {

#define TSIM_CUDA(x)                                                                  \
  do {                                                                                \
    cudaError_t e_ = (x);                                                             \
    if (e_ != cudaSuccess) fail(TSIM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

enum : int { ST_NOT_REAL = 1, ST_OVERFLOW = 2, ST_ZERO_PROB = 4 };

// device-wide status word: bits of the conditions above, read by tsim_sync
__device__ int g_status;

constexpr int kMaxChains = 16;
constexpr int kMaxOutWords = 64;  // 4096 outputs
constexpr int kThreads = 128;

struct DChan { uint32_t n_out, thr_off, sig_off, pad; };
struct DOut { int32_t random, cst, xbit, chain, table; uint32_t mask_off; };
struct DTable { uint32_t term_off, n_terms; int32_t base, pad; };
struct DTerm { uint32_t fac_off, n_fac; int32_t s0rel, j0; };

struct DevView {
  int W;
  int n_ch, n_out, n_chains, n_tab;
  int nmeas, ndet, nobs, mode;
  const DChan* ch;
  const uint32_t* thr;
  const uint64_t* sig;
  const DOut* out;
  const uint64_t* omask;
  const int32_t* chain_norm;
  const DTable* tab;
  const DTerm* term;
  const uint64_t* fuv;    // per factor: u[W], v[W]
  const uint32_t* flut;   // per factor: 4 packed increments
  const int32_t* dmap_off;
  const int32_t* dmap_idx;
  const int32_t* omap_off;
  const int32_t* omap_idx;
};

struct DeviceProgram {
  DevView v{};
  void* blob = nullptr;
  int device = -1;
};

void device_release(DeviceProgram* d) {
  if (!d) return;
  if (d->blob) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (d->device >= 0 && d->device != cur) cudaSetDevice(d->device);
    cudaFree(d->blob);
    if (d->device >= 0 && d->device != cur) cudaSetDevice(cur);
  }
  delete d;
}

bool monomial_of(const ZW& v, int* zero, int* s, int* j) {
  if (v.zero()) { *zero = 1; *s = 0; *j = 0; return true; }
  *zero = 0;
  for (int ss = -16; ss <= 16; ++ss)
    for (int jj = 0; jj < 8; ++jj) {
      ZW m = ZW::omega(jj + 4);  // -w^jj
      m.k = ss;
      if (zw_add(v, m).zero()) { *s = ss; *j = jj; return true; }
    }
  return false;
}

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 products.
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t o[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  o[0] = c0; o[1] = c1; o[2] = c2; o[3] = c3;
}

// ------------------------------------------------------- exact real values
struct RV {
  __int128 A, B;  // value = (A + B sqrt2) * 2^e
  int e;
};

__device__ __forceinline__ __int128 shl_chk(__int128 x, int s, int* st) {
  if (s <= 0) return x;
  __int128 ax = x < 0 ? -x : x;
  if (s >= 126 || (ax >> (126 - s)) != 0) { *st |= ST_OVERFLOW; return 0; }
  return x * ((__int128)1 << s);
}

__device__ __forceinline__ int sign_xy(__int128 X, __int128 Y, int* st) {
  if (X >= 0 && Y >= 0) return (X == 0 && Y == 0) ? 0 : 1;
  if (X <= 0 && Y <= 0) return -1;
  unsigned __int128 ax = X < 0 ? (unsigned __int128)(-X) : (unsigned __int128)X;
  unsigned __int128 ay = Y < 0 ? (unsigned __int128)(-Y) : (unsigned __int128)Y;
  if ((ax >> 63) || (ay >> 63)) { *st |= ST_OVERFLOW; return 0; }
  unsigned __int128 x2 = ax * ax, y2 = 2 * ay * ay;
  if (X > 0) return x2 > y2 ? 1 : -1;
  return y2 > x2 ? 1 : -1;
}

template <int W>
__device__ RV eval_table(const DevView& V, int t, const uint64_t (&X)[W], int* st) {
  const DTable tb = V.tab[t];
  long long c[4] = {0, 0, 0, 0};
  for (uint32_t q = 0; q < tb.n_terms; ++q) {
    const DTerm tm = V.term[tb.term_off + q];
    uint32_t acc = 0;
    for (uint32_t k = 0; k < tm.n_fac; ++k) {
      const size_t f = (size_t)tm.fac_off + k;
      const uint64_t* uv = V.fuv + f * (2 * W);
      uint64_t pa = 0, pb = 0;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        pa ^= __ldg(uv + w) & X[w];
        pb ^= __ldg(uv + W + w) & X[w];
      }
      int idx = (__popcll(pa) & 1) | ((__popcll(pb) & 1) << 1);
      acc += __ldg(V.flut + f * 4 + idx);
    }
    if (acc >> 21) continue;  // some factor vanished
    int J = (tm.j0 + (int)(acc & 0x7FF)) & 7;
    int d = tm.s0rel + (int)((acc >> 11) & 0x3FF);
    long long mag = 1ll << (d >> 1);
    if (d & 1) {
      // sqrt2 w^J = w^(J+1) - w^(J+3)
      int a = (J + 1) & 7, b = (J + 3) & 7;
      c[a & 3] += (a < 4) ? mag : -mag;
      c[b & 3] -= (b < 4) ? mag : -mag;
    } else {
      c[J & 3] += (J < 4) ? mag : -mag;
    }
  }
  // real part: Re(c0 + c1 w + c2 w^2 + c3 w^3) = (2 c0 + (c1 - c3) sqrt2) / 2
  if (c[2] != 0 || c[1] + c[3] != 0) *st |= ST_NOT_REAL;
  RV r;
  r.A = (__int128)2 * c[0];
  r.B = (__int128)c[1] - c[3];
  int K = tb.base - 2;
  if (K & 1) {
    __int128 t2 = r.A;
    r.A = 2 * r.B;
    r.B = t2;
    K -= 1;
  }
  r.e = K / 2;
  return r;
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_sample(DevView V, uint64_t seed, uint64_t shot0,
                                                     uint64_t nshots, uint64_t* __restrict__ meas,
                                                     uint64_t* __restrict__ det,
                                                     uint64_t* __restrict__ obs,
                                                     uint8_t* __restrict__ accept) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nshots) return;
  const uint64_t shot = shot0 + s;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const uint32_t c0 = (uint32_t)shot, c1 = (uint32_t)(shot >> 32);
  int st = 0;

  // 1. error mechanisms and f = T e
  uint64_t X[W];
#pragma unroll
  for (int w = 0; w < W; ++w) X[w] = 0;
  for (int c = 0; c < V.n_ch; c += 4) {
    uint32_t u[4];
    philox4x32_10(c0, c1, 0u, (uint32_t)(c >> 2), k0, k1, u);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int ci = c + l;
      if (ci >= V.n_ch) break;
      const DChan ch = V.ch[ci];
      const uint32_t U = u[l];
      const uint32_t* thr = V.thr + ch.thr_off;
      uint32_t o = 0;
      while (o + 1 < ch.n_out && U >= __ldg(thr + o)) ++o;
      if (o) {
        const uint64_t* sg = V.sig + ch.sig_off + (size_t)o * W;
#pragma unroll
        for (int w = 0; w < W; ++w) X[w] ^= __ldg(sg + w);
      }
    }
  }

  // 2-3. outputs in autoregressive order (Algorithm 1 per chain)
  RV pp[kMaxChains];
  for (int c = 0; c < V.n_chains; ++c) pp[c] = eval_table<W>(V, V.chain_norm[c], X, &st);
  uint64_t ob[kMaxOutWords];
  const int obw = (V.n_out + 63) >> 6;
  for (int w = 0; w < obw; ++w) ob[w] = 0;
  for (int i = 0; i < V.n_out; ++i) {
    const DOut o = V.out[i];
    int bit;
    if (!o.random) {
      const uint64_t* m = V.omask + o.mask_off;
      uint64_t acc = 0;
#pragma unroll
      for (int w = 0; w < W; ++w) acc ^= __ldg(m + w) & X[w];
      bit = (__popcll(acc) & 1) ^ o.cst;
    } else {
      const int xb = o.xbit;
      X[xb >> 6] |= 1ull << (xb & 63);
      const RV p1 = eval_table<W>(V, o.table, X, &st);
      const RV pv = pp[o.chain];
      if (sign_xy(pv.A, pv.B, &st) <= 0) st |= ST_ZERO_PROB;
      uint32_t u[4];
      philox4x32_10(c0, c1, 1u, (uint32_t)(i >> 2), k0, k1, u);
      const uint32_t U = u[i & 3];
      // bit = 1 iff U * P_prev < 2^32 * P_1
      const int e = min(pv.e, p1.e + 32);
      const __int128 LA = shl_chk(pv.A * (__int128)U, pv.e - e, &st);
      const __int128 LB = shl_chk(pv.B * (__int128)U, pv.e - e, &st);
      const __int128 RA = shl_chk(p1.A, p1.e + 32 - e, &st);
      const __int128 RB = shl_chk(p1.B, p1.e + 32 - e, &st);
      bit = sign_xy(LA - RA, LB - RB, &st) < 0;
      if (bit) {
        pp[o.chain] = p1;
      } else {
        const int e2 = min(pv.e, p1.e);
        RV d;
        d.A = shl_chk(pv.A, pv.e - e2, &st) - shl_chk(p1.A, p1.e - e2, &st);
        d.B = shl_chk(pv.B, pv.e - e2, &st) - shl_chk(p1.B, p1.e - e2, &st);
        d.e = e2;
        pp[o.chain] = d;
        X[xb >> 6] &= ~(1ull << (xb & 63));
      }
    }
    ob[i >> 6] |= (uint64_t)bit << (i & 63);
  }

  // 4. records
  auto bits_at = [&](int start, int w) -> uint64_t {  // 64 output bits from `start`
    const int q = start + 64 * w;
    const int wi = q >> 6, sh = q & 63;
    uint64_t lo = wi < obw ? ob[wi] : 0;
    if (!sh) return lo;
    uint64_t hi = wi + 1 < obw ? ob[wi + 1] : 0;
    return (lo >> sh) | (hi << (64 - sh));
  };
  auto tail = [](int n, int w) -> uint64_t {
    const int r = n - 64 * w;
    return r >= 64 ? ~0ull : ((1ull << r) - 1);
  };
  bool any_det = false;
  const int dw = (V.ndet + 63) >> 6, mw = (V.nmeas + 63) >> 6, ow = (V.nobs + 63) >> 6;
  if (V.mode == 0) {
    for (int w = 0; w < dw; ++w) {
      const uint64_t v = bits_at(0, w) & tail(V.ndet, w);
      any_det |= v != 0;
      if (det) det[s * dw + w] = v;
    }
    if (obs)
      for (int w = 0; w < ow; ++w) obs[s * ow + w] = bits_at(V.ndet, w) & tail(V.nobs, w);
  } else {
    if (meas)
      for (int w = 0; w < mw; ++w) meas[s * mw + w] = bits_at(0, w) & tail(V.nmeas, w);
    for (int w = 0; w < dw; ++w) {
      uint64_t v = 0;
      for (int b = 0; b < 64 && 64 * w + b < V.ndet; ++b) {
        const int d = 64 * w + b;
        int x = 0;
        for (int q = V.dmap_off[d]; q < V.dmap_off[d + 1]; ++q) {
          const int j = V.dmap_idx[q];
          x ^= (int)((ob[j >> 6] >> (j & 63)) & 1);
        }
        v |= (uint64_t)x << b;
      }
      any_det |= v != 0;
      if (det) det[s * dw + w] = v;
    }
    if (obs)
      for (int w = 0; w < ow; ++w) {
        uint64_t v = 0;
        for (int b = 0; b < 64 && 64 * w + b < V.nobs; ++b) {
          const int d = 64 * w + b;
          int x = 0;
          for (int q = V.omap_off[d]; q < V.omap_off[d + 1]; ++q) {
            const int j = V.omap_idx[q];
            x ^= (int)((ob[j >> 6] >> (j & 63)) & 1);
          }
          v |= (uint64_t)x << b;
        }
        obs[s * ow + w] = v;
      }
  }
  if (accept) accept[s] = any_det ? 0 : 1;
  if (st) atomicOr(&g_status, st);
}

// ------------------------------------------------------------------ upload
namespace {

int padded_words_or_zero(int W) {
  for (int p : {1, 2, 4, 8, 16, 32})
    if (W <= p) return p;
  return 0;
}

// Byte sinks for the table packer: sections start on 256-byte boundaries and
// alignment padding is zero.  VecSink grows a host vector; FixedSink writes
// into a caller-provided buffer of fixed capacity and never allocates.
struct VecSink {
  std::vector<unsigned char> b;
  size_t section() {
    b.resize((b.size() + 255) & ~(size_t)255, 0);
    return b.size();
  }
  void put(const void* p, size_t n) {
    size_t o = b.size();
    b.resize(o + n);
    if (n) std::memcpy(b.data() + o, p, n);
  }
  size_t size() const { return b.size(); }
};

struct FixedSink {
  unsigned char* base;
  size_t cap;
  size_t n = 0;
  bool overflow = false;
  size_t section() {
    size_t off = (n + 255) & ~(size_t)255;
    if (off > cap) overflow = true;
    else std::memset(base + n, 0, off - n);
    n = off;
    return off;
  }
  void put(const void* p, size_t k) {
    if (overflow || n + k > cap) { overflow = true; n += k; return; }
    if (k) std::memcpy(base + n, p, k);
    n += k;
  }
  size_t size() const { return n; }
};

struct Layout {
  size_t o_ch = 0, o_thr = 0, o_sig = 0, o_out = 0, o_om = 0, o_cn = 0, o_tab = 0, o_term = 0,
         o_fuv = 0, o_flut = 0, o_dmo = 0, o_dmi = 0, o_omo = 0, o_omi = 0, total = 0;
  int W = 1;
};

// Four packed increments of one factor, inc = j | s << 11 | zero << 21
// (J in bits 0-10, S in 11-20, vanishing factors in 21-31), with s relative
// to the factor's smallest magnitude exponent smin.
bool factor_lut(const ProgFactor& f, uint32_t inc[4], int* smin_out, int* spread) {
  Factor fc;
  fc.kind = f.kind;
  fc.alpha = f.alpha;
  fc.beta = f.beta;
  int zs[4], ss[4], js[4], smin = 1 << 20, smax = -(1 << 20);
  for (int idx = 0; idx < 4; ++idx) {
    if (!monomial_of(factor_value(fc, idx & 1, idx >> 1), &zs[idx], &ss[idx], &js[idx])) return false;
    if (!zs[idx]) { smin = std::min(smin, ss[idx]); smax = std::max(smax, ss[idx]); }
  }
  if (smin > smax) smin = smax = 0;
  if (smax - smin > 3) return false;
  for (int idx = 0; idx < 4; ++idx)
    inc[idx] = zs[idx] ? (1u << 21) : ((uint32_t)js[idx] | ((uint32_t)(ss[idx] - smin) << 11));
  *smin_out = smin;
  *spread = smax - smin;
  return true;
}

// raw sqrt2 exponent (s0 plus every factor's smin) and magnitude spread of a term
bool term_exponents(const ProgTerm& tm, int* raw_s0, int* spread) {
  uint32_t inc[4];
  int s0 = tm.s0, sp = 0;
  for (const ProgFactor& f : tm.f) {
    int smin, spr;
    if (!factor_lut(f, inc, &smin, &spr)) return false;
    s0 += smin;
    sp += spr;
  }
  *raw_s0 = s0;
  *spread = sp;
  return true;
}

// base exponent of a table = smallest raw term exponent; checks that the
// 64-bit coefficient accumulation cannot overflow
tsim_status table_base(const ProgTable& tb, int* base, const char** msg) {
  int b = 0, dmax = 0;
  bool first = true;
  for (const ProgTerm& tm : tb.terms) {
    int r, sp;
    if (tm.f.size() > 255) { *msg = "term with more than 255 factors"; return TSIM_ERR_OVERFLOW_BOUND; }
    if (!term_exponents(tm, &r, &sp)) { *msg = "factor value is not a monomial of bounded spread"; return TSIM_ERR_INTERNAL; }
    if (first || r < b) b = r;
    first = false;
  }
  for (const ProgTerm& tm : tb.terms) {
    int r, sp;
    term_exponents(tm, &r, &sp);
    dmax = std::max(dmax, r - b + sp);
  }
  int lg = 0;
  while ((1ull << lg) < (uint64_t)std::max<size_t>(1, tb.terms.size())) ++lg;
  // |coefficient| <= terms * 2^(dmax/2 + 1) must stay below 2^62
  if (dmax / 2 + 1 + lg >= 62) { *msg = "table magnitudes exceed 64-bit accumulation"; return TSIM_ERR_OVERFLOW_BOUND; }
  *base = b;
  return TSIM_OK;
}

template <class Sink>
void put_padded(Sink& s, const std::vector<uint64_t>& m, int W) {
  for (int i = 0; i < W; ++i) {
    uint64_t x = (size_t)i < m.size() ? m[(size_t)i] : 0;
    s.put(&x, 8);
  }
}

// Packs the program into the device table layout.  Heap-free apart from
// what the sink itself does.
template <class Sink>
tsim_status pack_tables(const Program& p, Sink& s, Layout& L, const char** msg) {
  const int W = padded_words_or_zero(p.W);
  if (!W) { *msg = "per-shot vector wider than 2048 bits is not supported"; return TSIM_ERR_ARG; }
  if ((int)p.chain_norm.size() > kMaxChains) { *msg = "too many autoregressive chains for the kernel"; return TSIM_ERR_ARG; }
  if ((int)p.outputs.size() > kMaxOutWords * 64) { *msg = "too many outputs for the kernel"; return TSIM_ERR_ARG; }
  L.W = W;
  // channels
  L.o_ch = s.section();
  {
    uint32_t thr_off = 0, sig_off = 0;
    for (const ProgChannel& c : p.channels) {
      DChan d{};
      d.n_out = (uint32_t)c.sig.size();
      d.thr_off = thr_off;
      d.sig_off = sig_off;
      thr_off += (uint32_t)c.thr.size();
      sig_off += (uint32_t)(c.sig.size() * (size_t)W);
      s.put(&d, sizeof d);
      for (size_t w = 0; !c.sig.empty() && w < c.sig[0].size(); ++w)
        if (c.sig[0][w]) { *msg = "channel outcome 0 must not flip anything"; return TSIM_ERR_INTERNAL; }
    }
  }
  L.o_thr = s.section();
  for (const ProgChannel& c : p.channels)
    for (uint32_t t : c.thr) s.put(&t, 4);
  { uint32_t z = 0; s.put(&z, 4); }
  L.o_sig = s.section();
  for (const ProgChannel& c : p.channels)
    for (const auto& sg : c.sig) put_padded(s, sg, W);
  // outputs
  L.o_out = s.section();
  {
    uint32_t mo = 0;
    for (const ProgOutput& o : p.outputs) {
      DOut d{};
      d.random = o.random ? 1 : 0;
      d.cst = o.cst;
      d.xbit = o.xbit;
      d.chain = o.chain;
      d.table = o.table;
      d.mask_off = mo;
      mo += (uint32_t)W;
      s.put(&d, sizeof d);
    }
  }
  L.o_om = s.section();
  for (const ProgOutput& o : p.outputs) put_padded(s, o.mask, W);
  L.o_cn = s.section();
  for (int c : p.chain_norm) { int32_t v = c; s.put(&v, 4); }
  { int32_t z = 0; s.put(&z, 4); }
  // tables
  L.o_tab = s.section();
  {
    uint32_t term_off = 0;
    for (const ProgTable& tb : p.tables) {
      DTable dt{};
      dt.term_off = term_off;
      dt.n_terms = (uint32_t)tb.terms.size();
      tsim_status st = table_base(tb, &dt.base, msg);
      if (st != TSIM_OK) return st;
      term_off += dt.n_terms;
      s.put(&dt, sizeof dt);
    }
  }
  L.o_term = s.section();
  {
    uint32_t fac_off = 0;
    for (const ProgTable& tb : p.tables) {
      int base = 0;
      table_base(tb, &base, msg);
      for (const ProgTerm& tm : tb.terms) {
        DTerm d{};
        int r, sp;
        term_exponents(tm, &r, &sp);
        d.fac_off = fac_off;
        d.n_fac = (uint32_t)tm.f.size();
        d.s0rel = r - base;
        d.j0 = tm.j0 & 7;
        fac_off += d.n_fac;
        s.put(&d, sizeof d);
      }
    }
  }
  L.o_fuv = s.section();
  for (const ProgTable& tb : p.tables)
    for (const ProgTerm& tm : tb.terms)
      for (const ProgFactor& f : tm.f) {
        put_padded(s, f.u, W);
        put_padded(s, f.v, W);
      }
  L.o_flut = s.section();
  for (const ProgTable& tb : p.tables)
    for (const ProgTerm& tm : tb.terms)
      for (const ProgFactor& f : tm.f) {
        uint32_t inc[4];
        int smin, spr;
        factor_lut(f, inc, &smin, &spr);
        s.put(inc, sizeof inc);
      }
  // measurement-mode detector / observable maps (CSR)
  auto csr = [&](const std::vector<std::vector<int>>& m, size_t* o_off, size_t* o_idx) {
    *o_off = s.section();
    int32_t acc = 0;
    s.put(&acc, 4);
    for (const auto& d : m) { acc += (int32_t)d.size(); s.put(&acc, 4); }
    *o_idx = s.section();
    for (const auto& d : m)
      for (int j : d) { int32_t v = j; s.put(&v, 4); }
    int32_t z = 0;
    s.put(&z, 4);
  };
  csr(p.detmap, &L.o_dmo, &L.o_dmi);
  csr(p.obsmap, &L.o_omo, &L.o_omi);
  L.total = s.section();
  return TSIM_OK;
}

DevView make_view(const unsigned char* base, const Layout& L, const Program& p) {
  DevView v{};
  v.W = L.W;
  v.n_ch = (int)p.channels.size();
  v.n_out = (int)p.outputs.size();
  v.n_chains = (int)p.chain_norm.size();
  v.n_tab = (int)p.tables.size();
  v.nmeas = p.nmeas;
  v.ndet = p.ndet;
  v.nobs = p.nobs;
  v.mode = p.mode;
  v.ch = (const DChan*)(base + L.o_ch);
  v.thr = (const uint32_t*)(base + L.o_thr);
  v.sig = (const uint64_t*)(base + L.o_sig);
  v.out = (const DOut*)(base + L.o_out);
  v.omask = (const uint64_t*)(base + L.o_om);
  v.chain_norm = (const int32_t*)(base + L.o_cn);
  v.tab = (const DTable*)(base + L.o_tab);
  v.term = (const DTerm*)(base + L.o_term);
  v.fuv = (const uint64_t*)(base + L.o_fuv);
  v.flut = (const uint32_t*)(base + L.o_flut);
  v.dmap_off = (const int32_t*)(base + L.o_dmo);
  v.dmap_idx = (const int32_t*)(base + L.o_dmi);
  v.omap_off = (const int32_t*)(base + L.o_omo);
  v.omap_idx = (const int32_t*)(base + L.o_omi);
  return v;
}

DeviceProgram* upload(const Program& p) {
  VecSink b;
  Layout L;
  const char* msg = "";
  tsim_status st = pack_tables(p, b, L, &msg);
  if (st != TSIM_OK) fail(st, msg);
  auto* d = new DeviceProgram();
  TSIM_CUDA(cudaGetDevice(&d->device));
  cudaError_t e = cudaMalloc(&d->blob, std::max<size_t>(b.size(), 256));
  if (e != cudaSuccess) {
    delete d;
    fail(TSIM_ERR_OOM, std::string("cudaMalloc of program tables: ") + cudaGetErrorString(e));
  }
  e = cudaMemcpy(d->blob, b.b.data(), b.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d->blob);
    delete d;
    fail(TSIM_ERR_CUDA, std::string("cudaMemcpy of program tables: ") + cudaGetErrorString(e));
  }
  d->v = make_view((const unsigned char*)d->blob, L, p);
  return d;
}

const DevView& ensure_uploaded(const Program& p) {
  int cur = -1;
  TSIM_CUDA(cudaGetDevice(&cur));
  auto& slot = const_cast<Program&>(p).dev;
  if (slot && slot->device != cur) {
    device_release(slot);
    slot = nullptr;
  }
  if (!slot) slot = upload(p);
  return slot->v;
}

template <int W>
void launch_w(const DevView& v, const SampleArgs& a, cudaStream_t s) {
  const uint64_t blocks = (a.shots + kThreads - 1) / kThreads;
  if (blocks > 0x7FFFFFFFull) fail(TSIM_ERR_ARG, "too many shots for one launch");
  k_sample<W><<<(unsigned)blocks, kThreads, 0, s>>>(v, a.seed, a.shot_offset, a.shots, a.meas, a.det,
                                                     a.obs, a.accept);
}

}  // namespace

void device_sample(const Program& p, const SampleArgs& a, void* stream) {
  if (p.mode == TSIM_MODE_DETECTORS && a.meas) fail(TSIM_ERR_ARG, "measurement records requested from a detector-mode program");
  if (a.shots == 0) return;
  const DevView& v = ensure_uploaded(p);
  cudaStream_t s = (cudaStream_t)stream;
  switch (v.W) {
    case 1: launch_w<1>(v, a, s); break;
    case 2: launch_w<2>(v, a, s); break;
    case 4: launch_w<4>(v, a, s); break;
    case 8: launch_w<8>(v, a, s); break;
    case 16: launch_w<16>(v, a, s); break;
    case 32: launch_w<32>(v, a, s); break;
    default: fail(TSIM_ERR_INTERNAL, "unsupported word count");
  }
  TSIM_CUDA(cudaGetLastError());
}

void device_sample_batch(const Program* const* progs, int n, const SampleArgs* args, void* stream) {
  for (int i = 0; i < n; ++i) device_sample(*progs[i], args[i], stream);
}

void device_sync(void* stream) {
  TSIM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int st = 0;
  TSIM_CUDA(cudaMemcpyFromSymbol(&st, g_status, sizeof st));
  if (st) {
    int z = 0;
    TSIM_CUDA(cudaMemcpyToSymbol(g_status, &z, sizeof z));
    if (st & ST_ZERO_PROB) fail(TSIM_ERR_ZERO_PROB, "device: a sampled prefix had P_prev <= 0");
    if (st & ST_NOT_REAL) fail(TSIM_ERR_INTERNAL, "device: a marginal was not real");
    fail(TSIM_ERR_OVERFLOW_BOUND, "device: exact arithmetic overflow");
  }
}

}  // namespace tsim

// ------------------------------------------------------------------------
// Sampling without device allocation.
//
// Some callers cannot call cudaMalloc: code running inside a memory pool or
// allocator they do not own, real-time loops that must not touch the driver's
// allocator, or hosts whose device memory is carved up ahead of time.  For
// them tsim_sample_noalloc runs the same sampling kernel, but the program's
// device tables -- the scratch that tsim_sample allocates once per program --
// live in the fixed array below instead.  Its size is kNoAllocBytes (4 MiB);
// every GPU that loads the library holds it until the process exits.
namespace tsim {
namespace {

constexpr size_t kNoAllocBytes = (size_t)4 << 20;
constexpr int kNoAllocMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// host staging of the packed tables (filled under the mutex, then copied)
alignas(256) unsigned char g_noalloc_host[kNoAllocBytes];
std::mutex g_noalloc_mutex;
// device address of g_noalloc_scratch, per device, from cudaGetSymbolAddress
void* g_noalloc_dev[kNoAllocMaxDevices];

tsim_status noalloc_error(tsim_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

}  // namespace
}  // namespace tsim

extern "C" tsim_status tsim_sample_noalloc(const tsim_program* prog, uint64_t shots, uint64_t seed,
                                           uint64_t shot_offset, uint64_t* d_meas, uint64_t* d_det,
                                           uint64_t* d_obs, uint8_t* d_accept, void* cuda_stream) {
  using namespace tsim;
  if (!prog || !prog->p) return noalloc_error(TSIM_ERR_ARG, "NULL program");
  const Program& p = *prog->p;
  if (p.mode == TSIM_MODE_DETECTORS && d_meas)
    return noalloc_error(TSIM_ERR_ARG, "measurement records requested from a detector-mode program");
  if (shots == 0) return TSIM_OK;
  const uint64_t blocks = (shots + kThreads - 1) / kThreads;
  if (blocks > 0x7FFFFFFFull) return noalloc_error(TSIM_ERR_ARG, "too many shots for one launch");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices)
    return noalloc_error(TSIM_ERR_CUDA, "cudaGetDevice failed or device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_dev[dev]) {
    // once per device, with that device current: the host-side symbol is not
    // a device address, so the kernel must be given the address looked up here
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr)
      return noalloc_error(TSIM_ERR_CUDA, "cudaGetSymbolAddress of the no-alloc scratch array failed");
    g_noalloc_dev[dev] = ptr;
  }
  FixedSink sink{g_noalloc_host, kNoAllocBytes};
  Layout L;
  const char* msg = "";
  tsim_status st = pack_tables(p, sink, L, &msg);
  if (st != TSIM_OK) return noalloc_error(st, msg);
  if (sink.overflow)
    return noalloc_error(TSIM_ERR_ARG, "program tables exceed the 4 MiB maximum of tsim_sample_noalloc");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // every byte the kernel reads is rewritten here, so nothing stale from the
  // previous call survives
  if (cudaMemcpyAsync(g_noalloc_dev[dev], g_noalloc_host, L.total, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return noalloc_error(TSIM_ERR_CUDA, "cudaMemcpyAsync into the no-alloc scratch array failed");
  const DevView v = make_view((const unsigned char*)g_noalloc_dev[dev], L, p);
  const unsigned nb = (unsigned)blocks;
  switch (v.W) {
    case 1: k_sample<1><<<nb, kThreads, 0, s>>>(v, seed, shot_offset, shots, d_meas, d_det, d_obs, d_accept); break;
    case 2: k_sample<2><<<nb, kThreads, 0, s>>>(v, seed, shot_offset, shots, d_meas, d_det, d_obs, d_accept); break;
    case 4: k_sample<4><<<nb, kThreads, 0, s>>>(v, seed, shot_offset, shots, d_meas, d_det, d_obs, d_accept); break;
    case 8: k_sample<8><<<nb, kThreads, 0, s>>>(v, seed, shot_offset, shots, d_meas, d_det, d_obs, d_accept); break;
    case 16: k_sample<16><<<nb, kThreads, 0, s>>>(v, seed, shot_offset, shots, d_meas, d_det, d_obs, d_accept); break;
    case 32: k_sample<32><<<nb, kThreads, 0, s>>>(v, seed, shot_offset, shots, d_meas, d_det, d_obs, d_accept); break;
    default: return noalloc_error(TSIM_ERR_INTERNAL, "unsupported word count");
  }
  if (cudaGetLastError() != cudaSuccess) return noalloc_error(TSIM_ERR_CUDA, "launch of the sampling kernel failed");
  return TSIM_OK;
}
