// GB300 (sm_103a) per-shot sampling kernels.
//
// One thread carries one shot end to end (Sec. "Complexity", paragraph
// "Sampling"):
//   1. error mechanisms: one Philox4x32-10 word per reduced channel, outcome by
//      integer threshold compare, X ^= column signature (Eq. detector_sampling);
//   2. outputs in autoregressive order: deterministic outputs are GF(2)
//      parities of X = (f, random outputs); random outputs follow Algorithm 1,
//      every marginal P = sum_t c^t prod_k h(...) evaluated exactly, in one of
//      two ways:
//        - per thread: the distinct factor parities of the table (Eq.
//          parities) are computed once per shot by AND + popcount; terms with
//          identical factor lists are merged ahead of time into one class;
//          per class each factor's two parity bits select one of four packed
//          (zero, sqrt2-exponent, w-exponent) increments, and the class value
//          C w^J sqrt2^S or 0 is accumulated into four int64 coefficients of
//          Z[w] (no floating point);
//        - per warp, bit-sliced (tables of Node, phase and pi-pair factors):
//          the warp's 32 shots share every 32-bit word, lane l carries term l
//          of a batch of 32, and each factor is one or two word operations on
//          the term's phase exponent mod 8 and vanishing flag (below);
//   3. the Bernoulli draw compares U * P_prev with 2^32 * P_1 exactly (int128);
//   4. bit-packed records (runs of single-bit detectors copied by word shifts).
// The program tables are read-only; per-thread table loads are uniform
// (broadcast) loads, the bit-sliced rows are lane-coalesced 16-byte loads.
// k_sample launches one program; k_batch runs persistent warps over the
// (program, shot-block) work items of many programs.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <unordered_map>

#include "device.h"
#include "zx.h"

namespace tsim {

#define TSIM_CUDA(x)                                                                  \
  do {                                                                                \
    cudaError_t e_ = (x);                                                             \
    if (e_ != cudaSuccess) fail(TSIM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

enum : int { ST_NOT_REAL = 1, ST_OVERFLOW = 2, ST_ZERO_PROB = 4, ST_TIMEOUT = 8 };

// device-wide status word: bits of the conditions above, read by tsim_sync
__device__ int g_status;

constexpr int kMaxChains = 16;
constexpr int kMaxOutWords = 64;  // measurement mode: 4096 outputs
constexpr int kMaxParities = 256;
constexpr int kThreads = 128;

// Output entries, in autoregressive order.  rec is the output index (its
// record bit); a run (detector mode) covers outputs rec .. rec + chain - 1,
// which are X bits a .. a + chain - 1 with no constant, in one record.
enum : int { OUT_MASK = 0, OUT_BIT = 1, OUT_RANDOM = 2, OUT_RUN = 3 };

struct DChan { uint32_t n_out, thr_off, sig_off, thr0; };
struct DOut { int32_t kind, cst, a, chain, table, rec; };
// Table layouts: SCALAR = distinct parities indexed per factor (one thread
// per shot), BASIS = parities as coordinates in a GF(2) basis of their span,
// SLICED = warp-cooperative bit-sliced evaluation (below).
enum : int { TAB_SCALAR = 0, TAB_BASIS = 1, TAB_SLICED = 2 };
struct DTable { uint32_t par_off, n_par, cls_off, n_cls; int32_t base, mode, sb_off, n_sb, stage, pad[3]; };
struct DClass { uint32_t fac_off, n_fac; int32_t mono, j0, d0, pad; long long c[4]; };

// Bit-sliced tables.  A warp evaluates 32 shots at once: bit s of every
// 32-bit word below belongs to shot (lane) s.  Per table the warp forms the
// words Par[q] of all distinct factor parities q (Eq. parities), then walks
// the terms in batches of 32, lane l carrying term l of the batch.  Every
// factor of a Clifford term whose value is a monomial of fixed magnitude
// reduces to operations on the term's phase exponent J (mod 8, three bit
// planes J0 J1 J2) and vanishing flag Z:
enum : int {
  SL_XOR4 = 0,   // J += 4a          (a sign (-1)^a)
  SL_ADD2 = 1,   // J += 2a          (i^a)
  SL_ADD6 = 2,   // J += 6a          ((-i)^a)
  SL_XOR4AB = 3, // J += 4ab         (pi-pair (-1)^(ab)); row = qa | qb << 16
  SL_ZERO = 4,   // vanishes if a = 1 (Node 1 + (-1)^a)
  SL_ZEROC = 5,  // vanishes if a = 0 (Node 1 - (-1)^a)
  SL_ADD1 = 6,   // J += a           (w^a, odd phase)
  kSlCodes = 7
};
constexpr uint32_t kSlOnes = 1;        // parity index whose word is all ones
constexpr int kSlMaxPar = 16384;       // parity words of one segment (4q fits 16 bits)
// One batch of 32 terms: rows of operation code c are cnt[c] (a multiple of
// 4) x 32 parity offsets, padded with no-op offsets and stored in groups of 4
// rows as [group][lane][4], starting at row_off.
// All terms of a batch share the magnitude sqrt2^d; j0m[b] holds bit b of
// each lane's constant phase; valid marks lanes that carry a term.
struct DSBatch { uint32_t row_off; uint16_t cnt[8]; int32_t d; uint32_t j0m[3]; uint32_t valid; };
// A sliced table is a list of segments: consecutive terms whose distinct
// parities (par_off, n_par masks) fit one shared buffer, and their batches.
struct DSeg { uint32_t par_off, n_par, sb_off, n_sb; };

struct DevView {
  int W;
  int n_ch, n_out, n_ent, n_chains, n_tab;
  int nmeas, ndet, nobs, mode;
  const DChan* ch;
  const uint4* thr0;      // outcome-0 threshold per channel, 4 per block, padded with 2^32-1
  const uint32_t* thr;
  const uint64_t* sig;
  const DOut* out;
  const uint64_t* omask;
  const int32_t* chain_norm;
  const DTable* tab;
  const uint64_t* par;    // per table: n_par masks of W words (mask 0 = zero)
  const DClass* cls;
  const uint32_t* fidx;   // per factor: parity index of a | parity index of b << 8
  const uint32_t* finc;   // per factor: 4 packed increments
  const uint64_t* fcoord; // basis tables: per factor the coordinates of a and b (2 words)
  const DSeg* seg;        // sliced tables: segments
  const DSBatch* sb;      // sliced tables: batches
  const uint32_t* rows;   // sliced tables: operation rows
  int sl_par;             // shared words for parity words per warp (0: no sliced table)
  int sl_rb;              // shared words of one row staging buffer (0: no staging)
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
  // strip common factors 2 = sqrt2^2; a monomial then has the coefficient
  // pattern of w^j (one entry +-1) or of sqrt2 w^j = w^(j+1) - w^(j+3)
  // (entries +-1 two places apart)
  __int128 c[4] = {v.c[0], v.c[1], v.c[2], v.c[3]};
  int k = v.k;
  while (!(c[0] & 1) && !(c[1] & 1) && !(c[2] & 1) && !(c[3] & 1)) {
    for (auto& x : c) x /= 2;
    k += 2;
  }
  int nz = 0;
  for (auto x : c) nz += x != 0;
  for (int jj = 0; jj < 8; ++jj) {
    ZW m1 = ZW::omega(jj);
    if (nz == 1 && m1.c[0] == c[0] && m1.c[1] == c[1] && m1.c[2] == c[2] && m1.c[3] == c[3]) {
      *s = k;
      *j = jj;
      return true;
    }
    ZW a = ZW::omega(jj + 1), b = ZW::omega(jj + 3);
    bool eq = nz == 2;
    for (int i = 0; i < 4 && eq; ++i) eq = (a.c[i] - b.c[i]) == c[i];
    if (eq) {
      *s = k + 1;
      *j = jj;
      return true;
    }
  }
  return false;
}

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 products;
// the round keys (key + r * Weyl constants) are the same for every call.
struct RoundKeys {
  uint32_t k0[10], k1[10];
};

// the round keys of key (seed lo, seed hi): key + r * (0x9E3779B9, 0xBB67AE85)
__host__ __device__ __forceinline__ RoundKeys round_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = k0;
    rk.k1[r] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return rk;
}

__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              const RoundKeys& rk, uint32_t o[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    c0 = hi1 ^ c1 ^ rk.k0[r];
    c1 = lo1;
    c2 = hi0 ^ c3 ^ rk.k1[r];
    c3 = lo0;
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

// coefficient k (0..7) of w^k in Z[w] basis {1, w, w^2, w^3}: w^k = +-w^(k mod 4)
__device__ __forceinline__ long long pick(const long long c[4], int k) {
  k &= 7;
  const int q = k & 3;
  const long long v = q == 0 ? c[0] : (q == 1 ? c[1] : (q == 2 ? c[2] : c[3]));
  return k < 4 ? v : -v;
}

// parity of (mask & X); masks are stored with ws words (ws <= W, the rest of X
// is zero for such a program)
template <int W>
__device__ __forceinline__ int parity_w(const uint64_t* m, const uint64_t (&X)[W], int ws) {
  uint64_t acc = 0;
#pragma unroll
  for (int w = 0; w < W; ++w)
    if (w < ws) acc ^= __ldg(m + w) & X[w];
  return __popcll(acc) & 1;
}

// exact table value (c0 + c1 w + c2 w^2 + c3 w^3) sqrt2^base
struct ZC {
  long long c[4];
  int base;
};

// real part of w^-rot (c0 + c1 w + c2 w^2 + c3 w^3) sqrt2^base as
// (A + B sqrt2) 2^e:  Re = (2 c0 + (c1 - c3) sqrt2) / 2.  A chain's tables
// share one parameter-dependent phase w^rot (the discarded scalars that the
// normalisation P restores, Sec. "Observables"); rotating it away leaves the
// real marginal.
__device__ __forceinline__ RV to_real_rot(const ZC& z, int rot, int* st) {
  long long c[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) c[i] = pick(z.c, i + rot);
  const int base = z.base;
  if (c[2] != 0 || c[1] + c[3] != 0) *st |= ST_NOT_REAL;
  RV r;
  r.A = (__int128)2 * c[0];
  r.B = (__int128)c[1] - c[3];
  int K = base - 2;
  if (K & 1) {
    const __int128 t2 = r.A;
    r.A = 2 * r.B;
    r.B = t2;
    K -= 1;
  }
  r.e = K / 2;
  return r;
}

// value w^J sqrt2^d C of one merged term, added into the four Z[w] coefficients
__device__ __forceinline__ void accumulate(const DClass& C, uint32_t acc, long long (&c)[4]) {
  const int J = (C.j0 + (int)(acc & 0x7FF)) & 7;
  const int d = C.d0 + (int)((acc >> 11) & 0x3FF);
  const int sh = d >> 1;
  if (C.mono) {
    const long long mag = 1ll << sh;
    if (d & 1) {  // sqrt2 w^J = w^(J+1) - w^(J+3)
      const int a = (J + 1) & 7, b = (J + 3) & 7;
      c[a & 3] += (a < 4) ? mag : -mag;
      c[b & 3] -= (b < 4) ? mag : -mag;
    } else {
      c[J & 3] += (J < 4) ? mag : -mag;
    }
  } else {
    // w^J C: coefficient i takes C's coefficient of w^(i - J)
    long long r[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) r[i] = pick(C.c, i - J + 8);
    if (d & 1) {  // times sqrt2 = w - w^3
      const long long t0 = r[1] - r[3], t1 = r[0] + r[2], t2 = r[1] + r[3], t3 = r[2] - r[0];
      r[0] = t0; r[1] = t1; r[2] = t2; r[3] = t3;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) c[i] += r[i] * (1ll << sh);
  }
}

// ---- shared-memory staging of operation rows (bulk copies through the
// tensor memory accelerator, completion tracked by an mbarrier per buffer)
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t lds(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// one elected lane: expect `bytes` on the barrier and start the bulk copy
// (global source and shared destination 16-byte aligned, bytes a multiple of 16)
// (no copy for 0 bytes: the arrival alone completes the phase)
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  if (bytes)
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Warp-uniform bounded wait for the phase of the given parity; false when it
// did not complete within the limit (the caller reports ST_TIMEOUT).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 22); ++it)
    if (__all_sync(0xFFFFFFFFu, mbar_test(bar, parity))) return true;
  return false;
}

// A warp's shared words for sliced tables: transposed X (64 W), parity words
// (par), two row staging buffers (rb each), two mbarriers and a state word
// (bit 0 / 1: next phase parity of buffer 0 / 1; bit 2: staging failed).
struct SlSmem {
  uint32_t xs, par, rb0, rb1, bar0, bar1, state;
  int rb;
};

__host__ __device__ __forceinline__ int sl_round32(int x) { return (x + 31) & ~31; }

__host__ __device__ __forceinline__ int sl_warp_words(int W, int par, int rb) {
  if (par <= 0) return 0;
  return sl_round32(64 * W + par) + (rb > 0 ? 2 * rb + 32 : 0);
}

__device__ __forceinline__ SlSmem sl_smem(uint32_t* warp_base, int W, int par, int rb) {
  SlSmem m;
  const uint32_t b = smem_u32(warp_base);
  m.xs = b;
  m.par = b + 4u * (uint32_t)(64 * W);
  const uint32_t st = b + 4u * (uint32_t)sl_round32(64 * W + par);
  m.rb0 = st;
  m.rb1 = st + 4u * (uint32_t)rb;
  m.bar0 = st + 8u * (uint32_t)rb;
  m.bar1 = m.bar0 + 8;
  m.state = m.bar0 + 16;
  m.rb = rb;
  return m;
}

// once per warp at kernel start, when rows are staged
__device__ __forceinline__ void sl_init(const SlSmem& m) {
  if (m.rb > 0) {
    if ((threadIdx.x & 31) == 0) {
      mbar_init(m.bar0, 1);
      mbar_init(m.bar1, 1);
      asm volatile("st.shared.u32 [%0], %1;" ::"r"(m.state), "r"(0u) : "memory");
      fence_mbar_init();
    }
    __syncwarp();
  }
}

// 32 x 32 bit-matrix transpose across the warp: on entry lane r holds row r
// (bit c = column c), on exit lane c holds column c (bit r = row r).  Stage j
// (16, 8, 4, 2, 1) swaps the off-diagonal j x j blocks between lanes r and
// r ^ j: each lane sends the half its partner keeps, and rotates what it
// receives into place (left by j in the lower lane, right by j in the upper
// one; the received bits never wrap).
struct Transposer {
  uint32_t mk[5];   // the bits a lane keeps at each stage
  uint32_t rot[5];  // left-rotation of the received bits
  __device__ __forceinline__ explicit Transposer(int lane) {
    const uint32_t keep[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int st = 0; st < 5; ++st) {
      const int j = 16 >> st;
      const bool upper = (lane & j) != 0;
      mk[st] = upper ? ~keep[st] : keep[st];
      rot[st] = upper ? 32u - (uint32_t)j : (uint32_t)j;
    }
  }
  __device__ __forceinline__ uint32_t operator()(uint32_t x) const {
#pragma unroll
    for (int st = 0; st < 5; ++st) {
      const uint32_t recv = __shfl_xor_sync(0xFFFFFFFFu, x & ~mk[st], 16 >> st);
      x = (x & mk[st]) | __funnelshift_l(recv, recv, rot[st]);
    }
    return x;
  }
};

// Operation rows read from global memory (through L1) or from a shared
// staging buffer.  A row holds the byte offset of a parity word (4q), or two
// of them (4qa | 4qb << 16) for pi-pairs.  Rows come in groups of 4: group g
// of a code is 32 lanes x 4 consecutive rows, so one 16-byte load per lane
// fetches 4 rows and a warp's load is 512 contiguous bytes.
struct RowsG {
  const uint4* p;  // this lane's current group
  __device__ __forceinline__ uint4 get4(int g) const { return __ldg(p + 32 * g); }
  __device__ __forceinline__ void adv4(int k) { p += 32 * k; }
};
struct RowsS {
  uint32_t a;  // shared address of this lane's current group
  __device__ __forceinline__ uint4 get4(int g) const {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(a + 512u * (uint32_t)g));
    return v;
  }
  __device__ __forceinline__ void adv4(int k) { a += 512u * (uint32_t)k; }
};

// The n rows (a multiple of 4) of one operation code, in chunks whose row
// loads and parity loads are all issued before the updates; f(way, a, b)
// spreads consecutive rows over 4 independent accumulators (way = row & 3)
// so that the update chains overlap.
template <bool PAIR, class Rows, class F>
__device__ __forceinline__ void sl_loop(int n, Rows& R, uint32_t par, F&& f) {
  int k = 0;
  for (; k + 16 <= n; k += 16, R.adv4(4)) {
    uint32_t r[16], a[16], b[16];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const uint4 v = R.get4(g);
      r[4 * g] = v.x;
      r[4 * g + 1] = v.y;
      r[4 * g + 2] = v.z;
      r[4 * g + 3] = v.w;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      a[i] = lds(par + (PAIR ? (r[i] & 0xFFFFu) : r[i]));
      b[i] = PAIR ? lds(par + (r[i] >> 16)) : 0u;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) f(i & 3, a[i], b[i]);
  }
  for (; k < n; k += 4, R.adv4(1)) {
    const uint4 v = R.get4(0);
    const uint32_t r[4] = {v.x, v.y, v.z, v.w};
    uint32_t a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[i] = lds(par + (PAIR ? (r[i] & 0xFFFFu) : r[i]));
      b[i] = PAIR ? lds(par + (r[i] >> 16)) : 0u;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) f(i, a[i], b[i]);
  }
}

// (x1, x2) += (y1, y2) for 2-bit bit-sliced counters mod 4
__device__ __forceinline__ void add2bit(uint32_t& x1, uint32_t& x2, uint32_t y1, uint32_t y2) {
  x2 ^= y2 ^ (x1 & y1);
  x1 ^= y1;
}

// All operation rows of one batch; returns the planes (J0, J1, J2, Z).
template <class Rows>
__device__ __forceinline__ void sl_batch(const DSBatch& B, Rows R, uint32_t par, int lane, uint32_t& J0, uint32_t& J1,
                                         uint32_t& J2, uint32_t& Z) {
  J0 = 0u - ((B.j0m[0] >> lane) & 1u);
  J1 = 0u - ((B.j0m[1] >> lane) & 1u);
  J2 = 0u - ((B.j0m[2] >> lane) & 1u);
  Z = 0u - ((~B.valid >> lane) & 1u);
  // per way: J2 flips k, vanishing flags z, and a 2-bit counter (c1, c2) of
  // the rows that add 2 to J (J2 flips and vanishing flags commute with it)
  uint32_t k[4] = {0, 0, 0, 0}, z[4] = {0, 0, 0, 0}, c1[4] = {0, 0, 0, 0}, c2[4] = {0, 0, 0, 0};
  sl_loop<false>(B.cnt[SL_XOR4], R, par, [&](int w, uint32_t a, uint32_t) { k[w] ^= a; });
  sl_loop<false>(B.cnt[SL_ADD2], R, par, [&](int w, uint32_t a, uint32_t) {
    c2[w] ^= c1[w] & a;
    c1[w] ^= a;
  });
  // J += 6a = 2a + 4a
  sl_loop<false>(B.cnt[SL_ADD6], R, par, [&](int w, uint32_t a, uint32_t) {
    c2[w] ^= c1[w] & a;
    c1[w] ^= a;
    k[w] ^= a;
  });
  sl_loop<true>(B.cnt[SL_XOR4AB], R, par, [&](int w, uint32_t a, uint32_t b) { k[w] ^= a & b; });
  sl_loop<false>(B.cnt[SL_ZERO], R, par, [&](int w, uint32_t a, uint32_t) { z[w] |= a; });
  sl_loop<false>(B.cnt[SL_ZEROC], R, par, [&](int w, uint32_t a, uint32_t) { z[w] |= ~a; });
  add2bit(c1[0], c2[0], c1[1], c2[1]);
  add2bit(c1[2], c2[2], c1[3], c2[3]);
  add2bit(c1[0], c2[0], c1[2], c2[2]);
  add2bit(J1, J2, c1[0], c2[0]);
  J2 ^= (k[0] ^ k[1]) ^ (k[2] ^ k[3]);
  Z |= (z[0] | z[1]) | (z[2] | z[3]);
  // J += a (odd phases; rare): a three-plane increment
  sl_loop<false>(B.cnt[SL_ADD1], R, par, [&](int, uint32_t a, uint32_t) {
    const uint32_t cy = J0 & a;
    J0 ^= a;
    J2 ^= J1 & cy;
    J1 ^= cy;
  });
}

__device__ __forceinline__ uint32_t sl_batch_rows(const DSBatch& B) {
  uint32_t n = 0;
#pragma unroll
  for (int c = 0; c < kSlCodes; ++c) n += B.cnt[c];
  return n;
}

// Warp-cooperative exact value of a sliced table for the 32 shots of the
// warp (every lane must call it; lane s receives shot s's value).
template <int W>
__device__ ZC eval_table_sliced(const DevView& V, const DTable& tb, const uint64_t (&X)[W], const SlSmem& S) {
  const int lane = threadIdx.x & 31;
  const Transposer transpose32(lane);
  __syncwarp();
  uint32_t state = S.rb > 0 ? lds(S.state) : 4u;
  const bool staged = tb.stage && !(state & 4u);
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const uint32_t lo = transpose32((uint32_t)X[w]), hi = transpose32((uint32_t)(X[w] >> 32));
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(S.xs + 4u * (uint32_t)(64 * w + lane)), "r"(lo) : "memory");
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(S.xs + 4u * (uint32_t)(64 * w + 32 + lane)), "r"(hi) : "memory");
  }
  ZC z{{0, 0, 0, 0}, tb.base};
  long long (&c)[4] = z.c;
  bool ok = true;
  // signed counts of the batches since the magnitude sqrt2^d last changed
  // (batches are sorted by d within a segment; |n| <= 32 per batch)
  int n[4] = {0, 0, 0, 0};
  int d_cur = 0;
  auto flush = [&]() {
    const int sh = d_cur >> 1;
    long long r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      r[q] = (long long)n[q] << sh;
      n[q] = 0;
    }
    if (d_cur & 1) {  // times sqrt2 = w - w^3
      c[0] += r[1] - r[3];
      c[1] += r[0] + r[2];
      c[2] += r[1] + r[3];
      c[3] += r[2] - r[0];
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) c[q] += r[q];
    }
  };
  const int ws = V.W;  // masks have V.W <= W words (a batched launch may run with a larger W)
  uint32_t bi = 0;     // batches so far: the staging buffer alternates with it
  for (int g = 0; g < tb.n_sb; ++g) {
    const DSeg sg = V.seg[tb.sb_off + g];
    const DSBatch* bt = V.sb + sg.sb_off;
    DSBatch next = sg.n_sb > 0 ? bt[0] : DSBatch{};
    __syncwarp();  // every lane is done with the previous segment's parity words
    // rows of batches that fit the buffers go through shared memory; the
    // segment's first copy overlaps its parity computation below
    if (staged && ok && lane == 0 && sg.n_sb > 0) {
      fence_proxy_async();
      bulk_load((bi & 1) ? S.rb1 : S.rb0, V.rows + next.row_off, 128u * sl_batch_rows(next), (bi & 1) ? S.bar1 : S.bar0);
    }
    // the segment's parities as XORs of the X bits in their masks, 32 shots
    // at once; four per lane at a time so that their mask loads overlap
    const uint64_t* pm = V.par + (size_t)sg.par_off * ws;
    for (uint32_t q0 = lane; q0 < sg.n_par; q0 += 128) {
      uint64_t m[4][W];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t q = q0 + 32u * (uint32_t)u;
#pragma unroll
        for (int w = 0; w < W; ++w) m[u][w] = (w < ws && q < sg.n_par) ? __ldg(pm + (size_t)q * ws + w) : 0ull;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t q = q0 + 32u * (uint32_t)u;
        uint32_t acc = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
          uint64_t x = m[u][w];
          while (x) {
            acc ^= lds(S.xs + 4u * (uint32_t)(64 * w + __ffsll((long long)x) - 1));
            x &= x - 1;
          }
        }
        if (q < sg.n_par)
          asm volatile("st.shared.u32 [%0], %1;" ::"r"(S.par + 4u * q), "r"(q == kSlOnes ? 0xFFFFFFFFu : acc)
                       : "memory");
      }
    }
    __syncwarp();
    for (uint32_t b = 0; b < sg.n_sb; ++b, ++bi) {
      const DSBatch B = next;
      if (b + 1 < sg.n_sb) next = bt[b + 1];  // the next header's load overlaps this batch
      uint32_t J0, J1, J2, Z;
      if (staged && ok) {
        const uint32_t buf = bi & 1;
        // the other buffer held the previous batch, which every lane has finished
        if (lane == 0 && b + 1 < sg.n_sb) {
          fence_proxy_async();
          bulk_load(buf ? S.rb0 : S.rb1, V.rows + next.row_off, 128u * sl_batch_rows(next), buf ? S.bar0 : S.bar1);
        }
        const uint32_t bar = buf ? S.bar1 : S.bar0;
        if (!mbar_wait_bounded(bar, (state >> buf) & 1u)) {
          // a copy that does not land in time: report it, let the copies in
          // flight finish (bounded), and read rows from global memory
          if (lane == 0) atomicOr(&g_status, ST_TIMEOUT);
          mbar_wait_bounded(S.bar0, state & 1u);
          mbar_wait_bounded(S.bar1, (state >> 1) & 1u);
          ok = false;
          state |= 4u;
        } else {
          state ^= 1u << buf;
          sl_batch(B, RowsS{(buf ? S.rb1 : S.rb0) + 16u * (uint32_t)lane}, S.par, lane, J0, J1, J2, Z);
        }
      }
      if (!staged || !ok)
        sl_batch(B, RowsG{reinterpret_cast<const uint4*>(V.rows + B.row_off) + lane}, S.par, lane, J0, J1, J2, Z);
      if (staged) __syncwarp();  // the buffer just read is refilled next batch
      // lane s now needs, for each of the 32 terms, its phase and flag at shot s
      const uint32_t T0 = transpose32(J0), T1 = transpose32(J1);
      const uint32_t T2 = transpose32(J2), TZ = transpose32(Z);
      const uint32_t nz = ~TZ;
      const uint32_t M[4] = {~T0 & ~T1 & nz, T0 & ~T1 & nz, ~T0 & T1 & nz, T0 & T1 & nz};
      if (B.d != d_cur) {
        flush();
        d_cur = B.d;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)  // terms with J = q count +1, with J = q + 4 count -1
        n[q] += __popc(M[q]) - 2 * __popc(M[q] & T2);
    }
  }
  flush();
  if (S.rb > 0) {
    __syncwarp();
    if (lane == 0) asm volatile("st.shared.u32 [%0], %1;" ::"r"(S.state), "r"(state) : "memory");
    __syncwarp();
  }
  return z;
}

// SL: the program has sliced tables (kernels without them never contain the
// warp-cooperative code and keep their register budget)
template <int W, bool SL>
__device__ ZC eval_table(const DevView& V, int t, const uint64_t (&X)[W], const SlSmem& sm) {
  const DTable tb = V.tab[t];
  if constexpr (SL) {
    if (tb.mode == TAB_SLICED) return eval_table_sliced<W>(V, tb, X, sm);
  }
  ZC z{{0, 0, 0, 0}, tb.base};
  long long (&c)[4] = z.c;
  if (tb.mode == TAB_BASIS) {
    // parities in a GF(2) basis of the table's mask span: Y holds the basis
    // parities and every factor parity is <coordinates, Y>
    uint64_t Y = 0;
    for (uint32_t q = 0; q < tb.n_par; ++q)
      Y |= (uint64_t)parity_w<W>(V.par + (size_t)(tb.par_off + q) * V.W, X, V.W) << q;
    for (uint32_t q = 0; q < tb.n_cls; ++q) {
      const DClass& C = V.cls[tb.cls_off + q];
      const uint32_t fo = C.fac_off, nf = C.n_fac;
      uint32_t acc = 0;
      for (uint32_t k = 0; k < nf; ++k) {
        const uint64_t ua = __ldg(V.fcoord + 2 * (size_t)(fo + k)), ub = __ldg(V.fcoord + 2 * (size_t)(fo + k) + 1);
        const uint32_t a = __popcll(ua & Y) & 1, b = __popcll(ub & Y) & 1;
        acc += __ldg(V.finc + (size_t)(fo + k) * 4 + (a | (b << 1)));
      }
      if (acc >> 21) continue;
      accumulate(C, acc, c);
    }
    return z;
  }
  // distinct factor parities of this table, once per shot, into 256 bits
  // (q is the same for every thread of a warp, so the word choice is uniform)
  uint64_t P0 = 0, P1 = 0, P2 = 0, P3 = 0;
  for (uint32_t q = 1; q < tb.n_par; ++q) {
    const uint64_t bit = (uint64_t)parity_w<W>(V.par + (size_t)(tb.par_off + q) * V.W, X, V.W) << (q & 63);
    if (q < 64) P0 |= bit;
    else if (q < 128) P1 |= bit;
    else if (q < 192) P2 |= bit;
    else P3 |= bit;
  }
  auto pbit = [&](uint32_t i) -> uint32_t {
    const uint64_t w = i < 128 ? (i < 64 ? P0 : P1) : (i < 192 ? P2 : P3);
    return (uint32_t)((w >> (i & 63)) & 1);
  };
  for (uint32_t q = 0; q < tb.n_cls; ++q) {
    const DClass& C = V.cls[tb.cls_off + q];
    const uint32_t fo = C.fac_off, nf = C.n_fac;
    uint32_t acc = 0;
    for (uint32_t k = 0; k < nf; ++k) {
      const uint32_t ix = __ldg(V.fidx + fo + k);
      const uint32_t ia = ix & 0xFF, ib = (ix >> 8) & 0xFF;
      const uint32_t a = pbit(ia), b = pbit(ib);
      acc += __ldg(V.finc + (size_t)(fo + k) * 4 + (a | (b << 1)));
    }
    if (acc >> 21) continue;  // some factor vanished
    accumulate(C, acc, c);
  }
  return z;
}

// the power of w that makes a chain's normalisation real and positive
__device__ __forceinline__ int chain_rotation(const ZC& z, int* st) {
  for (int rot = 0; rot < 8; ++rot) {
    long long c[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) c[i] = pick(z.c, i + rot);
    if (c[2] == 0 && c[1] + c[3] == 0) {
      const __int128 A = (__int128)2 * c[0], B = (__int128)c[1] - c[3];
      if (sign_xy(A, B, st) > 0) return rot;
    }
  }
  *st |= ST_NOT_REAL;
  return 0;
}

template <int W>
__device__ __forceinline__ void set_xbit(uint64_t (&X)[W], int b, bool on) {
#pragma unroll
  for (int w = 0; w < W; ++w)
    if (w == (b >> 6)) X[w] = on ? (X[w] | (1ull << (b & 63))) : (X[w] & ~(1ull << (b & 63)));
}

template <int W>
__device__ __forceinline__ int get_xbit(const uint64_t (&X)[W], int b) {
  uint64_t v = 0;
#pragma unroll
  for (int w = 0; w < W; ++w)
    if (w == (b >> 6)) v = X[w];
  return (int)((v >> (b & 63)) & 1);
}

// `take` (1..64) bits of X starting at bit x
template <int W>
__device__ __forceinline__ uint64_t get_xbits(const uint64_t (&X)[W], int x, int take) {
  const int wi = x >> 6, sh = x & 63;
  uint64_t lo = 0, hi = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    if (w == wi) lo = X[w];
    if (w == wi + 1) hi = X[w];
  }
  const uint64_t v = sh ? (lo >> sh) | (hi << (64 - sh)) : lo;
  return take >= 64 ? v : v & ((1ull << take) - 1);
}

// One shot s of a launch (global shot index shot0 + s), records at row s.
// Every lane of a warp calls it together (sliced tables are evaluated by the
// whole warp); lanes past the end of the launch have valid = false and
// compute a shot whose records are not written.  sm: the warp's shared words.
template <int W, bool SL>
__device__ void sample_one(const DevView& V, uint64_t s, bool valid, const RoundKeys& rk, uint64_t shot0,
                           uint64_t* __restrict__ meas, uint64_t* __restrict__ det,
                           uint64_t* __restrict__ obs, uint8_t* __restrict__ accept, const SlSmem& sm) {
  const uint64_t shot = shot0 + s;
  const uint32_t c0 = (uint32_t)shot, c1 = (uint32_t)(shot >> 32);
  int st = 0;

  // 1. error mechanisms and f = T e
  uint64_t X[W];
#pragma unroll
  for (int w = 0; w < W; ++w) X[w] = 0;
  // four channels per Philox block: their outcome-0 thresholds in one
  // 16-byte load and one test; the rare block where some channel fires walks
  // its channels
  for (int c = 0; c < V.n_ch; c += 4) {
    uint32_t u[4];
    philox4x32_10(c0, c1, 0u, (uint32_t)(c >> 2), rk, u);
    const uint4 t0 = __ldg(V.thr0 + (c >> 2));
    if (!((u[0] >= t0.x) | (u[1] >= t0.y) | (u[2] >= t0.z) | (u[3] >= t0.w))) continue;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int ci = c + l;
      if (ci >= V.n_ch) break;
      const DChan ch = V.ch[ci];
      const uint32_t U = u[l];
      if (U < ch.thr0) continue;  // outcome 0: nothing fires
      const uint32_t* thr = V.thr + ch.thr_off;
      uint32_t o = 1;
      while (o + 1 < ch.n_out && U >= __ldg(thr + o)) ++o;
      if (o >= ch.n_out) continue;
      const uint64_t* sg = V.sig + ch.sig_off + (size_t)o * V.W;
#pragma unroll
      for (int w = 0; w < W; ++w)
        if (w < V.W) X[w] ^= __ldg(sg + w);
    }
  }

  // 2-3. outputs in autoregressive order (Algorithm 1 per chain)
  RV pp[kMaxChains];
  int rot[kMaxChains];
  for (int c = 0; c < V.n_chains; ++c) {
    const ZC z = eval_table<W, SL>(V, V.chain_norm[c], X, sm);
    rot[c] = chain_rotation(z, &st);
    pp[c] = to_real_rot(z, rot[c], &st);
  }
  const int dw = (V.ndet + 63) >> 6, mw = (V.nmeas + 63) >> 6, ow = (V.nobs + 63) >> 6;
  uint64_t ob[kMaxOutWords];  // measurement mode only
  uint64_t cur = 0;  // detector mode: record word cw (detector words, then observable words)
  int cw = -1;
  bool any_det = false;
  auto flush = [&]() {
    if (cw < 0) return;
    if (cw < dw) {
      any_det |= cur != 0;
      if (det && valid) det[s * dw + cw] = cur;
    } else if (obs && valid) {
      obs[s * ow + (cw - dw)] = cur;
    }
    cur = 0;
  };
  // bits of outputs i, i + 1, ... (within one record word) into the record
  auto put = [&](int i, uint64_t bits) {
    const bool is_det = i < V.ndet;
    const int j = is_det ? i : i - V.ndet;
    const int gw = is_det ? (j >> 6) : dw + (j >> 6);
    if (gw != cw) {
      flush();
      cw = gw;
    }
    cur |= bits << (j & 63);
  };
  for (int e = 0; e < V.n_ent; ++e) {
    const DOut o = V.out[e];
    const int i = o.rec;
    if (o.kind == OUT_RUN) {  // consecutive X bits straight into the record
      int ii = i, x = o.a, n = o.chain;
      while (n > 0) {
        const int j = ii < V.ndet ? ii : ii - V.ndet;
        const int take = min(n, 64 - (j & 63));
        put(ii, get_xbits<W>(X, x, take));
        ii += take;
        x += take;
        n -= take;
      }
      continue;
    }
    int bit;
    if (o.kind == OUT_BIT) {
      bit = get_xbit<W>(X, o.a) ^ o.cst;
    } else if (o.kind == OUT_MASK) {
      bit = parity_w<W>(V.omask + o.a, X, V.W) ^ o.cst;
    } else {
      set_xbit<W>(X, o.a, true);
      const RV p1 = to_real_rot(eval_table<W, SL>(V, o.table, X, sm), rot[o.chain], &st);
      const RV pv = pp[o.chain];
      if (sign_xy(pv.A, pv.B, &st) <= 0) st |= ST_ZERO_PROB;
      uint32_t u[4];
      philox4x32_10(c0, c1, 1u, (uint32_t)(i >> 2), rk, u);
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
        set_xbit<W>(X, o.a, false);
      }
    }
    if (V.mode == 0) {
      put(i, (uint64_t)bit);  // detectors are outputs [0, ndet), observables [ndet, ndet + nobs)
    } else {
      if ((i & 63) == 0) ob[i >> 6] = 0;
      ob[i >> 6] |= (uint64_t)bit << (i & 63);
    }
  }
  if (V.mode == 0) flush();

  // 4. measurement-mode records
  if (V.mode != 0) {
    if (meas && valid)
      for (int w = 0; w < mw; ++w) meas[s * mw + w] = ob[w];
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
      if (det && valid) det[s * dw + w] = v;
    }
    if (obs && valid)
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
  if (!valid) return;
  if (accept) accept[s] = any_det ? 0 : 1;
  if (st) atomicOr(&g_status, st);
}

// dynamic shared memory: sl_warp_words(...) per warp for programs with sliced tables
extern __shared__ __align__(128) uint32_t g_warp_smem[];

// Register bounds (resident blocks of up to 128 threads per SM) for X of up
// to 4 words: kernels for programs with sliced tables at 80 registers (6
// blocks: occupancy hides the latency of the operation rows read through
// L1), the others at 48 (10 blocks for the Philox-bound noise loop).  Wider X
// needs 2W registers of its own, so the bounds relax with W.
constexpr int min_blocks(int W, bool sl) {
  return sl ? (W <= 4 ? 6 : W <= 8 ? 4 : 2) : (W <= 4 ? 10 : W <= 8 ? 6 : 2);
}
// the batched kernel keeps its work-item state live across the whole shot
// loop: one block less for programs with sliced tables (96 registers)
constexpr int min_blocks_batch(int W, bool sl) { return sl && W <= 4 ? 5 : min_blocks(W, sl); }

template <int W, bool SL>
__global__ void __launch_bounds__(kThreads, min_blocks(W, SL)) k_sample(DevView V, RoundKeys rk, uint64_t shot0,
                                                     uint64_t nshots, uint64_t* __restrict__ meas,
                                                     uint64_t* __restrict__ det,
                                                     uint64_t* __restrict__ obs,
                                                     uint8_t* __restrict__ accept) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  SlSmem sm{};
  if constexpr (SL) {
    sm = sl_smem(g_warp_smem + (threadIdx.x >> 5) * sl_warp_words(W, V.sl_par, V.sl_rb), W, V.sl_par, V.sl_rb);
    sl_init(sm);
  }
  sample_one<W, SL>(V, s, s < nshots, rk, shot0, meas, det, obs, accept, sm);
}

// ------------------------------------------------------- batched launch
// One persistent launch over many programs: work item i is a block of `sb`
// shots (a multiple of 32) of one program; warps take items from an atomic
// counter until all are done (no waiting on other warps or blocks).  Program p owns items
// [item_start[p], item_start[p+1]).
struct BatchProg {
  DevView v;
  uint64_t shots, seed, shot_offset;
  uint64_t* meas;
  uint64_t* det;
  uint64_t* obs;
  uint8_t* accept;
};

template <int W, bool SL>
__global__ void __launch_bounds__(kThreads, min_blocks_batch(W, SL)) k_batch(const BatchProg* __restrict__ progs, int n,
                                                    const uint64_t* __restrict__ item_start,
                                                    uint64_t total_items, uint32_t sb,
                                                    unsigned long long* counter, int sl_par, int sl_rb) {
  SlSmem sm{};
  if constexpr (SL) {
    sm = sl_smem(g_warp_smem + (threadIdx.x >> 5) * sl_warp_words(W, sl_par, sl_rb), W, sl_par, sl_rb);
    sl_init(sm);
  }
  // every warp takes its own work items (no block-wide synchronisation)
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(counter, 1ull);
    it = __shfl_sync(0xFFFFFFFFu, it, 0);
    if (it >= total_items) return;
    int lo = 0, hi = n - 1;  // last program with item_start <= it
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (item_start[mid] <= it) lo = mid;
      else hi = mid - 1;
    }
    const BatchProg& P = progs[lo];
    const uint64_t first = (it - item_start[lo]) * sb;
    const uint64_t last = min(first + sb, P.shots);
    const RoundKeys rk = round_keys(P.seed);
    for (uint64_t s0 = first; s0 < last; s0 += 32) {
      const uint64_t s = s0 + lane;
      sample_one<W, SL>(P.v, s, s < last, rk, P.shot_offset, P.meas, P.det, P.obs, P.accept, sm);
    }
  }
}

// ------------------------------------------------------ host-side packing
namespace {

int padded_words_or_zero(int W) {
  for (int p : {1, 2, 4, 8, 16, 32})
    if (W <= p) return p;
  return 0;
}

struct Packer {
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
  void put_padded(const std::vector<uint64_t>& m, int W) {
    for (int i = 0; i < W; ++i) {
      uint64_t x = (size_t)i < m.size() ? m[(size_t)i] : 0;
      put(&x, 8);
    }
  }
};

// Four packed increments of one factor, inc = j | s << 11 | zero << 21
// (J in bits 0-10, S in 11-20, vanishing factors in 21-31), s relative to the
// factor's smallest magnitude exponent smin.
bool factor_lut(int kind, int alpha, int beta, uint32_t inc[4], int* smin_out, int* spread) {
  Factor fc;
  fc.kind = kind;
  fc.alpha = alpha;
  fc.beta = beta;
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

int log2_ceil(unsigned __int128 x) {
  int l = 0;
  while (l < 127 && ((unsigned __int128)1 << l) < x) ++l;
  return l;
}

struct PackError {
  tsim_status st;
  const char* msg;
};

struct Lut {
  uint32_t inc[4];
  int smin, spread;
};

struct FacKey {
  int kind, alpha, beta, ia, ib;
  bool operator<(const FacKey& o) const {
    return std::tie(kind, alpha, beta, ia, ib) < std::tie(o.kind, o.alpha, o.beta, o.ia, o.ib);
  }
};

// A term of a sliced table: constant phase j, magnitude exponent d, and the
// parity indices of each operation code (sorted); dead terms vanish for
// every shot.
struct SlTerm {
  int d = 0, j = 0;
  bool dead = false;
  std::vector<uint64_t> ops[kSlCodes];  // parity indices (qa | qb << 32 for pi-pairs)
};

// How one factor acts on (J, Z): J += j00 + da a + db b + dab ab (mod 8) on
// the (a, b) where it does not vanish, and the vanishing condition zop
// (0 never, 1 a = 1, 2 a = 0, 3 b = 1, 4 b = 0).  za / zb: a / b is the zero
// parity; same: a and b are the same parity.
struct SlDec {
  bool ok = false, dead = false;
  int j00 = 0, da = 0, db = 0, dab = 0, zop = 0;
};

SlDec sliced_decompose(const Lut& l, bool za, bool zb, bool same) {
  SlDec r;
  if (l.spread != 0) return r;  // magnitude depends on the shot
  bool reach[2][2], zero[2][2];
  int jv[2][2];
  int nreach = 0, nzero = 0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      reach[a][b] = (!za || a == 0) && (!zb || b == 0) && (!same || a == b);
      const uint32_t inc = l.inc[a | (b << 1)];
      zero[a][b] = (inc >> 21) != 0;
      jv[a][b] = (int)(inc & 0x7FF) & 7;
      nreach += reach[a][b];
      nzero += reach[a][b] && zero[a][b];
    }
  r.ok = true;
  if (nzero == nreach) { r.dead = true; return r; }
  if (nzero) {
    auto fits = [&](int op) {
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          if (!reach[a][b]) continue;
          const bool want = op == 1 ? a == 1 : op == 2 ? a == 0 : op == 3 ? b == 1 : b == 0;
          if (zero[a][b] != want) return false;
        }
      return true;
    };
    r.zop = 0;
    for (int op = 1; op <= 4 && !r.zop; ++op) {
      if ((op <= 2 && za) || (op >= 3 && zb)) continue;
      if (fits(op)) r.zop = op;
    }
    if (!r.zop) { r.ok = false; return r; }
  }
  // fewest nonzero increments that reproduce J on the non-vanishing entries
  int best = 99;
  for (int dab = 0; dab <= 4; dab += 4)
    for (int da = 0; da < 8; ++da)
      for (int db = 0; db < 8; ++db)
        for (int j00 = 0; j00 < 8; ++j00) {
          if (za && (da || dab)) continue;           // a is always 0
          if (zb && (db || dab)) continue;           // b is always 0
          if (same && (db || dab)) continue;         // a = b: all of it in da
          bool ok = true;
          for (int a = 0; a < 2 && ok; ++a)
            for (int b = 0; b < 2 && ok; ++b)
              if (reach[a][b] && !zero[a][b]) ok = ((j00 + da * a + db * b + dab * a * b) & 7) == jv[a][b];
          const int cost = (da != 0) + (db != 0) + (dab != 0);
          if (ok && cost < best) {
            best = cost;
            r.j00 = j00;
            r.da = da;
            r.db = db;
            r.dab = dab;
          }
        }
  if (best == 99) r.ok = false;
  return r;
}

// Sliced form of one term (factor list f, coefficient phase j, magnitude
// exponent d); false when some factor has no such form.
template <class LutFn>
bool sliced_term(const std::vector<FacKey>& f, int j, int d, LutFn& lut, SlTerm& t) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int>, SlDec> cache;
  t.d = d;
  int jc = j;
  std::map<uint32_t, int> delta;
  std::set<uint64_t> pairs;
  std::set<uint32_t> zp, zn;
  for (const FacKey& k : f) {
    const uint32_t qa = k.ia ? (uint32_t)k.ia + 1 : 0u, qb = k.ib ? (uint32_t)k.ib + 1 : 0u;
    const bool za = qa == 0, zb = qb == 0, same = qa != 0 && qa == qb;
    const int flags = (int)za | ((int)zb << 1) | ((int)same << 2);
    SlDec dec;
    {
      const auto key = std::make_tuple(k.kind, k.alpha & 7, k.beta & 7, flags);
      std::lock_guard<std::mutex> g(mu);
      auto it = cache.find(key);
      if (it == cache.end()) it = cache.emplace(key, sliced_decompose(lut(k.kind, k.alpha, k.beta), za, zb, same)).first;
      dec = it->second;
    }
    if (!dec.ok) return false;
    if (dec.dead) { t.dead = true; return true; }
    jc += dec.j00;
    if (dec.da) delta[qa] = (delta[qa] + dec.da) & 7;
    if (dec.db) delta[qb] = (delta[qb] + dec.db) & 7;
    if (dec.dab) {
      const uint64_t key = (uint64_t)std::min(qa, qb) | ((uint64_t)std::max(qa, qb) << 32);
      if (!pairs.erase(key)) pairs.insert(key);  // (-1)^(ab) twice is 1
    }
    if (dec.zop == 1) zp.insert(qa);
    if (dec.zop == 2) zn.insert(qa);
    if (dec.zop == 3) zp.insert(qb);
    if (dec.zop == 4) zn.insert(qb);
  }
  for (uint32_t q : zp)
    if (zn.count(q)) { t.dead = true; return true; }
  t.j = jc & 7;
  // table-wide parity indices q (qa | qb << 32 for pi-pairs)
  for (const auto& [q, dl] : delta) {
    if (dl & 1) t.ops[SL_ADD1].push_back(q);
    const int rem = dl & 6;
    if (rem == 2) t.ops[SL_ADD2].push_back(q);
    if (rem == 4) t.ops[SL_XOR4].push_back(q);
    if (rem == 6) t.ops[SL_ADD6].push_back(q);
  }
  for (uint64_t pq : pairs) t.ops[SL_XOR4AB].push_back(pq);
  for (uint32_t q : zp) t.ops[SL_ZERO].push_back(q);
  for (uint32_t q : zn) t.ops[SL_ZEROC].push_back(q);
  return true;
}

void pack(const Program& p, DeviceTables& out, int64_t sliced_min, int stage_rows, int seg_par) {
  std::map<std::tuple<int, int, int>, Lut> lut_cache;
  auto lut = [&](int kind, int alpha, int beta) -> const Lut& {
    auto key = std::make_tuple(kind, alpha & 7, beta & 7);
    auto it = lut_cache.find(key);
    if (it != lut_cache.end()) return it->second;
    Lut l{};
    if (!factor_lut(kind, alpha, beta, l.inc, &l.smin, &l.spread))
      throw PackError{TSIM_ERR_INTERNAL, "factor value is not a monomial of bounded spread"};
    return lut_cache.emplace(key, l).first->second;
  };
  const int W = padded_words_or_zero(p.W);
  if (!W) throw PackError{TSIM_ERR_ARG, "per-shot vector wider than 2048 bits is not supported"};
  if ((int)p.chain_norm.size() > kMaxChains) throw PackError{TSIM_ERR_ARG, "too many autoregressive chains for the kernel"};
  if (p.mode == TSIM_MODE_MEASUREMENTS && (int)p.outputs.size() > kMaxOutWords * 64)
    throw PackError{TSIM_ERR_ARG, "too many measurement outputs for the kernel"};
  Packer s;
  DeviceLayout& L = out.layout;
  L = DeviceLayout();
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
      d.thr0 = c.thr.empty() ? 0xFFFFFFFFu : c.thr[0];
      thr_off += (uint32_t)c.thr.size();
      sig_off += (uint32_t)(c.sig.size() * (size_t)W);
      s.put(&d, sizeof d);
      for (size_t w = 0; !c.sig.empty() && w < c.sig[0].size(); ++w)
        if (c.sig[0][w]) throw PackError{TSIM_ERR_INTERNAL, "channel outcome 0 must not flip anything"};
    }
  }
  L.o_t0 = s.section();
  for (size_t i = 0; i < (p.channels.size() + 3) / 4 * 4; ++i) {
    const uint32_t t = i < p.channels.size() && !p.channels[i].thr.empty() ? p.channels[i].thr[0] : 0xFFFFFFFFu;
    s.put(&t, 4);
  }
  L.o_thr = s.section();
  for (const ProgChannel& c : p.channels)
    for (uint32_t t : c.thr) s.put(&t, 4);
  { uint32_t z = 0; s.put(&z, 4); }
  L.o_sig = s.section();
  for (const ProgChannel& c : p.channels)
    for (const auto& sg : c.sig) s.put_padded(sg, W);
  // outputs; in detector mode consecutive single-bit outputs without a
  // constant on consecutive X bits, in the same record, become one run
  L.o_out = s.section();
  {
    int32_t mo = 0;
    std::vector<DOut> ents;
    for (size_t i = 0; i < p.outputs.size(); ++i) {
      const ProgOutput& o = p.outputs[i];
      DOut d{};
      d.cst = o.cst;
      d.rec = (int32_t)i;
      if (o.random) {
        d.kind = OUT_RANDOM;
        d.a = o.xbit;
        d.chain = o.chain;
        d.table = o.table;
      } else {
        int ones = 0, pos = -1;
        for (size_t w = 0; w < o.mask.size(); ++w)
          for (int bb = 0; bb < 64; ++bb)
            if ((o.mask[w] >> bb) & 1) { ++ones; pos = (int)(w * 64 + (size_t)bb); }
        if (ones == 1) { d.kind = OUT_BIT; d.a = pos; }
        else { d.kind = OUT_MASK; d.a = mo; }
      }
      mo += W;
      if (p.mode == TSIM_MODE_DETECTORS && d.kind == OUT_BIT && d.cst == 0 && !ents.empty()) {
        DOut& prev = ents.back();
        const bool same_rec = ((int)i < p.ndet) == (prev.rec < p.ndet);
        if (same_rec && prev.kind == OUT_BIT && prev.cst == 0 && prev.a + 1 == d.a && prev.rec + 1 == d.rec) {
          prev.kind = OUT_RUN;
          prev.chain = 2;
          continue;
        }
        if (same_rec && prev.kind == OUT_RUN && prev.a + prev.chain == d.a && prev.rec + prev.chain == d.rec) {
          prev.chain++;
          continue;
        }
      }
      ents.push_back(d);
    }
    if (!ents.empty()) s.put(ents.data(), ents.size() * sizeof(DOut));
    L.n_ent = (int)ents.size();
    for (const DOut& d : ents)
      if (d.kind == OUT_RUN) {
        L.runs++;
        L.run_outputs += (uint64_t)d.chain;
      }
  }
  L.o_om = s.section();
  for (const ProgOutput& o : p.outputs) s.put_padded(o.mask, W);
  L.o_cn = s.section();
  for (int c : p.chain_norm) { int32_t v = c; s.put(&v, 4); }
  { int32_t z = 0; s.put(&z, 4); }

  // tables: distinct parities, then terms merged into classes with equal factors
  struct Cls {
    std::vector<FacKey> f;
    ZW coef;
  };
  std::vector<DTable> tabs;
  std::vector<uint64_t> par;
  std::vector<DClass> cls;
  std::vector<uint32_t> fidx, finc;
  std::vector<uint64_t> fcoord;
  std::vector<DSBatch> sbs;
  std::vector<DSeg> segs;
  std::vector<uint32_t> rows;
  for (const ProgTable& tb : p.tables) {
    DTable dt{};
    dt.par_off = (uint32_t)(par.size() / (size_t)W);
    std::map<std::vector<uint64_t>, int> pidx;
    std::vector<std::vector<uint64_t>> plist;
    auto parity_index = [&](const std::vector<uint64_t>& m) {
      std::vector<uint64_t> key((size_t)W, 0);
      for (size_t i = 0; i < m.size() && i < (size_t)W; ++i) key[i] = m[i];
      auto it = pidx.find(key);
      if (it != pidx.end()) return it->second;
      int id = (int)plist.size();
      pidx[key] = id;
      plist.push_back(key);
      return id;
    };
    parity_index(std::vector<uint64_t>((size_t)W, 0));  // index 0: the zero parity
    std::map<std::vector<FacKey>, size_t> cidx;
    std::vector<Cls> cl;
    for (const ProgTerm& tm : tb.terms) {
      std::vector<FacKey> fk;
      for (const ProgFactor& f : tm.f) {
        FacKey k{f.kind, f.alpha & 7, f.beta & 7, parity_index(f.u), parity_index(f.v)};
        fk.push_back(k);
      }
      std::sort(fk.begin(), fk.end());
      ZW c = ZW::omega(tm.j0);
      c.k = tm.s0;
      auto it = cidx.find(fk);
      if (it == cidx.end()) {
        cidx[fk] = cl.size();
        cl.push_back({fk, c});
      } else {
        cl[it->second].coef = zw_add(cl[it->second].coef, c);
      }
    }
    // per class: exponent of its smallest possible magnitude
    struct Prep { size_t i; int raw, spread, mono, j, zero; };
    std::vector<Prep> prep;
    for (size_t i = 0; i < cl.size(); ++i) {
      if (cl[i].coef.zero()) continue;  // exact cancellation between terms
      if (cl[i].f.size() > 255) throw PackError{TSIM_ERR_OVERFLOW_BOUND, "term with more than 255 factors"};
      int smin_sum = 0, spread = 0;
      for (const FacKey& k : cl[i].f) {
        const Lut& l = lut(k.kind, k.alpha, k.beta);
        smin_sum += l.smin;
        spread += l.spread;
      }
      int z, ms, mj;
      Prep pr{i, 0, spread, 0, 0, 0};
      if (monomial_of(cl[i].coef, &z, &ms, &mj)) {
        pr.mono = 1;
        pr.j = mj;
        pr.raw = ms + smin_sum;
      } else {
        pr.raw = cl[i].coef.k + smin_sum;
      }
      prep.push_back(pr);
    }
    int base = 0;
    for (size_t q = 0; q < prep.size(); ++q) base = q ? std::min(base, prep[q].raw) : prep[q].raw;
    dt.base = base;
    dt.n_cls = (uint32_t)prep.size();
    // every coefficient of the accumulated sum stays below 2^62 in absolute value
    unsigned __int128 bound = 0;
    for (const Prep& pr : prep) {
      const Cls& c = cl[pr.i];
      unsigned __int128 mag = 1;
      if (!pr.mono) {
        mag = 0;
        for (int i = 0; i < 4; ++i) {
          if (c.coef.c[i] > ((__int128)1 << 60) || c.coef.c[i] < -((__int128)1 << 60))
            throw PackError{TSIM_ERR_OVERFLOW_BOUND, "merged term coefficient exceeds 60 bits"};
          mag += (unsigned __int128)(c.coef.c[i] < 0 ? -c.coef.c[i] : c.coef.c[i]);
        }
        mag *= 2;  // the sqrt2 multiplication at most doubles the largest coefficient
      }
      const int dm = pr.raw - base + pr.spread;
      if (dm / 2 + log2_ceil(mag) >= 100) throw PackError{TSIM_ERR_OVERFLOW_BOUND, "table magnitudes exceed 64-bit accumulation"};
      bound += mag << (dm / 2 + 1);
    }
    if (bound >= ((unsigned __int128)1 << 62)) throw PackError{TSIM_ERR_OVERFLOW_BOUND, "table magnitudes exceed 64-bit accumulation"};

    // ---- bit-sliced layout (large tables whose factors all reduce to
    // operations on J and Z, every term a monomial)
    bool sliced = sliced_min >= 0 && prep.size() >= (size_t)std::max<int64_t>(sliced_min, 1);
    std::vector<SlTerm> sterms;
    for (size_t q = 0; sliced && q < prep.size(); ++q) {
      const Prep& pr = prep[q];
      if (!pr.mono) { sliced = false; break; }
      SlTerm t;
      if (!sliced_term(cl[pr.i].f, pr.j, pr.raw - base, lut, t)) { sliced = false; break; }
      if (!t.dead) sterms.push_back(std::move(t));
    }
    uint64_t real_ops = 0, padded_rows = 0, sliced_work = 0, nbatches = 0;
    if (sliced) {
      dt.mode = TAB_SLICED;
      dt.sb_off = (int32_t)segs.size();  // sliced: the table's segments
      // integer lane-operations of one warp (32 shots) on this table: the
      // bit transpose of X (2W transposes of 5 stages of 4 ops, 32 lanes), per
      // segment each parity (load, store, and per mask bit: find, load, XOR),
      // each padded row on 32 lanes (index load, parity load and the word
      // operations of its code), and per batch 4 transposes, the signed
      // counts and their accumulation (about 110 per lane)
      static const int kRowOps[kSlCodes] = {3, 4, 5, 6, 3, 3, 6};
      uint64_t w32 = 2ull * (uint64_t)W * 5 * 4 * 32;
      uint32_t most = 0;
      auto parities_of = [](const SlTerm& t, std::vector<uint32_t>& out) {
        out.clear();
        for (int c = 0; c < kSlCodes; ++c)
          for (uint64_t r : t.ops[c]) {
            out.push_back((uint32_t)r);
            if (c == SL_XOR4AB) out.push_back((uint32_t)(r >> 32));
          }
      };
      // segments: consecutive terms (the decomposition's order keeps their
      // parities local) while the parity list stays within seg_par words
      std::vector<uint32_t> tp;
      for (size_t t0 = 0; t0 < sterms.size();) {
        std::set<uint32_t> ps;
        size_t t1 = t0;
        while (t1 < sterms.size()) {
          parities_of(sterms[t1], tp);
          size_t add = 0;
          for (uint32_t q : tp) add += q > kSlOnes && !ps.count(q);
          if (t1 > t0 && ps.size() + add + 2 > (size_t)seg_par) break;
          for (uint32_t q : tp)
            if (q > kSlOnes) ps.insert(q);
          ++t1;
        }
        if (ps.size() + 2 > (size_t)kSlMaxPar) throw PackError{TSIM_ERR_ARG, "a sliced term has too many parities"};
        // the segment's terms, sorted by magnitude then by operation counts
        // (so that a batch's terms need similar numbers of rows per code)
        std::vector<SlTerm> lt(sterms.begin() + (long)t0, sterms.begin() + (long)t1);
        std::stable_sort(lt.begin(), lt.end(), [](const SlTerm& a, const SlTerm& b) {
          if (a.d != b.d) return a.d < b.d;
          size_t na = 0, nb = 0;
          for (int c = 0; c < kSlCodes; ++c) { na += a.ops[c].size(); nb += b.ops[c].size(); }
          if (na != nb) return na > nb;
          for (int c = 0; c < kSlCodes; ++c)
            if (a.ops[c].size() != b.ops[c].size()) return a.ops[c].size() > b.ops[c].size();
          return false;
        });
        // batches of 32 terms and their rows, as table-wide parity indices
        // (0 and kSlOnes for padding, qa | qb << 32 for pi-pairs)
        struct PBatch {
          size_t b0, b1;
          uint16_t cnt[kSlCodes];
        };
        std::vector<PBatch> pb;
        std::vector<std::array<uint64_t, 32>> prow;
        std::vector<int> prow_code;
        for (size_t b0 = 0; b0 < lt.size();) {
          size_t b1 = b0;
          while (b1 < lt.size() && b1 - b0 < 32 && lt[b1].d == lt[b0].d) ++b1;
          PBatch B{b0, b1, {}};
          for (int c = 0; c < kSlCodes; ++c) {
            size_t n = 0;
            for (size_t l = b0; l < b1; ++l) n = std::max(n, lt[l].ops[c].size());
            n = (n + 3) & ~(size_t)3;  // whole groups of 4 rows: no single-row tail loop on the device
            if (n > 0xFFFF) throw PackError{TSIM_ERR_ARG, "too many operations of one kind in a term"};
            B.cnt[c] = (uint16_t)n;
            for (size_t k = 0; k < n; ++k) {
              std::array<uint64_t, 32> r;
              for (size_t l = 0; l < 32; ++l) {
                const size_t ti = b0 + l;
                r[l] = (ti < b1 && k < lt[ti].ops[c].size()) ? lt[ti].ops[c][k] : (c == SL_ZEROC ? kSlOnes : 0u);
              }
              prow.push_back(r);
              prow_code.push_back(c);
            }
          }
          pb.push_back(B);
          b0 = b1;
        }
        // shared-memory slot of every parity: word q of the buffer lies in
        // bank q mod 32, and the 32 lanes of a row read their words at once,
        // so distinct parities of one row go to distinct banks where possible
        // (greedy, in row order; slot = bank + 32 x fill)
        std::unordered_map<uint32_t, uint32_t> slot;
        slot.reserve(ps.size() * 2 + 4);
        slot[0] = 0;
        slot[kSlOnes] = kSlOnes;
        uint32_t fill[32] = {0};
        fill[0] = fill[1] = 1;
        const uint32_t cap = (uint32_t)((ps.size() + 2 + 31) / 32) + 1;
        for (size_t ri = 0; ri < prow.size(); ++ri) {
          uint32_t qs[64];
          int nq = 0;
          for (uint64_t v : prow[ri]) {
            qs[nq++] = (uint32_t)v;
            if (prow_code[ri] == SL_XOR4AB && (v >> 32)) qs[nq++] = (uint32_t)(v >> 32);
          }
          std::sort(qs, qs + nq);
          nq = (int)(std::unique(qs, qs + nq) - qs);
          int used[32] = {0};
          for (int k = 0; k < nq; ++k) {
            auto it = slot.find(qs[k]);
            if (it != slot.end()) used[it->second & 31]++;
          }
          for (int k = 0; k < nq; ++k) {
            if (slot.count(qs[k])) continue;
            int best = -1;
            for (int b = 0; b < 32; ++b)
              if (fill[b] < cap && (best < 0 || used[b] < used[best] || (used[b] == used[best] && fill[b] < fill[best])))
                best = b;
            slot[qs[k]] = (uint32_t)best + 32u * fill[best];
            fill[best]++;
            used[best]++;
          }
        }
        uint32_t nslot = 2;
        for (const auto& kv : slot) nslot = std::max(nslot, kv.second + 1);
        if (nslot > (uint32_t)kSlMaxPar) throw PackError{TSIM_ERR_ARG, "a sliced term has too many parities"};
        DSeg g{};
        g.par_off = (uint32_t)(par.size() / (size_t)W);
        g.n_par = nslot;
        {
          std::vector<uint32_t> of_slot(nslot, 0);  // table parity index per slot (0: none)
          for (const auto& kv : slot)
            if (kv.first > kSlOnes) of_slot[kv.second] = kv.first;
          for (uint32_t sl = 0; sl < nslot; ++sl) {
            // slot 0: the zero parity; kSlOnes: all ones (set on the device);
            // unused slots: zero masks
            if (of_slot[sl]) par.insert(par.end(), plist[of_slot[sl] - 1].begin(), plist[of_slot[sl] - 1].end());
            else par.insert(par.end(), (size_t)W, 0ull);
          }
        }
        for (uint32_t q : ps) {
          uint64_t pop = 0;
          for (uint64_t m : plist[q - 1]) pop += (uint64_t)__builtin_popcountll(m);
          w32 += 3 + 3 * pop;
        }
        w32 += 3 * (uint64_t)(nslot - ps.size());
        // rows hold byte offsets of the slots' words: 4 slot, or
        // 4 slot_a | 4 slot_b << 16 for pi-pairs; groups of 4 rows are
        // [group][lane][4], so a lane's 4 rows are 16 contiguous bytes
        g.sb_off = (uint32_t)sbs.size();
        size_t ri = 0;
        for (const PBatch& P : pb) {
          DSBatch B{};
          B.row_off = (uint32_t)rows.size();
          B.d = lt[P.b0].d;
          for (size_t l = 0; l < P.b1 - P.b0; ++l) {
            const SlTerm& t = lt[P.b0 + l];
            B.valid |= 1u << l;
            for (int bit = 0; bit < 3; ++bit) B.j0m[bit] |= (uint32_t)((t.j >> bit) & 1) << l;
          }
          uint32_t nrows = 0;
          for (int c = 0; c < kSlCodes; ++c) {
            const size_t n = P.cnt[c];
            B.cnt[c] = (uint16_t)n;
            for (size_t gi = 0; gi < n / 4; ++gi)
              for (size_t l = 0; l < 32; ++l)
                for (size_t k = 4 * gi; k < 4 * gi + 4; ++k) {
                  const uint64_t v = prow[ri + k][l];
                  uint32_t r;
                  if (c == SL_XOR4AB) r = (4 * slot.at((uint32_t)v)) | ((4 * slot.at((uint32_t)(v >> 32))) << 16);
                  else r = 4 * slot.at((uint32_t)v);
                  const size_t ti = P.b0 + l;
                  if (ti < P.b1 && k < lt[ti].ops[c].size()) ++real_ops;
                  rows.push_back(r);
                }
            ri += n;
            padded_rows += n;
            nrows += (uint32_t)n;
            w32 += (uint64_t)n * 32 * (uint64_t)kRowOps[c];
          }
          w32 += 32 * 110;
          most = std::max(most, nrows);
          if (rows.size() > 0xFFFFFFFFull) throw PackError{TSIM_ERR_ARG, "sliced tables too large"};
          sbs.push_back(B);
        }
        g.n_sb = (uint32_t)(sbs.size() - g.sb_off);
        nbatches += g.n_sb;
        L.sl_par_max = std::max<uint32_t>(L.sl_par_max, g.n_par);
        segs.push_back(g);
        t0 = t1;
      }
      dt.n_sb = (int32_t)(segs.size() - (size_t)dt.sb_off);
      dt.n_par = 0;
      // stage the rows through shared memory when every batch fits a buffer
      dt.stage = stage_rows > 0 && most <= (uint32_t)stage_rows ? 1 : 0;
      if (dt.stage) L.sl_rows_max = std::max(L.sl_rows_max, most);
      sliced_work = w32;
    } else {
      // few distinct parities: evaluate each once per shot and index them;
      // many: evaluate a GF(2) basis of their span and give every parity its
      // coordinates in that basis
      std::vector<uint64_t> coords(plist.size(), 0);
      dt.par_off = (uint32_t)(par.size() / (size_t)W);
      if (plist.size() <= (size_t)kMaxParities) {
        for (const auto& m : plist) par.insert(par.end(), m.begin(), m.end());
        dt.n_par = (uint32_t)plist.size();
      } else {
        dt.mode = TAB_BASIS;
        std::vector<std::vector<uint64_t>> bvec, borig;
        std::vector<uint64_t> bcomb;
        std::vector<int> bpiv;
        for (size_t i = 1; i < plist.size(); ++i) {
          std::vector<uint64_t> v = plist[i];
          uint64_t comb = 0;
          for (size_t j = 0; j < bvec.size(); ++j)
            if ((v[(size_t)bpiv[j] >> 6] >> (bpiv[j] & 63)) & 1) {
              for (int w = 0; w < W; ++w) v[(size_t)w] ^= bvec[j][(size_t)w];
              comb ^= bcomb[j];
            }
          int piv = -1;
          for (int w = 0; w < W && piv < 0; ++w)
            if (v[(size_t)w]) piv = w * 64 + __builtin_ctzll(v[(size_t)w]);
          if (piv < 0) { coords[i] = comb; continue; }
          if (borig.size() >= 64) throw PackError{TSIM_ERR_ARG, "table parities span more than 64 dimensions"};
          const uint64_t me = 1ull << borig.size();
          borig.push_back(plist[i]);
          bvec.push_back(v);
          bcomb.push_back(comb ^ me);
          bpiv.push_back(piv);
          coords[i] = me;
        }
        for (const auto& m : borig) par.insert(par.end(), m.begin(), m.end());
        dt.n_par = (uint32_t)borig.size();
      }
      const bool basis = dt.mode == TAB_BASIS;
      dt.cls_off = (uint32_t)cls.size();
      for (const Prep& pr : prep) {
        const Cls& c = cl[pr.i];
        DClass d{};
        d.fac_off = (uint32_t)fidx.size();
        d.n_fac = (uint32_t)c.f.size();
        d.mono = pr.mono;
        d.j0 = pr.j;
        d.d0 = pr.raw - base;
        if (!pr.mono)
          for (int i = 0; i < 4; ++i) d.c[i] = (long long)c.coef.c[i];
        for (const FacKey& k : c.f) {
          const Lut& l = lut(k.kind, k.alpha, k.beta);
          fidx.push_back(basis ? 0u : ((uint32_t)k.ia | ((uint32_t)k.ib << 8)));
          finc.insert(finc.end(), l.inc, l.inc + 4);
          fcoord.push_back(basis ? coords[(size_t)k.ia] : 0);
          fcoord.push_back(basis ? coords[(size_t)k.ib] : 0);
        }
        cls.push_back(d);
      }
    }
    L.classes += prep.size();
    L.parities += plist.size() - 1;
    L.table_classes.push_back(prep.size());
    L.table_parities.push_back(plist.size() - 1);
    {
      uint64_t nf = 0;
      for (const Prep& pr : prep) nf += cl[pr.i].f.size();
      L.table_class_factors.push_back(nf);
      L.class_factors += nf;
    }
    L.table_mode.push_back(dt.mode);
    L.table_batches.push_back(nbatches);
    L.table_rows.push_back(padded_rows);
    L.table_ops.push_back(real_ops);
    L.table_work32.push_back(sliced_work);
    tabs.push_back(dt);
  }
  L.o_tab = s.section();
  if (!tabs.empty()) s.put(tabs.data(), tabs.size() * sizeof(DTable));
  L.o_par = s.section();
  if (!par.empty()) s.put(par.data(), par.size() * 8);
  L.o_cls = s.section();
  if (!cls.empty()) s.put(cls.data(), cls.size() * sizeof(DClass));
  L.o_fidx = s.section();
  if (!fidx.empty()) s.put(fidx.data(), fidx.size() * 4);
  L.o_finc = s.section();
  if (!finc.empty()) s.put(finc.data(), finc.size() * 4);
  L.o_fco = s.section();
  if (!fcoord.empty()) s.put(fcoord.data(), fcoord.size() * 8);
  L.o_seg = s.section();
  if (!segs.empty()) s.put(segs.data(), segs.size() * sizeof(DSeg));
  L.o_sb = s.section();
  if (!sbs.empty()) s.put(sbs.data(), sbs.size() * sizeof(DSBatch));
  L.o_row = s.section();
  if (!rows.empty()) s.put(rows.data(), rows.size() * 4);
  L.sl_par = L.sl_par_max ? (int)((L.sl_par_max + 3) & ~3u) : 0;
  L.sl_rb = (int)L.sl_rows_max * 32;
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
  out.blob.swap(s.b);
}

DevView make_view(const unsigned char* base, const DeviceLayout& L, const Program& p) {
  DevView v{};
  v.W = L.W;
  v.n_ch = (int)p.channels.size();
  v.n_out = (int)p.outputs.size();
  v.n_ent = L.n_ent;
  v.n_chains = (int)p.chain_norm.size();
  v.n_tab = (int)p.tables.size();
  v.nmeas = p.nmeas;
  v.ndet = p.ndet;
  v.nobs = p.nobs;
  v.mode = p.mode;
  v.ch = (const DChan*)(base + L.o_ch);
  v.thr0 = (const uint4*)(base + L.o_t0);
  v.thr = (const uint32_t*)(base + L.o_thr);
  v.sig = (const uint64_t*)(base + L.o_sig);
  v.out = (const DOut*)(base + L.o_out);
  v.omask = (const uint64_t*)(base + L.o_om);
  v.chain_norm = (const int32_t*)(base + L.o_cn);
  v.tab = (const DTable*)(base + L.o_tab);
  v.par = (const uint64_t*)(base + L.o_par);
  v.cls = (const DClass*)(base + L.o_cls);
  v.fidx = (const uint32_t*)(base + L.o_fidx);
  v.finc = (const uint32_t*)(base + L.o_finc);
  v.fcoord = (const uint64_t*)(base + L.o_fco);
  v.seg = (const DSeg*)(base + L.o_seg);
  v.sb = (const DSBatch*)(base + L.o_sb);
  v.rows = (const uint32_t*)(base + L.o_row);
  v.sl_par = L.sl_par;
  v.sl_rb = L.sl_rb;
  v.dmap_off = (const int32_t*)(base + L.o_dmo);
  v.dmap_idx = (const int32_t*)(base + L.o_dmi);
  v.omap_off = (const int32_t*)(base + L.o_omo);
  v.omap_idx = (const int32_t*)(base + L.o_omi);
  return v;
}

const DeviceTables& tables_of(const Program& p) {
  if (!p.devtab) fail(TSIM_ERR_INTERNAL, "program has no device tables");
  if (p.devtab->status != TSIM_OK) fail(p.devtab->status, p.devtab->message);
  return *p.devtab;
}

DeviceProgram* upload(const Program& p) {
  const DeviceTables& T = tables_of(p);
  auto* d = new DeviceProgram();
  TSIM_CUDA(cudaGetDevice(&d->device));
  cudaError_t e = cudaMalloc(&d->blob, std::max<size_t>(T.blob.size(), 256));
  if (e != cudaSuccess) {
    delete d;
    fail(TSIM_ERR_OOM, std::string("cudaMalloc of program tables: ") + cudaGetErrorString(e));
  }
  e = cudaMemcpy(d->blob, T.blob.data(), T.blob.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d->blob);
    delete d;
    fail(TSIM_ERR_CUDA, std::string("cudaMemcpy of program tables: ") + cudaGetErrorString(e));
  }
  d->v = make_view((const unsigned char*)d->blob, T.layout, p);
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

// Threads per block and dynamic shared memory of a launch: programs with
// sliced tables get sl_words words per warp (sl_warp_words) and as many warps
// per block (1 to 4) as fit in kSmemPerBlock; the others use kThreads
// threads and none.
constexpr int kSmemPerBlock = 48 * 1024;

struct LaunchShape {
  unsigned threads;
  size_t smem;
};

LaunchShape shape_of(int sl_words) {
  if (sl_words <= 0) return {(unsigned)kThreads, 0};
  const size_t per_warp = (size_t)sl_words * 4;
  const int warps = (int)std::max<size_t>(1, std::min<size_t>(kThreads / 32, kSmemPerBlock / per_warp));
  return {(unsigned)(32 * warps), per_warp * (size_t)warps};
}

// allow a kernel more than the default 48 KB of dynamic shared memory
template <class K>
cudaError_t allow_smem(K kernel, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int W>
cudaError_t launch_w(const DevView& v, cudaStream_t s, uint64_t seed, uint64_t off, uint64_t shots, uint64_t* meas,
                     uint64_t* det, uint64_t* obs, uint8_t* acc) {
  const LaunchShape sh = shape_of(sl_warp_words(W, v.sl_par, v.sl_rb));
  const uint64_t blocks = (shots + sh.threads - 1) / sh.threads;
  if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
  if (v.sl_par > 0) {
    cudaError_t e = allow_smem(k_sample<W, true>, sh.smem);
    if (e != cudaSuccess) return e;
    k_sample<W, true><<<(unsigned)blocks, sh.threads, sh.smem, s>>>(v, round_keys(seed), off, shots, meas, det, obs,
                                                                     acc);
  } else {
    k_sample<W, false><<<(unsigned)blocks, sh.threads, 0, s>>>(v, round_keys(seed), off, shots, meas, det, obs, acc);
  }
  return cudaGetLastError();
}

cudaError_t launch(const DevView& v, cudaStream_t s, uint64_t seed, uint64_t off, uint64_t shots, uint64_t* meas,
                   uint64_t* det, uint64_t* obs, uint8_t* acc) {
  switch (v.W) {
    case 1: return launch_w<1>(v, s, seed, off, shots, meas, det, obs, acc);
    case 2: return launch_w<2>(v, s, seed, off, shots, meas, det, obs, acc);
    case 4: return launch_w<4>(v, s, seed, off, shots, meas, det, obs, acc);
    case 8: return launch_w<8>(v, s, seed, off, shots, meas, det, obs, acc);
    case 16: return launch_w<16>(v, s, seed, off, shots, meas, det, obs, acc);
    case 32: return launch_w<32>(v, s, seed, off, shots, meas, det, obs, acc);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// Host emulation of the warp-cooperative evaluation of a sliced table, read
// from the packed tables exactly as the kernel reads them: 32 per-shot
// vectors X at once (bit s of every word belongs to vector s).  Returns the
// exact value of table t for each vector.
std::vector<ZW> emulate_sliced_table(const Program& p, const DeviceTables& T, int t,
                                     const std::vector<std::vector<uint64_t>>& xs) {
  const DeviceLayout& L = T.layout;
  const unsigned char* b = T.blob.data();
  const DTable& tb = ((const DTable*)(b + L.o_tab))[t];
  const DSeg* seg = (const DSeg*)(b + L.o_seg);
  const DSBatch* sbv = (const DSBatch*)(b + L.o_sb);
  const uint32_t* rows = (const uint32_t*)(b + L.o_row);
  const uint64_t* par = (const uint64_t*)(b + L.o_par);
  const int W = L.W;
  std::vector<ZW> val(32);
  std::vector<uint32_t> Xs((size_t)64 * W, 0);
  for (int sh = 0; sh < 32; ++sh)
    for (int i = 0; i < 64 * W; ++i)
      if ((xs[(size_t)sh][(size_t)i >> 6] >> (i & 63)) & 1) Xs[(size_t)i] |= 1u << sh;
  for (int g = 0; g < tb.n_sb; ++g) {
    const DSeg& sg = seg[tb.sb_off + g];
    std::vector<uint32_t> Par(sg.n_par, 0);
    for (uint32_t q = 0; q < sg.n_par; ++q) {
      uint32_t acc = 0;
      for (int w = 0; w < W; ++w)
        for (int bit = 0; bit < 64; ++bit)
          if ((par[((size_t)sg.par_off + q) * W + (size_t)w] >> bit) & 1) acc ^= Xs[(size_t)(64 * w + bit)];
      Par[q] = q == kSlOnes ? 0xFFFFFFFFu : acc;
    }
    auto word = [&](uint32_t off) {
      if (off % 4 || off / 4 >= sg.n_par) fail(TSIM_ERR_INTERNAL, "sliced row outside its segment's parity words");
      return Par[off / 4];
    };
    for (uint32_t bi = 0; bi < sg.n_sb; ++bi) {
      const DSBatch& B = sbv[sg.sb_off + bi];
      uint32_t J0[32], J1[32], J2[32], Z[32];
      for (int l = 0; l < 32; ++l) {
        J0[l] = 0u - ((B.j0m[0] >> l) & 1u);
        J1[l] = 0u - ((B.j0m[1] >> l) & 1u);
        J2[l] = 0u - ((B.j0m[2] >> l) & 1u);
        Z[l] = 0u - ((~B.valid >> l) & 1u);
      }
      size_t at = B.row_off;
      for (int c = 0; c < kSlCodes; ++c) {
        const uint32_t n = B.cnt[c];
        if (n % 4) fail(TSIM_ERR_INTERNAL, "sliced rows not in groups of 4");
        for (uint32_t k = 0; k < n; ++k)
          for (int l = 0; l < 32; ++l) {
            const uint32_t r = rows[at + (size_t)(k / 4) * 128 + (size_t)l * 4 + (k % 4)];
            const uint32_t a = c == SL_XOR4AB ? word(r & 0xFFFFu) & word(r >> 16) : word(r);
            auto add = [&](uint32_t m, int times) {  // J += times * m (mod 8), one plane step at a time
              for (int i = 0; i < times; ++i) {
                const uint32_t c0 = J0[l] & m;
                J0[l] ^= m;
                const uint32_t c1 = J1[l] & c0;
                J1[l] ^= c0;
                J2[l] ^= c1;
              }
            };
            switch (c) {
              case SL_XOR4: case SL_XOR4AB: add(a, 4); break;
              case SL_ADD2: add(a, 2); break;
              case SL_ADD6: add(a, 6); break;
              case SL_ADD1: add(a, 1); break;
              case SL_ZERO: Z[l] |= a; break;
              case SL_ZEROC: Z[l] |= ~a; break;
            }
          }
        at += (size_t)n * 32;
      }
      for (int sh = 0; sh < 32; ++sh)
        for (int l = 0; l < 32; ++l) {
          if ((Z[l] >> sh) & 1) continue;
          const int J = (int)((J0[l] >> sh) & 1) | (int)(((J1[l] >> sh) & 1) << 1) | (int)(((J2[l] >> sh) & 1) << 2);
          ZW term = ZW::omega(J);
          term.k = B.d + tb.base;
          val[(size_t)sh] = zw_add(val[(size_t)sh], term);
        }
    }
  }
  return val;
}

void selftest_sliced(const Program& p, uint64_t seed, int rounds) {
  const DeviceTables& T = tables_of(p);
  const int W = T.layout.W;
  uint64_t st = seed ^ 0x5EED5EEDull;
  auto rnd = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  for (size_t t = 0; t < p.tables.size(); ++t) {
    if (T.layout.table_mode[t] != TAB_SLICED) continue;
    for (int r = 0; r < rounds; ++r) {
      std::vector<std::vector<uint64_t>> xs(32, std::vector<uint64_t>((size_t)W, 0));
      for (auto& x : xs)
        for (int i = 0; i < p.nx; ++i)  // X bits beyond n_x stay zero, as on the device
          if (rnd() & 1) x[(size_t)i >> 6] |= 1ull << (i & 63);
      const std::vector<ZW> got = emulate_sliced_table(p, T, (int)t, xs);
      for (int sh = 0; sh < 32; ++sh) {
        ZW want = eval_table_host(p, (int)t, xs[(size_t)sh].data());
        for (auto& c : want.c) c = -c;
        if (!zw_add(got[(size_t)sh], want).zero())
          fail(TSIM_ERR_INTERNAL, "sliced table " + std::to_string(t) + " differs from the exact evaluation");
      }
    }
  }
}

void prepare_device_tables(Program& p, int64_t sliced_min, int stage_rows, int seg_par) {
  auto* t = new DeviceTables();
  try {
    pack(p, *t, sliced_min, stage_rows < 0 ? kDefaultStageRows : stage_rows,
         seg_par <= 0 ? kDefaultSegmentParities : std::max(seg_par, 16));
  } catch (const PackError& e) {
    t->status = e.st;
    t->message = e.msg;
    t->blob.clear();
  }
  delete p.devtab;
  p.devtab = t;
}

void device_sample(const Program& p, const SampleArgs& a, void* stream) {
  if (p.mode == TSIM_MODE_DETECTORS && a.meas) fail(TSIM_ERR_ARG, "measurement records requested from a detector-mode program");
  tables_of(p);  // report a program that cannot run on the device before any CUDA call
  if (a.shots == 0) return;
  if (a.shots > 0x7FFFFFFFull * 32) fail(TSIM_ERR_ARG, "too many shots for one launch");
  const DevView& v = ensure_uploaded(p);
  cudaError_t e = launch(v, (cudaStream_t)stream, a.seed, a.shot_offset, a.shots, a.meas, a.det, a.obs, a.accept);
  if (e != cudaSuccess) fail(TSIM_ERR_CUDA, std::string("sampling kernel launch: ") + cudaGetErrorString(e));
}

// ----------------------------------------------------------- batch plans
// Programs of a batch fall in two groups, without and with sliced tables:
// each group is one persistent launch with its own register budget (the
// kernels with sliced tables keep fewer warps resident).
struct BatchGroup {
  int off = 0, n = 0;       // programs [off, off + n) of the plan's (reordered) list
  int wmax = 1, sl_par = 0, sl_rb = 0;
  uint64_t total_items = 0;
  uint64_t* d_item_start = nullptr;   // n + 1 entries
  unsigned long long* d_counter = nullptr;
};

struct BatchPlan {
  int device = -1, n = 0, sms = 1;
  uint32_t sb = 128;        // shots per work item
  int blocks_per_sm = 8;
  BatchGroup grp[2];
  std::vector<BatchProg> h_progs;  // group 0 first, then group 1
  unsigned char* dmem = nullptr;
  BatchProg* d_progs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  float tuned_ms = 0;
  int form = 0;  // 0: persistent launches over the work items; 1: each program's own launch
  uint64_t total_items() const { return grp[0].total_items + grp[1].total_items; }
  int wmax() const { return std::max(grp[0].wmax, grp[1].wmax); }
};

namespace {

void plan_items(BatchPlan& b, cudaStream_t s) {
  for (BatchGroup& g : b.grp) {
    std::vector<uint64_t> start((size_t)g.n + 1, 0);
    for (int i = 0; i < g.n; ++i)
      start[(size_t)i + 1] = start[(size_t)i] + (b.h_progs[(size_t)(g.off + i)].shots + b.sb - 1) / b.sb;
    g.total_items = start[(size_t)g.n];
    TSIM_CUDA(cudaMemcpyAsync(g.d_item_start, start.data(), start.size() * 8, cudaMemcpyHostToDevice, s));
  }
  TSIM_CUDA(cudaStreamSynchronize(s));
}

template <int W>
cudaError_t launch_group_w(const BatchPlan& b, const BatchGroup& g, cudaStream_t s, unsigned grid) {
  // every warp gets room for the transposed X at the launch's W, the
  // largest sliced parity buffer and the largest row buffers of the group
  const LaunchShape sh = shape_of(sl_warp_words(W, g.sl_par, g.sl_rb));
  if (g.sl_par > 0) {
    cudaError_t e = allow_smem(k_batch<W, true>, sh.smem);
    if (e != cudaSuccess) return e;
    k_batch<W, true><<<grid, sh.threads, sh.smem, s>>>(b.d_progs + g.off, g.n, g.d_item_start, g.total_items, b.sb,
                                                       g.d_counter, g.sl_par, g.sl_rb);
  } else {
    k_batch<W, false><<<grid, sh.threads, 0, s>>>(b.d_progs + g.off, g.n, g.d_item_start, g.total_items, b.sb,
                                                  g.d_counter, 0, 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch(const BatchPlan& b, cudaStream_t s) {
  if (b.form == 1) {  // the programs' own sampling launches, one after another
    for (const BatchProg& p : b.h_progs) {
      if (!p.shots) continue;
      cudaError_t e = launch(p.v, s, p.seed, p.shot_offset, p.shots, p.meas, p.det, p.obs, p.accept);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  for (const BatchGroup& g : b.grp) {
    if (!g.total_items) continue;
    cudaError_t e = cudaMemsetAsync(g.d_counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const uint64_t want = (uint64_t)b.sms * (uint64_t)b.blocks_per_sm;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, g.total_items));
    switch (g.wmax) {
      case 1: e = launch_group_w<1>(b, g, s, grid); break;
      case 2: e = launch_group_w<2>(b, g, s, grid); break;
      case 4: e = launch_group_w<4>(b, g, s, grid); break;
      case 8: e = launch_group_w<8>(b, g, s, grid); break;
      case 16: e = launch_group_w<16>(b, g, s, grid); break;
      case 32: e = launch_group_w<32>(b, g, s, grid); break;
      default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

BatchPlan* batch_create(const Program* const* progs, int n, const SampleArgs* args, int autotune) {
  auto b = std::make_unique<BatchPlan>();
  b->n = n;
  TSIM_CUDA(cudaGetDevice(&b->device));
  TSIM_CUDA(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device));
  std::vector<BatchProg> per_group[2];
  for (int i = 0; i < n; ++i) {
    const Program& p = *progs[i];
    if (p.mode == TSIM_MODE_DETECTORS && args[i].meas)
      fail(TSIM_ERR_ARG, "measurement records requested from a detector-mode program");
    tables_of(p);
    BatchProg bp{};
    bp.v = ensure_uploaded(p);
    bp.shots = args[i].shots;
    bp.seed = args[i].seed;
    bp.shot_offset = args[i].shot_offset;
    bp.meas = args[i].meas;
    bp.det = args[i].det;
    bp.obs = args[i].obs;
    bp.accept = args[i].accept;
    const int gi = bp.v.sl_par > 0 ? 1 : 0;
    BatchGroup& g = b->grp[gi];
    g.wmax = std::max(g.wmax, bp.v.W);
    g.sl_par = std::max(g.sl_par, bp.v.sl_par);
    g.sl_rb = std::max(g.sl_rb, bp.v.sl_rb);
    per_group[gi].push_back(bp);
  }
  b->grp[0].off = 0;
  b->grp[0].n = (int)per_group[0].size();
  b->grp[1].off = b->grp[0].n;
  b->grp[1].n = (int)per_group[1].size();
  for (const auto& v : per_group) b->h_progs.insert(b->h_progs.end(), v.begin(), v.end());
  const size_t bytes = (size_t)n * sizeof(BatchProg) + ((size_t)n + 2) * 8 + 2 * 64;
  cudaError_t e = cudaMalloc(&b->dmem, bytes);
  if (e != cudaSuccess) fail(TSIM_ERR_OOM, std::string("cudaMalloc of the batch plan: ") + cudaGetErrorString(e));
  b->d_progs = (BatchProg*)b->dmem;
  {
    uint64_t* starts = (uint64_t*)(b->dmem + (size_t)n * sizeof(BatchProg));
    b->grp[0].d_item_start = starts;
    b->grp[1].d_item_start = starts + b->grp[0].n + 1;
    unsigned char* ctr = b->dmem + (size_t)n * sizeof(BatchProg) + ((size_t)n + 2) * 8;
    b->grp[0].d_counter = (unsigned long long*)ctr;
    b->grp[1].d_counter = (unsigned long long*)(ctr + 64);
  }
  cudaStream_t s = nullptr;
  TSIM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  struct SD { cudaStream_t s; ~SD() { cudaStreamDestroy(s); } } sd{s};
  if (n) TSIM_CUDA(cudaMemcpyAsync(b->d_progs, b->h_progs.data(), (size_t)n * sizeof(BatchProg), cudaMemcpyHostToDevice, s));
  b->sb = 128;
  plan_items(*b, s);
  if (autotune == 2) b->form = 1;
  if (autotune == 1 && b->total_items()) {
    // shot-block size x resident blocks per SM: time every candidate twice on
    // the real batch (records are overwritten with identical values)
    cudaEvent_t e0, e1;
    TSIM_CUDA(cudaEventCreate(&e0));
    TSIM_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    uint32_t best_sb = b->sb;
    int best_bps = b->blocks_per_sm;
    // work items of 32, 128 or 512 shots (one warp each)
    for (uint32_t sb : {32u, 128u, 512u}) {
      b->sb = sb;
      plan_items(*b, s);
      for (int bps : {4, 8, 16}) {
        b->blocks_per_sm = bps;
        float t = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
          TSIM_CUDA(cudaEventRecord(e0, s));
          TSIM_CUDA(launch_batch(*b, s));
          TSIM_CUDA(cudaEventRecord(e1, s));
          TSIM_CUDA(cudaEventSynchronize(e1));
          float ms = 0;
          TSIM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          t = std::min(t, ms);
        }
        if (t < best) { best = t; best_sb = sb; best_bps = bps; }
      }
    }
    // the other launch form: every program's own kernel (few large programs
    // can run faster that way than through the persistent loop)
    {
      b->form = 1;
      float t = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        TSIM_CUDA(cudaEventRecord(e0, s));
        TSIM_CUDA(launch_batch(*b, s));
        TSIM_CUDA(cudaEventRecord(e1, s));
        TSIM_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        TSIM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        t = std::min(t, ms);
      }
      b->form = t < best ? 1 : 0;
      best = std::min(best, t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->sb = best_sb;
    b->blocks_per_sm = best_bps;
    b->tuned_ms = best;
    plan_items(*b, s);
  }
  // capture counter reset + persistent launch as one graph
  TSIM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = launch_batch(*b, s);
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(s, &g);
  if (le != cudaSuccess || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    fail(TSIM_ERR_CUDA, std::string("graph capture of the batched launch: ") +
                            cudaGetErrorString(le != cudaSuccess ? le : ce));
  }
  b->graph = g;
  TSIM_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
  return b.release();
}

void batch_launch(BatchPlan* b, void* stream) {
  int cur = -1;
  TSIM_CUDA(cudaGetDevice(&cur));
  if (cur != b->device) fail(TSIM_ERR_ARG, "batch launched on another device than it was created on");
  TSIM_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
}

void batch_free(BatchPlan* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->dmem) cudaFree(b->dmem);
  delete b;
}

void batch_info(const BatchPlan* b, int64_t out[7]) {
  out[0] = b->sb;
  out[1] = b->blocks_per_sm;
  out[2] = (int64_t)b->total_items();
  out[3] = b->exec ? 1 : 0;
  out[4] = b->wmax();
  out[5] = (int64_t)(b->tuned_ms * 1000.0f);
  out[6] = b->form;
}

void device_sample_batch(const Program* const* progs, int n, const SampleArgs* args, void* stream) {
  BatchPlan* b = batch_create(progs, n, args, 0);
  struct F { BatchPlan* b; ~F() { batch_free(b); } } f{b};
  batch_launch(b, stream);
  TSIM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
}

void device_sync(void* stream) {
  TSIM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int st = 0;
  TSIM_CUDA(cudaMemcpyFromSymbol(&st, g_status, sizeof st));
  if (st) {
    int z = 0;
    TSIM_CUDA(cudaMemcpyToSymbol(g_status, &z, sizeof z));
    if (st & ST_TIMEOUT) fail(TSIM_ERR_TIMEOUT, "device: a shared-memory staging copy did not complete in time");
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
  if (!p.devtab) return noalloc_error(TSIM_ERR_INTERNAL, "program has no device tables");
  // the packed tables were built on the host when the program was compiled
  // or loaded; this call only copies them
  const DeviceTables& T = *p.devtab;
  if (T.status != TSIM_OK) return noalloc_error(T.status, "program tables cannot run on the device");
  if (T.layout.total > kNoAllocBytes)
    return noalloc_error(TSIM_ERR_ARG, "program tables exceed the 4 MiB maximum of tsim_sample_noalloc");
  if (shots == 0) return TSIM_OK;
  if (shots > 0x7FFFFFFFull * 32) return noalloc_error(TSIM_ERR_ARG, "too many shots for one launch");
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
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // every byte the kernel reads is rewritten here, so nothing stale from the
  // previous call survives
  if (cudaMemcpyAsync(g_noalloc_dev[dev], T.blob.data(), T.layout.total, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return noalloc_error(TSIM_ERR_CUDA, "cudaMemcpyAsync into the no-alloc scratch array failed");
  const DevView v = make_view((const unsigned char*)g_noalloc_dev[dev], T.layout, p);
  if (launch(v, s, seed, shot_offset, shots, d_meas, d_det, d_obs, d_accept) != cudaSuccess)
    return noalloc_error(TSIM_ERR_CUDA, "launch of the sampling kernel failed");
  return TSIM_OK;
}
