// GB300 (sm_103a) per-shot sampling kernels, included by the per-width
// translation units kern_w*.cu (one explicit instantiation of the launchers
// per padded X width, compiled in parallel).
//
// One thread carries one shot end to end (Sec. "Complexity", paragraph
// "Sampling"):
//   1. error mechanisms: one Philox4x32-10 word per reduced channel, or
//      geometric gaps between firing channels (Sec. "Detectors"); each
//      outcome that fires does X ^= its column signature (Eq.
//      detector_sampling);
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
//   3. the Bernoulli draw compares U * P_prev < 2^32 * P_1 exactly (64-bit
//      integers when bounds on the operands rule out overflow, else int128);
//   4. bit-packed records (runs of single-bit detectors copied by word shifts).
// The program tables are read-only; per-thread table loads are uniform
// (broadcast) loads, the bit-sliced rows are lane-coalesced 16-byte loads.
// k_sample launches one program; k_batch runs persistent warps over the
// (program, shot-block) work items of many programs (one launch per group of
// programs with equal X width, with or without sliced tables).  Conditions that make a
// result untrustworthy (overflow, a non-real marginal, P_prev <= 0, a staging
// wait that gave up) set bits of the launch's status word, read by tsim_sync.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "devtypes.h"

namespace tsim {

// The key schedule of Philox4x32-10: round r uses key + r (0x9E3779B9,
// 0xBB67AE85).  RoundKeys holds all ten (a kernel parameter of one launch);
// SeedKey derives them from the key, one add per round (no registers held
// across a persistent loop that serves many programs).
struct SeedKey {
  uint32_t k0, k1;
  __device__ __forceinline__ uint32_t key0(int r) const { return k0 + (uint32_t)r * 0x9E3779B9u; }
  __device__ __forceinline__ uint32_t key1(int r) const { return k1 + (uint32_t)r * 0xBB67AE85u; }
};
__device__ __forceinline__ uint32_t key0_of(const RoundKeys& rk, int r) { return rk.k0[r]; }
__device__ __forceinline__ uint32_t key1_of(const RoundKeys& rk, int r) { return rk.k1[r]; }
__device__ __forceinline__ uint32_t key0_of(const SeedKey& sk, int r) { return sk.key0(r); }
__device__ __forceinline__ uint32_t key1_of(const SeedKey& sk, int r) { return sk.key1(r); }

template <class K>
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              const K& rk, uint32_t o[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    c0 = hi1 ^ c1 ^ key0_of(rk, r);
    c1 = lo1;
    c2 = hi0 ^ c3 ^ key1_of(rk, r);
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

// x as a 64-bit integer and its magnitude, when it fits
__device__ __forceinline__ bool to64(__int128 x, long long& v, unsigned long long& mag) {
  v = (long long)x;
  mag = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  return (__int128)v == x;
}

// sign of X + Y sqrt2 for |X|, |Y| < 2^63 (exact: X^2 against 2 Y^2 in 128 bits
// when the signs differ; sqrt2 is irrational, so the squares never tie)
__device__ __forceinline__ int sign_xy64(long long X, long long Y) {
  if (X >= 0 && Y >= 0) return (X | Y) != 0;
  if (X <= 0 && Y <= 0) return -1;
  const unsigned long long ax = X < 0 ? 0ull - (unsigned long long)X : (unsigned long long)X;
  const unsigned long long ay = Y < 0 ? 0ull - (unsigned long long)Y : (unsigned long long)Y;
  const unsigned __int128 x2 = (unsigned __int128)ax * ax, y2 = 2 * ((unsigned __int128)ay * ay);
  if (X > 0) return x2 > y2 ? 1 : -1;
  return y2 > x2 ? 1 : -1;
}

// Algorithm 1's decision U * P_prev < 2^32 * P_1 and the next P_prev (P_1 if
// the bit is 1, P_prev - P_1 otherwise) in 64-bit integers, exactly as the
// int128 path computes them, whenever no operand reaches 2^62: P_prev's
// coefficients below 2^30 (they meet U < 2^32), P_1's below 2^(62 - s) for
// its shift s, so that every difference stays below 2^63.  Returns the bit,
// or -1 when the int128 path must decide.  *pos receives whether P_prev > 0.
__device__ __forceinline__ int bern_fast(const RV& pv, const RV& p1, uint32_t U, RV& next, bool* pos) {
  long long a, b, a1, b1;
  unsigned long long ma, mb, ma1, mb1;
  if (!(to64(pv.A, a, ma) && to64(pv.B, b, mb) && to64(p1.A, a1, ma1) && to64(p1.B, b1, mb1))) return -1;
  const unsigned long long mp = ma | mb, m1 = ma1 | mb1;
  const int s = p1.e + 32 - pv.e;  // P_1's shift against an unshifted U * P_prev
  if ((mp >> 30) || s < 0 || s > 62 || (m1 >> (62 - s))) return -1;
  *pos = sign_xy64(a, b) > 0;
  const long long X = a * (long long)U - a1 * (1ll << s);
  const long long Y = b * (long long)U - b1 * (1ll << s);
  if (sign_xy64(X, Y) < 0) {
    next = p1;
    return 1;
  }
  const int e2 = min(pv.e, p1.e);
  const int sp = pv.e - e2, s1 = p1.e - e2;  // one of them is 0
  if (sp > 62 || s1 > 62 || (mp >> (62 - sp)) || (m1 >> (62 - s1))) return -1;
  next.A = (__int128)(a * (1ll << sp) - a1 * (1ll << s1));
  next.B = (__int128)(b * (1ll << sp) - b1 * (1ll << s1));
  next.e = e2;
  return 0;
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

// Two 32 x 32 bit-matrix transposes across the warp at once: on entry lane
// r holds row r of each matrix (bit c = column c), on exit lane c holds
// column c (bit r = row r).  Stage j (16, 8, 4, 2, 1) swaps the off-diagonal
// j x j blocks between lanes r and r ^ j.  Each lane keeps half of its bits
// (mk) and sends the other half; one shuffle carries both matrices: the
// half of B that leaves rides, rotated by j, in the positions of A that
// stay.  The receiver rotates A's half into place; B's half arrives in
// place.  (Rotations never wrap a kept bit: they move bits within a 2j
// block.)
struct Transposer2 {
  uint32_t mk[5];   // the bits a lane keeps at each stage
  uint32_t rot[5];  // left-rotation that brings received bits of A into place
  __device__ __forceinline__ explicit Transposer2(int lane) {
    const uint32_t keep[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int st = 0; st < 5; ++st) {
      const int j = 16 >> st;
      const bool upper = (lane & j) != 0;
      mk[st] = upper ? ~keep[st] : keep[st];
      rot[st] = upper ? 32u - (uint32_t)j : (uint32_t)j;
    }
  }
  __device__ __forceinline__ void operator()(uint32_t& a, uint32_t& b) const {
#pragma unroll
    for (int st = 0; st < 5; ++st) {
      const uint32_t bs = __funnelshift_r(b, b, rot[st]);
      const uint32_t send = (a & ~mk[st]) | (bs & mk[st]);
      const uint32_t r = __shfl_xor_sync(0xFFFFFFFFu, send, 16 >> st);
      a = (a & mk[st]) | (__funnelshift_l(r, r, rot[st]) & ~mk[st]);
      b = (b & mk[st]) | (r & ~mk[st]);
    }
  }
};

// Operation rows, read through a generic pointer: a shared staging buffer
// or the rows in global memory (one code path for both).  A row holds the
// byte offset of a parity word (4q), or two of them (4qa | 4qb << 16) for
// pi-pairs.  Rows come in groups of 4: group g of a code is 32 lanes x 4
// consecutive rows, so one 16-byte load per lane fetches 4 rows and a warp's
// load is 512 contiguous bytes.
struct Rows {
  const uint4* p;  // this lane's current group
  __device__ __forceinline__ uint4 get4(int g) const { return p[32 * g]; }
  __device__ __forceinline__ void adv4(int k) { p += 32 * k; }
};

// Rows per chunk of sl_loop: every row and parity load of a chunk is issued
// before its updates.
constexpr int kSlChunk = 16;

// Consecutive rows of one code are spread over kSlWays independent
// accumulators so that their update chains overlap (2 ways: fewer
// registers, measured as fast as 4).
#ifndef TSIM_SL_WAYS
#define TSIM_SL_WAYS 2
#endif
constexpr int kSlWays = TSIM_SL_WAYS;
static_assert(kSlWays == 2 || kSlWays == 4, "2 or 4 accumulator ways");

// NR rows (a multiple of 4) of one code: all their row loads, then all
// their parity loads, then the updates (one memory round trip).
template <bool PAIR, int NR, class F>
__device__ __forceinline__ void sl_chunk(Rows& R, uint32_t par, F&& f) {
  uint32_t r[NR], a[NR], b[NR];
#pragma unroll
  for (int g = 0; g < NR / 4; ++g) {
    const uint4 v = R.get4(g);
    r[4 * g] = v.x;
    r[4 * g + 1] = v.y;
    r[4 * g + 2] = v.z;
    r[4 * g + 3] = v.w;
  }
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    a[i] = lds(par + (PAIR ? (r[i] & 0xFFFFu) : r[i]));
    b[i] = PAIR ? lds(par + (r[i] >> 16)) : 0u;
  }
#pragma unroll
  for (int i = 0; i < NR; i += 2) f((i / 2) % kSlWays, a[i], b[i], a[i + 1], b[i + 1]);
  R.adv4(NR / 4);
}

// The n rows (a multiple of 4) of one code: chunks of kSlChunk rows, then
// the rest (4, 8 or 12 rows) as one chunk, so that a code costs one memory
// round trip per started chunk (the rest taken 4 rows at a time cost 7.5 %
// on the 256-program batch); f(way, a, b, a2, b2) applies two rows' updates.
template <bool PAIR, class F>
__device__ __forceinline__ void sl_loop(int n, Rows& R, uint32_t par, F&& f) {
  int k = 0;
  for (; k + kSlChunk <= n; k += kSlChunk) sl_chunk<PAIR, kSlChunk>(R, par, f);
  switch (n - k) {
    case 4: sl_chunk<PAIR, 4>(R, par, f); break;
    case 8: sl_chunk<PAIR, 8>(R, par, f); break;
    case 12: sl_chunk<PAIR, 12>(R, par, f); break;
    default: break;
  }
}

// (x1, x2) += (y1, y2) for 2-bit bit-sliced counters mod 4
__device__ __forceinline__ void add2bit(uint32_t& x1, uint32_t& x2, uint32_t y1, uint32_t y2) {
  x2 ^= y2 ^ (x1 & y1);
  x1 ^= y1;
}

// All operation rows of one batch; returns the planes (J0, J1, J2, Z).
__device__ __forceinline__ void sl_batch(const DSBatch& B, Rows R, uint32_t par, int lane, uint32_t& J0, uint32_t& J1,
                                         uint32_t& J2, uint32_t& Z) {
  J0 = 0u - ((B.j0m[0] >> lane) & 1u);
  J1 = 0u - ((B.j0m[1] >> lane) & 1u);
  J2 = 0u - ((B.j0m[2] >> lane) & 1u);
  Z = 0u - ((~B.valid >> lane) & 1u);
  // per way: J2 flips k, vanishing flags z, and a 2-bit counter (c1, c2) of
  // the rows that add 2 to J (J2 flips and vanishing flags commute with it)
  uint32_t k[kSlWays] = {}, z[kSlWays] = {}, c1[kSlWays] = {}, c2[kSlWays] = {};
  // two rows per update: 3-input word operations take both (a 2-bit
  // counter adds two bits as c1 ^ a ^ b with carry maj(c1, a, b))
  sl_loop<false>(B.cnt[SL_XOR4], R, par,
                 [&](int w, uint32_t a, uint32_t, uint32_t a2, uint32_t) { k[w] ^= a ^ a2; });
  sl_loop<false>(B.cnt[SL_ADD2], R, par, [&](int w, uint32_t a, uint32_t, uint32_t a2, uint32_t) {
    const uint32_t c = c1[w];
    c2[w] ^= (c & (a | a2)) | (a & a2);
    c1[w] = c ^ a ^ a2;
  });
  // J += 6a = 2a + 4a
  sl_loop<false>(B.cnt[SL_ADD6], R, par, [&](int w, uint32_t a, uint32_t, uint32_t a2, uint32_t) {
    const uint32_t c = c1[w];
    c2[w] ^= (c & (a | a2)) | (a & a2);
    c1[w] = c ^ a ^ a2;
    k[w] ^= a ^ a2;
  });
  sl_loop<true>(B.cnt[SL_XOR4AB], R, par,
                [&](int w, uint32_t a, uint32_t b, uint32_t a2, uint32_t b2) { k[w] ^= (a & b) ^ (a2 & b2); });
  sl_loop<false>(B.cnt[SL_ZERO], R, par,
                 [&](int w, uint32_t a, uint32_t, uint32_t a2, uint32_t) { z[w] |= a | a2; });
  sl_loop<false>(B.cnt[SL_ZEROC], R, par,
                 [&](int w, uint32_t a, uint32_t, uint32_t a2, uint32_t) { z[w] |= ~(a & a2); });
  add2bit(c1[0], c2[0], c1[1], c2[1]);
  if constexpr (kSlWays == 4) {
    add2bit(c1[2], c2[2], c1[3], c2[3]);
    add2bit(c1[0], c2[0], c1[2], c2[2]);
    J2 ^= (k[0] ^ k[1]) ^ (k[2] ^ k[3]);
    Z |= (z[0] | z[1]) | (z[2] | z[3]);
  } else {
    J2 ^= k[0] ^ k[1];
    Z |= z[0] | z[1];
  }
  add2bit(J1, J2, c1[0], c2[0]);
  // J += a (odd phases; rare): a three-plane increment
  sl_loop<false>(B.cnt[SL_ADD1], R, par, [&](int, uint32_t a, uint32_t, uint32_t a2, uint32_t) {
    const uint32_t cy = J0 & a;
    J0 ^= a;
    J2 ^= J1 & cy;
    J1 ^= cy;
    const uint32_t cy2 = J0 & a2;
    J0 ^= a2;
    J2 ^= J1 & cy2;
    J1 ^= cy2;
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
  const Transposer2 transpose2(lane);
  __syncwarp();  // the transposed X (kept current by the caller) is visible
  uint32_t state = S.rb > 0 ? lds(S.state) : 4u;
  const bool staged = tb.stage && !(state & 4u);
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
    // a parity's word from its mask (one shared load per X bit)
    auto walk = [&](uint32_t q) {
      uint32_t acc = 0;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        uint64_t x = w < ws ? __ldg(pm + (size_t)q * ws + w) : 0ull;
        while (x) {
          acc ^= lds(S.xs + 4u * (uint32_t)(64 * w + __ffsll((long long)x) - 1));
          x &= x - 1;
        }
      }
      return acc;
    };
    for (uint32_t q0 = lane; q0 < sg.n_par; q0 += 128) {
      if constexpr (W <= 4) {
        // parities name at most four (k8 = 0) or eight X bits: as many
        // shared loads, the same number in every lane (no loop over mask bits)
        const uint2* pi = V.pidx + sg.par_off;
        uint2 ix[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t q = q0 + 32u * (uint32_t)u;
          ix[u] = q < sg.n_par ? __ldg(pi + q) : make_uint2(0u, 0u);
        }
        auto four = [&](uint32_t v) {
          return lds(S.xs + 4u * (v & 0xFFu)) ^ lds(S.xs + 4u * ((v >> 8) & 0xFFu)) ^
                 lds(S.xs + 4u * ((v >> 16) & 0xFFu)) ^ lds(S.xs + 4u * (v >> 24));
        };
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t q = q0 + 32u * (uint32_t)u;
          if (q >= sg.n_par) continue;
          const uint2 v = ix[u];
          const uint32_t acc = v.x == kSlWalk ? walk(q) : (sg.k8 ? four(v.x) ^ four(v.y) : four(v.x));
          asm volatile("st.shared.u32 [%0], %1;" ::"r"(S.par + 4u * q), "r"(q == kSlOnes ? 0xFFFFFFFFu : acc)
                       : "memory");
        }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t q = q0 + 32u * (uint32_t)u;
          if (q >= sg.n_par) continue;
          const uint32_t acc = walk(q);
          asm volatile("st.shared.u32 [%0], %1;" ::"r"(S.par + 4u * q), "r"(q == kSlOnes ? 0xFFFFFFFFu : acc)
                       : "memory");
        }
      }
    }
    __syncwarp();
    for (uint32_t b = 0; b < sg.n_sb; ++b, ++bi) {
      // the header at use (keeping the next one in registers across the
      // batch cost more in spills than it saved in latency); staging needs
      // the next one to start its copy
      const DSBatch B = bt[b];
      if (staged && b + 1 < sg.n_sb) next = bt[b + 1];
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
          if (lane == 0) atomicOr(V.status, ST_TIMEOUT);
          mbar_wait_bounded(S.bar0, state & 1u);
          mbar_wait_bounded(S.bar1, (state >> 1) & 1u);
          ok = false;
          state |= 4u;
        } else {
          state ^= 1u << buf;
        }
      }
      // rows from this batch's staging buffer, or from global memory
      const uint4* rp = (staged && ok)
                            ? reinterpret_cast<const uint4*>(__cvta_shared_to_generic((bi & 1) ? S.rb1 : S.rb0))
                            : reinterpret_cast<const uint4*>(V.rows + B.row_off);
      sl_batch(B, Rows{rp + lane}, S.par, lane, J0, J1, J2, Z);
      if (staged) __syncwarp();  // the buffer just read is refilled next batch
      // lane s now needs, for each of the 32 terms, its phase and flag at shot s
      uint32_t T0 = J0, T1 = J1, T2 = J2, TZ = Z;
      transpose2(T0, T1);
      transpose2(T2, TZ);
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

// The warp's transposed X in shared memory: word b holds bit b of X of the
// warp's 32 shots (bit s = lane s).  Written whole after the noise, then one
// word per change of X (the random outputs' bits), so that table
// evaluations read it without transposing X again.
template <int W>
__device__ __forceinline__ void xs_store_all(const SlSmem& S, const uint64_t (&X)[W]) {
  const int lane = threadIdx.x & 31;
  const Transposer2 transpose2(lane);
#pragma unroll
  for (int w = 0; w < W; ++w) {
    uint32_t lo = (uint32_t)X[w], hi = (uint32_t)(X[w] >> 32);
    transpose2(lo, hi);
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(S.xs + 4u * (uint32_t)(64 * w + lane)), "r"(lo) : "memory");
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(S.xs + 4u * (uint32_t)(64 * w + 32 + lane)), "r"(hi) : "memory");
  }
}
__device__ __forceinline__ void xs_store_bit(const SlSmem& S, int b, uint32_t word) {
  if ((threadIdx.x & 31) == 0)
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(S.xs + 4u * (uint32_t)b), "r"(word) : "memory");
}

// SL: the program has sliced tables (kernels without them never contain the
// warp-cooperative code and keep their register budget)
template <int W, bool SL>
__device__ ZC eval_table(const DevView& V, int t, const uint64_t (&X)[W], const SlSmem& sm) {
  const DTable tb = V.tab[t];
  if (tb.cst) {  // precomputed: the value does not depend on the shot
    const DConst k = V.tconst[t];
    return ZC{{k.c[0], k.c[1], k.c[2], k.c[3]}, tb.base};
  }
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

// Value of a FLOAT table (complex double): per class, the exact factors give
// w^J sqrt2^S (or vanish) as in the SCALAR layout, the arbitrary-angle
// factors give e^(i pi phi) with phi the sum of the angles whose parity is 1,
// and the class adds coef w^J sqrt2^S e^(i pi phi).
struct ZF {
  double re, im;
};

template <int W>
__device__ ZF eval_table_f(const DevView& V, int t, const uint64_t (&X)[W]) {
  const DTable tb = V.tab[t];
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
  ZF z{0.0, 0.0};
  for (uint32_t q = 0; q < tb.n_cls; ++q) {
    const DClass& C = V.cls[tb.cls_off + q];
    const uint32_t fo = C.fac_off, nf = C.n_fac;
    uint32_t acc = 0;
    for (uint32_t k = 0; k < nf; ++k) {
      const uint32_t ix = __ldg(V.fidx + fo + k);
      const uint32_t a = pbit(ix & 0xFF), b = pbit((ix >> 8) & 0xFF);
      acc += __ldg(V.finc + (size_t)(fo + k) * 4 + (a | (b << 1)));
    }
    if (acc >> 21) continue;  // some factor vanished
    double phi = (double)(acc & 7) * 0.25;  // w^J = e^(i pi J / 4)
    for (int k = 0; k < C.pad; ++k)
      if (pbit(__ldg(V.ffidx + C.j0 + k))) phi += __ldg(V.ffang + C.j0 + k);
    const int S = (int)((acc >> 11) & 0x3FF);
    const double m = ldexp((S & 1) ? 1.4142135623730951 : 1.0, S >> 1);
    double sn, cs;
    sincospi(phi, &sn, &cs);
    const double cr = __longlong_as_double(C.c[0]), ci = __longlong_as_double(C.c[1]);
    z.re += m * (cr * cs - ci * sn);
    z.im += m * (cr * sn + ci * cs);
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

// Error mechanisms of one shot: X ^= the signature of every channel outcome
// that fires (Eq. detector_sampling).
//  - noise_mode 0: one Philox word per channel (stream 0, word c of the
//    shot); the outcome-0 thresholds of the four channels of a Philox call
//    come in one 16-byte load and one test; the rare block where some channel
//    fires walks its channels;
//  - noise_mode 1, geometric gaps (Sec. "Detectors"): per group, a word U
//    gives the number of channels skipped before the next candidate, the
//    largest k <= (channels left) with U < T_k; a candidate's own word V,
//    mapped onto [Q, 2^32), picks its outcome by the channel's thresholds.
//    Words come from stream 2 in the order they are used.
template <int W, class K>
__device__ __forceinline__ void sample_noise(const DevView& V, uint32_t c0, uint32_t c1, const K& rk,
                                             uint64_t (&X)[W]) {
  if (V.noise_mode == 0) {
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
    return;
  }
  // The first eight words of stream 2 come from two Philox calls that every
  // lane makes up front, together (a shot draws one word per group plus two
  // per candidate, rarely more than eight); they are consumed in order from
  // a register queue, and only a lane that needs more generates further
  // blocks on its own.
  uint32_t j = 0;  // next word of stream 2
  uint32_t q0[4], q1[4];
  philox4x32_10(c0, c1, 2u, 0u, rk, q0);
  philox4x32_10(c0, c1, 2u, 1u, rk, q1);
  uint32_t blk[4] = {0, 0, 0, 0};
  auto word = [&]() {
    uint32_t v;
    if (j < 8) {
      v = q0[0];
      q0[0] = q0[1]; q0[1] = q0[2]; q0[2] = q0[3]; q0[3] = q1[0];
      q1[0] = q1[1]; q1[1] = q1[2]; q1[2] = q1[3];
    } else {
      if ((j & 3) == 0) philox4x32_10(c0, c1, 2u, j >> 2, rk, blk);
      const uint32_t q = j & 3;
      v = q == 0 ? blk[0] : q == 1 ? blk[1] : q == 2 ? blk[2] : blk[3];
    }
    ++j;
    return v;
  };
  // the next group's descriptor is loaded while the current one is drawn
  DGroup G = V.n_grp > 0 ? V.grp[0] : DGroup{};
  for (int g = 0; g < V.n_grp; ++g) {
    const DGroup Gn = g + 1 < V.n_grp ? V.grp[g + 1] : G;
    const uint32_t* T = V.gT + G.off;  // T_k at T[k - 1]
    uint32_t pos = 0;
    while (pos < G.n) {
      const uint32_t U = word();
      const uint32_t rem = G.n - pos;
      if (U < (pos == 0 ? G.tn : __ldg(T + rem - 1))) break;  // gap = rem: no candidate among the rest
      // the gap: the largest k < rem with U < T_k (T_0 = 2^32 > U, U >= T_rem).
      // T_k is close to 2^32 q^k (q = Q / 2^32), so k is about
      // log2(U / 2^32) / log2 q: a float estimate (the hardware log2; the
      // group's 1 / log2 q from the host), then exact steps on the table
      // (usually one or two loads instead of a binary search's log2(rem)
      // dependent ones)
      float x = __log2f((float)U * 2.3283064365386963e-10f) * G.rlq;
      if (!(x < (float)rem)) x = (float)rem;  // also NaN and infinity
      int k = (int)ceilf(x) - 1;
      k = k < 0 ? 0 : (k >= (int)rem ? (int)rem - 1 : k);
      while (k + 1 < (int)rem && U < __ldg(T + k)) ++k;  // T_{k+1} is T[k]
      while (k > 0 && U >= __ldg(T + k - 1)) --k;
      const uint32_t lo = (uint32_t)k;
      pos += lo;
      const DChan ch = V.ch[__ldg(V.gmem + G.off + pos)];
      const uint32_t Vw = word();
      const uint32_t Vp = G.Q + (uint32_t)(((uint64_t)Vw * ((1ull << 32) - G.Q)) >> 32);
      if (Vp >= ch.thr0) {
        const uint32_t* thr = V.thr + ch.thr_off;
        uint32_t o = 1;
        while (o + 1 < ch.n_out && Vp >= __ldg(thr + o)) ++o;
        const uint64_t* sg = V.sig + ch.sig_off + (size_t)o * V.W;
#pragma unroll
        for (int w = 0; w < W; ++w)
          if (w < V.W) X[w] ^= __ldg(sg + w);
      }
      pos += 1;
    }
    G = Gn;
  }
}

// debug record of one table evaluation (see kDumpHead)
template <int W>
__device__ __forceinline__ void dump_eval(long long* rec, int t, const ZC& z, const uint64_t (&X)[W], int ws) {
  rec[0] = t;
#pragma unroll
  for (int i = 0; i < 4; ++i) rec[1 + i] = z.c[i];
  rec[5] = z.base;
#pragma unroll
  for (int w = 0; w < W; ++w)
    if (w < ws) rec[kDumpHead + w] = (long long)X[w];
}

template <int W>
__device__ __forceinline__ void dump_eval_f(long long* rec, int t, const ZF& z, const uint64_t (&X)[W], int ws) {
  rec[0] = t;
  rec[1] = __double_as_longlong(z.re);
  rec[2] = __double_as_longlong(z.im);
  rec[3] = 0;
  rec[4] = 0;
  rec[5] = kDumpFloat;
#pragma unroll
  for (int w = 0; w < W; ++w)
    if (w < ws) rec[kDumpHead + w] = (long long)X[w];
}

// One shot s of a launch (global shot index shot0 + s), records at row s.
// Every lane of a warp calls it together (sliced tables are evaluated by the
// whole warp); lanes past the end of the launch have valid = false and
// compute a shot whose records are not written.  sm: the warp's shared words.
// DBG: dump (may be NULL) receives one record per table evaluation.
template <int W, bool SL, bool DBG, class K>
__device__ void sample_one(const DevView& V, uint64_t s, bool valid, const K& rk, uint64_t shot0,
                           uint64_t* __restrict__ meas, uint64_t* __restrict__ det,
                           uint64_t* __restrict__ obs, uint8_t* __restrict__ accept, const SlSmem& sm,
                           long long* dump = nullptr) {
  const uint64_t shot = shot0 + s;
  const uint32_t c0 = (uint32_t)shot, c1 = (uint32_t)(shot >> 32);
  int st = 0;
  const int drow = kDumpHead + V.W;
  int nd = 0;  // debug records written

  // 1. error mechanisms and f = T e
  uint64_t X[W];
#pragma unroll
  for (int w = 0; w < W; ++w) X[w] = 0;
  sample_noise<W, K>(V, c0, c1, rk, X);
  if constexpr (SL) xs_store_all<W>(sm, X);

  // 2-3. outputs in autoregressive order (Algorithm 1 per chain)
  RV pp[kMaxChains];
  int rot[kMaxChains];
  // chains with arbitrary rotations: P_prev and the normalisation's value
  // (its phase is the chain's common phase, its modulus the first P_prev)
  double fprev[kMaxChains], fnre[kMaxChains], fnim[kMaxChains], fnmag[kMaxChains];
  for (int c = 0; c < V.n_chains; ++c) {
    if (V.chain_float[c]) {
      const ZF z = eval_table_f<W>(V, V.chain_norm[c], X);
      if (DBG && dump) dump_eval_f<W>(dump + (size_t)drow * nd++, V.chain_norm[c], z, X, V.W);
      const double m = sqrt(z.re * z.re + z.im * z.im);
      if (!(m > 0.0)) st |= ST_ZERO_PROB;
      fnre[c] = z.re;
      fnim[c] = z.im;
      fnmag[c] = m;
      fprev[c] = m;
      continue;
    }
    const ZC z = eval_table<W, SL>(V, V.chain_norm[c], X, sm);
    if (DBG && dump) dump_eval<W>(dump + (size_t)drow * nd++, V.chain_norm[c], z, X, V.W);
    const int pre = V.tab[V.chain_norm[c]].rot;  // precomputed for a constant normalisation
    rot[c] = pre >= 0 ? pre : chain_rotation(z, &st);
    pp[c] = to_real_rot(z, rot[c], &st);
  }
  const int dw = (V.ndet + 63) >> 6, ow = (V.nobs + 63) >> 6;
  const int mw = (V.nmeas + 63) >> 6;
  uint64_t mcur = 0;  // measurement mode: the record word being filled
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
    } else if (V.chain_float[o.chain]) {
      // Algorithm 1 in double precision; the ratio is rounded to FP32 before
      // the comparison with U / 2^32
      const int c = o.chain;
      set_xbit<W>(X, o.a, true);
      if constexpr (SL) xs_store_bit(sm, o.a, 0xFFFFFFFFu);
      const ZF z1 = eval_table_f<W>(V, o.table, X);
      if (DBG && dump) dump_eval_f<W>(dump + (size_t)drow * nd++, o.table, z1, X, V.W);
      const double p1 = (z1.re * fnre[c] + z1.im * fnim[c]) / fnmag[c];
      if (!(fprev[c] > 0.0)) st |= ST_ZERO_PROB;
      uint32_t u[4];
      philox4x32_10(c0, c1, 1u, (uint32_t)(i >> 2), rk, u);
      const uint32_t q4 = (uint32_t)i & 3;
      const uint32_t U = q4 == 0 ? u[0] : q4 == 1 ? u[1] : q4 == 2 ? u[2] : u[3];
      const float q = __double2float_rn(p1 / fprev[c]);
      bit = (double)U < (double)q * 4294967296.0;
      if (bit) {
        fprev[c] = p1;
      } else {
        fprev[c] = fprev[c] - p1;
        set_xbit<W>(X, o.a, false);
      }
    } else {
      set_xbit<W>(X, o.a, true);
      if constexpr (SL) xs_store_bit(sm, o.a, 0xFFFFFFFFu);
      const ZC z1 = eval_table<W, SL>(V, o.table, X, sm);
      if (DBG && dump) dump_eval<W>(dump + (size_t)drow * nd++, o.table, z1, X, V.W);
      const RV p1 = to_real_rot(z1, rot[o.chain], &st);
      const RV pv = pp[o.chain];
      uint32_t u[4];
      philox4x32_10(c0, c1, 1u, (uint32_t)(i >> 2), rk, u);
      const uint32_t q4 = (uint32_t)i & 3;
      const uint32_t U = q4 == 0 ? u[0] : q4 == 1 ? u[1] : q4 == 2 ? u[2] : u[3];
      // bit = 1 iff U * P_prev < 2^32 * P_1: in 64-bit integers when the
      // values are small (the common case), else in int128
      RV nx;
      bool pos = true;
      const int fb = bern_fast(pv, p1, U, nx, &pos);
      if (fb >= 0) {
        if (!pos) st |= ST_ZERO_PROB;
        bit = fb;
        pp[o.chain] = nx;
        if (!bit) set_xbit<W>(X, o.a, false);
      } else {
        if (sign_xy(pv.A, pv.B, &st) <= 0) st |= ST_ZERO_PROB;
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
    }
    // every lane walks the same outputs, so the warp is converged here
    if constexpr (SL)
      if (o.kind == OUT_RANDOM) xs_store_bit(sm, o.a, __ballot_sync(0xFFFFFFFFu, bit != 0));
    if (V.mode == 0) {
      put(i, (uint64_t)bit);  // detectors are outputs [0, ndet), observables [ndet, ndet + nobs)
    } else {
      // measurement records in output order, one word at a time
      mcur |= (uint64_t)bit << (i & 63);
      if ((i & 63) == 63 || i == V.n_out - 1) {
        if (meas && valid) meas[s * mw + (i >> 6)] = mcur;
        mcur = 0;
      }
    }
  }
  if (V.mode == 0) flush();

  // 4. measurement mode: every detector and observable (Eq. xor) is one
  // parity of the final X (its measurements' masks and drawn bits, XORed
  // ahead of time) plus a constant
  if (V.mode != 0) {
    for (int w = 0; w < dw; ++w) {
      uint64_t v = 0;
      for (int b = 0; b < 64 && 64 * w + b < V.ndet; ++b) {
        const int d = 64 * w + b;
        v |= (uint64_t)(parity_w<W>(V.dmask + (size_t)d * V.W, X, V.W) ^ V.dcst[d]) << b;
      }
      any_det |= v != 0;
      if (det && valid) det[s * dw + w] = v;
    }
    if (obs && valid)
      for (int w = 0; w < ow; ++w) {
        uint64_t v = 0;
        for (int b = 0; b < 64 && 64 * w + b < V.nobs; ++b) {
          const int d = 64 * w + b;
          v |= (uint64_t)(parity_w<W>(V.omask2 + (size_t)d * V.W, X, V.W) ^ V.ocst[d]) << b;
        }
        obs[s * ow + w] = v;
      }
  }
  if (!valid) return;
  if (accept) accept[s] = any_det ? 0 : 1;
  if (st) atomicOr(V.status, st);
}


// dynamic shared memory: sl_warp_words(...) per warp for programs with sliced tables
extern __shared__ __align__(128) uint32_t g_warp_smem[];

// Register bounds (resident blocks of up to 128 threads per SM) for X of up
// to 4 words: kernels for programs with sliced tables at 72 registers (7
// blocks: occupancy hides the latency of the operation rows read through
// L1; on the colour code 7 blocks were 4.5 % faster than 8 at 64 registers,
// which spill more, and 15 % faster than 6 at 80), the others at 48 (10
// blocks for the Philox-bound noise loop).  Wider X needs 2W registers of
// its own, so the bounds relax with W.
#ifndef TSIM_MINB_SL
#define TSIM_MINB_SL 7
#endif
#ifndef TSIM_BATCH_SEEDKEY
#define TSIM_BATCH_SEEDKEY 1
#endif
#ifndef TSIM_MINB_SL_BATCH
#define TSIM_MINB_SL_BATCH 6
#endif
constexpr int min_blocks(int W, bool sl) {
  return sl ? (W <= 4 ? TSIM_MINB_SL : W <= 8 ? 4 : 2) : (W <= 4 ? 10 : W <= 8 ? 6 : 2);
}
// the batched kernel keeps its work-item state live across the whole shot
// loop: fewer blocks for programs with sliced tables (6: 80 registers)
constexpr int min_blocks_batch(int W, bool sl) { return sl && W <= 4 ? TSIM_MINB_SL_BATCH : min_blocks(W, sl); }

// One program's launch: thread s samples shot shot0 + s.  DBG: shots with
// dump_row[s] >= 0 also write a record of every table evaluation.
template <int W, bool SL, bool DBG>
__global__ void __launch_bounds__(kThreads, min_blocks(W, SL)) k_sample(DevView V, RoundKeys rk, uint64_t shot0,
                                                     uint64_t nshots, uint64_t* __restrict__ meas,
                                                     uint64_t* __restrict__ det,
                                                     uint64_t* __restrict__ obs,
                                                     uint8_t* __restrict__ accept, long long* dump,
                                                     const int32_t* __restrict__ dump_row, int dump_stride) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  SlSmem sm{};
  if constexpr (SL) {
    sm = sl_smem(g_warp_smem + (threadIdx.x >> 5) * sl_warp_words(W, V.sl_par, V.sl_rb), W, V.sl_par, V.sl_rb);
    sl_init(sm);
  }
  long long* rec = nullptr;
  if constexpr (DBG) {
    const int r = s < nshots ? dump_row[s] : -1;
    if (r >= 0) rec = dump + (size_t)r * (size_t)dump_stride;
  }
  sample_one<W, SL, DBG, RoundKeys>(V, s, s < nshots, rk, shot0, meas, det, obs, accept, sm, rec);
}

// ------------------------------------------------------- batched launch
// One persistent launch over many programs: work item i is a block of `sb`
// shots (a multiple of 32) of one program; warps take items from an atomic
// counter until all are done (no waiting on other warps or blocks).  Program p owns items
// [item_start[p], item_start[p+1]).
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
#if TSIM_BATCH_SEEDKEY
    const SeedKey rk{(uint32_t)P.seed, (uint32_t)(P.seed >> 32)};
    for (uint64_t s0 = first; s0 < last; s0 += 32) {
      const uint64_t s = s0 + lane;
      sample_one<W, SL, false, SeedKey>(P.v, s, s < last, rk, P.shot_offset, P.meas, P.det, P.obs, P.accept, sm);
    }
#else
    const RoundKeys rk = round_keys(P.seed);
    for (uint64_t s0 = first; s0 < last; s0 += 32) {
      const uint64_t s = s0 + lane;
      sample_one<W, SL, false, RoundKeys>(P.v, s, s < last, rk, P.shot_offset, P.meas, P.det, P.obs, P.accept, sm);
    }
#endif
  }
}

// ------------------------------------------------------------ launchers
// Threads per block and dynamic shared memory of a launch: programs with
// sliced tables get sl_words words per warp (sl_warp_words) and as many warps
// per block (1 to 4) as fit in kSmemPerBlock; the others use kThreads
// threads and none.
constexpr int kSmemPerBlock = 48 * 1024;

struct LaunchShape {
  unsigned threads;
  size_t smem;
};

inline LaunchShape shape_of(int sl_words) {
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

template <int W, bool SL, bool DBG>
cudaError_t launch_sample_k(const LaunchArgs& a, const LaunchShape& sh, unsigned blocks) {
  auto k = k_sample<W, SL, DBG>;
  cudaError_t e = allow_smem(k, sh.smem);
  if (e != cudaSuccess) return e;
  k<<<blocks, sh.threads, sh.smem, a.stream>>>(a.v, round_keys(a.seed), a.shot_offset, a.shots, a.meas, a.det, a.obs,
                                               a.accept, a.dump, a.dump_row, a.dump_stride);
  return cudaGetLastError();
}

template <int W>
cudaError_t launch_sample(const LaunchArgs& a) {
  const DevView& v = a.v;
  const LaunchShape sh = shape_of(sl_warp_words(W, v.sl_par, v.sl_rb));
  const uint64_t blocks = (a.shots + sh.threads - 1) / sh.threads;
  if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
  const bool dbg = a.dump != nullptr;
  if (v.sl_par > 0)
    return dbg ? launch_sample_k<W, true, true>(a, sh, (unsigned)blocks)
               : launch_sample_k<W, true, false>(a, sh, (unsigned)blocks);
  return dbg ? launch_sample_k<W, false, true>(a, sh, (unsigned)blocks)
             : launch_sample_k<W, false, false>(a, sh, (unsigned)blocks);
}

template <int W>
cudaError_t launch_batch_group(const BatchLaunchArgs& a) {
  // every warp gets room for the transposed X at the launch's W, the
  // largest sliced parity buffer and the largest row buffers of the group
  const LaunchShape sh = shape_of(sl_warp_words(W, a.sl_par, a.sl_rb));
  if (a.sl_par > 0) {
    cudaError_t e = allow_smem(k_batch<W, true>, sh.smem);
    if (e != cudaSuccess) return e;
    k_batch<W, true><<<a.grid, sh.threads, sh.smem, a.stream>>>(a.progs, a.n, a.item_start, a.total_items, a.sb,
                                                                a.counter, a.sl_par, a.sl_rb);
  } else {
    k_batch<W, false><<<a.grid, sh.threads, 0, a.stream>>>(a.progs, a.n, a.item_start, a.total_items, a.sb,
                                                           a.counter, 0, 0);
  }
  return cudaGetLastError();
}

}  // namespace tsim
