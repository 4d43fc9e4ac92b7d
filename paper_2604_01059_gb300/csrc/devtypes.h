// Types shared by the host-side packer (device.cu) and the sampling kernels
// (kernels.cuh, instantiated per X width in kern_w*.cu): the packed program
// view and its records, the Philox round keys, and the launch arguments.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace tsim {

enum : int { ST_NOT_REAL = 1, ST_OVERFLOW = 2, ST_ZERO_PROB = 4, ST_TIMEOUT = 8 };

constexpr int kMaxChains = 16;
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
// FLOAT = the tables of a chain with arbitrary rotation angles: per thread,
// as SCALAR, with each class's coefficient a complex double and its
// arbitrary-angle factors e^(i pi t a) summed into one phase.
enum : int { TAB_SCALAR = 0, TAB_BASIS = 1, TAB_SLICED = 2, TAB_FLOAT = 3 };
// A marginal table.  cst = 1: its value does not depend on the shot (no
// factor has a nonzero parity) and is precomputed in DevView::tconst, with
// the chain rotation of a normalisation in rot (-1 when not precomputed).
struct DTable { uint32_t par_off, n_par, cls_off, n_cls; int32_t base, mode, sb_off, n_sb, stage, cst, rot, pad; };
// the precomputed value (c0 + c1 w + c2 w^2 + c3 w^3) sqrt2^base of a constant table
struct DConst { long long c[4]; };
// A class of merged terms.  SCALAR / BASIS: coefficient w^j0 (mono) or c[4]
// in Z[w], magnitude sqrt2^d0 over the table base.  FLOAT: fac_off / n_fac
// its exact factors, j0 / pad the offset and count of its arbitrary-angle
// factors, c[0] and c[1] the bits of the real and imaginary parts of its
// complex coefficient (all magnitudes included).
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
constexpr uint32_t kSlWalk = 0xFFFFFFFFu;  // parity bit indices absent (> 8 bits): walk the mask
constexpr int kSlMaxPar = 16384;       // parity words of one segment (4q fits 16 bits)
// One batch of 32 terms: rows of operation code c are cnt[c] (a multiple of
// 4) x 32 parity offsets, padded with no-op offsets and stored in groups of 4
// rows as [group][lane][4], starting at row_off.
// All terms of a batch share the magnitude sqrt2^d; j0m[b] holds bit b of
// each lane's constant phase; valid marks lanes that carry a term.
struct DSBatch { uint32_t row_off; uint16_t cnt[8]; int32_t d; uint32_t j0m[3]; uint32_t valid; };
// A sliced table is a list of segments: consecutive terms whose distinct
// parities (par_off, n_par masks) fit one shared buffer, and their batches.
// k8 = 1 when some parity of the segment names more than four X bits (its
// words are then formed from eight bit indices, else from four).
struct DSeg { uint32_t par_off, n_par, sb_off, n_sb, k8; };

// One group of the geometric-gap noise rule: Q, member count n, the offset
// of its member channel indices and of its table T_1..T_n (the same offset
// into both arrays), T_n (a word U < T_n leaves no candidate in the group:
// the common case, decided without reading the table), and 1 / log2(Q / 2^32)
// (the slope of the gap estimate; the gap itself is decided on the table).
struct DGroup { uint32_t Q, n, off, tn; float rlq; };

struct DevView {
  int W;
  int n_ch, n_out, n_ent, n_chains, n_tab;
  int nmeas, ndet, nobs, mode;
  int* status;            // status word of the launch's device: bits ST_*, read by tsim_sync
  int noise_mode, n_grp;  // 0: one word per channel; 1: geometric gaps over the groups
  const DGroup* grp;
  const uint32_t* gmem;   // member channel indices of every group
  const uint32_t* gT;     // per group T_1..T_n (T_k at index k - 1)
  const DChan* ch;
  const uint4* thr0;      // outcome-0 threshold per channel, 4 per block, padded with 2^32-1
  const uint32_t* thr;
  const uint64_t* sig;
  const DOut* out;
  const uint64_t* omask;
  const int32_t* chain_norm;
  const DTable* tab;
  const uint64_t* par;    // per table: n_par masks of W words (mask 0 = zero)
  const uint2* pidx;      // per parity slot: eight 8-bit X bit indices, or .x = kSlWalk
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
  const DConst* tconst;        // per table: its value when constant
  const uint64_t* dmask;       // measurement mode: per detector a mask over X (W words) ...
  const uint64_t* omask2;      // ... and per observable; the constants in dcst / ocst
  const int32_t* dcst;
  const int32_t* ocst;
  const int32_t* chain_float;  // per chain: 1 when its tables are FLOAT
  const uint32_t* ffidx;       // FLOAT tables: parity index of each arbitrary-angle factor
  const double* ffang;         // FLOAT tables: its angle, in units of pi
};

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


// A warp's shared words for sliced tables: transposed X (64 W), parity words
// (par), two row staging buffers (rb each), two mbarriers and a state word.
__host__ __device__ __forceinline__ int sl_round32(int x) { return (x + 31) & ~31; }

__host__ __device__ __forceinline__ int sl_warp_words(int W, int par, int rb) {
  if (par <= 0) return 0;
  return sl_round32(64 * W + par) + (rb > 0 ? 2 * rb + 32 : 0);
}

// One program of a batched launch (device copy of the plan).
struct BatchProg {
  DevView v;
  uint64_t shots, seed, shot_offset;
  uint64_t* meas;
  uint64_t* det;
  uint64_t* obs;
  uint8_t* accept;
};

// Arguments of one program's sampling launch.  dump / dump_row: debug
// record of every table evaluation of the shots with dump_row[s] >= 0 (NULL
// in production launches).
struct LaunchArgs {
  DevView v;
  cudaStream_t stream;
  uint64_t seed, shot_offset, shots;
  uint64_t* meas;
  uint64_t* det;
  uint64_t* obs;
  uint8_t* accept;
  long long* dump;
  const int32_t* dump_row;
  int dump_stride;  // long longs per dumped shot
};

// Arguments of one persistent launch over the work items of a batch group.
struct BatchLaunchArgs {
  const BatchProg* progs;
  int n;
  const uint64_t* item_start;
  uint64_t total_items;
  uint32_t sb;
  unsigned long long* counter;
  int sl_par, sl_rb;
  cudaStream_t stream;
  unsigned grid;
};

// Words of one debug record: table, the four Z[w] coefficients, the sqrt2
// exponent, then the W words of X at which the table was evaluated.  For a
// FLOAT table the first two coefficient words hold the bits of the real and
// imaginary parts of its complex value and the exponent word is kDumpFloat.
constexpr int kDumpHead = 6;
constexpr long long kDumpFloat = -2147483648ll;

// Sampling launchers, one instantiation per padded X width W (kern_w<W>.cu).
template <int W>
cudaError_t launch_sample(const LaunchArgs& a);
template <int W>
cudaError_t launch_batch_group(const BatchLaunchArgs& a);

}  // namespace tsim
