// Compiled program: the contiguous tables the sampler evaluates per shot
// (Sec. "Methods": the compiled sampler; Appendix "Parameterized evaluation of
// Clifford ZX diagrams": the tensors c^t, alpha_k^t, beta_k^t, u_ki^t, v_ki^t).
//
// Per shot the sampler keeps a bit vector X of n_x bits laid out as
//   [ f bits used by marginal tables (nft) | random outputs (nr) | other f bits ]
// where f = T e mod 2 (Eq. detector_sampling) and "random outputs" are the
// outputs drawn by Algorithm 1.  Every parity of the program is a mask over X.
#pragma once
#include <atomic>
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "common.h"

namespace tsim {

struct ProgFactor {
  int kind = 0, alpha = 0, beta = 0;    // FactorKind, angles in units of pi/4
  double t = 0;                         // F_PHASE_F: e^(i pi t a), t in units of pi
  std::vector<uint64_t> u, v;           // parities a = <u, X>, b = <v, X>
};

struct ProgTerm {
  int s0 = 0, j0 = 0;                   // c^t = w^j0 * sqrt2^s0 (* e^(i pi fph))
  double fph = 0;                       // constant phase of arbitrary rotations, units of pi
  std::vector<ProgFactor> f;
};

struct ProgTable {
  std::vector<ProgTerm> terms;
  // some term has an arbitrary phase: the table is evaluated in floating point
  bool is_float() const;
};

struct ProgOutput {
  bool random = false;
  std::vector<uint64_t> mask;           // deterministic: bit = <mask, X> ^ cst
  int cst = 0;
  int xbit = -1, chain = -1, table = -1;  // random: X bit written, chain, marginal table
};

struct ProgChannel {
  std::vector<uint32_t> thr;            // outcome o (< n-1) iff U < thr[o] (first such)
  std::vector<std::vector<uint64_t>> sig;  // per outcome: X ^= sig
  std::vector<double> probs;            // outcome probabilities (double, before quantisation)
};

// Noise by geometric gaps (Sec. "Detectors": the gap between successive
// firing events is geometric).  Group g holds channels whose outcome-0
// thresholds are all >= Q; candidates are Bernoulli(1 - Q / 2^32) trials
// along the group, placed by one geometric gap per word, and a candidate
// channel keeps its own outcome distribution through a second word mapped
// onto [Q, 2^32).
struct NoiseGroup {
  uint32_t Q = 0;
  std::vector<int> member;  // channel indices, in sampling order
};

struct RawInfo {
  int nbits = 0;
  std::vector<double> probs;                 // 2^nbits
  std::vector<std::vector<uint64_t>> cols;   // per bit: its column of T in the X layout
};

struct DeviceProgram;  // opaque device-side cache (uploaded tables)
struct DeviceTables;   // host-side packed device tables

struct Program {
  int mode = 0;
  int nq = 0, nmeas = 0, ndet = 0, nobs = 0, E = 0;
  int nx = 0, W = 1, nf = 0, nr = 0, nft = 0;
  std::vector<ProgOutput> outputs;
  std::vector<int> chain_norm;           // normalisation table of each chain
  std::vector<ProgChannel> channels;
  int noise_mode = 0;                    // 0: one word per channel; 1: geometric gaps over `groups`
  std::vector<NoiseGroup> groups;
  std::vector<ProgTable> tables;
  std::vector<std::vector<int>> detmap, obsmap;  // measurement mode only
  std::vector<RawInfo> raw;
  DeviceProgram* dev = nullptr;
  DeviceTables* devtab = nullptr;
  ~Program();
};

Program* compile_program(const std::string& text, const tsim_compile_opts& opts);
void save_program(const Program& p, const std::string& path);
Program* load_program(const std::string& path);
ZW eval_table_host(const Program& p, int t, const uint64_t* x);
// any table (with or without arbitrary phases) in complex double
std::complex<double> eval_table_host_c(const Program& p, int t, const uint64_t* x);
// Noise sampling mode: 0 one word per channel, 1 geometric gaps, -1 the
// cheaper of the two by expected random words per shot (groups are formed
// from the channels' outcome-0 thresholds).  Does not re-pack device tables.
void set_noise_sampling(Program& p, int mode);
// expected random words per shot of each mode: [0] one per channel, [1] geometric
void noise_word_estimate(const Program& p, double out[2]);

struct Graph;
// The diagram of every marginal of a circuit after the Clifford rewrites, in
// the order the compiler decomposes them (nothing is decomposed).
std::vector<Graph> marginal_diagrams(const std::string& text, int mode);

// Scores the spiders of a decomposition root (indexed by uid) for the learned
// cut order; returns false when no model or no GPU is available.
using CutScorer = bool (*)(const Graph&, std::vector<double>&);
extern std::atomic<CutScorer> g_cut_scorer;
// learned-order bookkeeping: [0] scorer calls, [1] calls that returned scores,
// [2] marginals where the learned order was kept, [3] where the heuristic won
extern std::atomic<uint64_t> g_cut_stats[4];

// message for tsim_last_error(); copies into a fixed thread-local buffer
void set_last_error(const char* msg);

}  // namespace tsim

// the opaque handle behind tsim_program*
struct tsim_program {
  tsim::Program* p;
};
