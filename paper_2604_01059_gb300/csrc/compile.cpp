// Host compiler: circuit -> compiled program.
//
// Pipeline (Sec. "Simulation pipeline"):
//  1. The noisy circuit becomes a doubled parameterised diagram of the joint
//     output distribution P(outputs | e): every gate acts on a ket copy and a
//     conjugated bra copy (Appendix "Doubled ZX notation"), Pauli noise enters
//     as parameters e_i (Appendix "Pauli noise channels"), measurements tie the
//     two copies together (Eq. measurement), outputs are XORs of measurement
//     outcomes (Eq. xor) and unrecorded wires are traced (Eq. trace).
//  2. Clifford rewriting reduces it.  Outputs that end up fixed by a single
//     parity constraint are deterministic given e and earlier outputs (each
//     detector "is directly determined by a single f_i", Sec. "Detectors");
//     the remaining outputs split into connected components, each sampled by
//     its own autoregressive chain (Sec. "Observables").
//  3. For every chain: the normalisation diagram (all outputs traced) and one
//     marginal diagram per output (later outputs traced), each decomposed into
//     Clifford terms (Appendix "Stabilizer decompositions") whose values are
//     products of phase factors (Appendix "Parameterized evaluation").
//  4. GF(2) elimination picks a minimal set of f_i (Eq. detector_sampling) and
//     the noise channels are reduced (Appendix "Channel reduction").
#include <algorithm>
#include <thread>
#include <mutex>
#include <exception>
#include <atomic>
#include <array>
#include <cmath>
#include <functional>
#include <map>
#include <memory>
#include <numeric>
#include <unordered_map>

#include <cuda_runtime.h>

#include "circuit.h"
#include "device.h"
#include "program.h"
#include "zx.h"

namespace tsim {
namespace {

struct Builder {
  const Circuit& C;
  int mode;
  int E, nout;
  size_t np;
  std::vector<char> is_param;  // per output
  Graph g;
  std::vector<Form> ket, bra, mk, mb;

  Builder(const Circuit& c, int mode_, const std::vector<char>& param_outputs)
      : C(c), mode(mode_), is_param(param_outputs) {
    E = c.num_error_bits;
    nout = (int)param_outputs.size();
    np = (size_t)E + (size_t)nout;
    g = Graph(np);
  }

  Form zero() const { return form_const(np, 0); }

  void hgate(Form& f) {
    int y = g.add_var(0);
    g.add_sign(form_var(np, y), f);
    g.s2 -= 1;
    f = form_var(np, y);
  }
  void H(int q) { hgate(ket[(size_t)q]); hgate(bra[(size_t)q]); }
  void phase(int q, int th) {
    g.add_phase(th, ket[(size_t)q]);
    g.add_phase(-th, bra[(size_t)q]);
  }
  // R_Z(t) = diag(e^(-i pi t/2), e^(i pi t/2)) ~ diag(1, e^(i pi t)): the
  // global phase cancels between the two copies
  void phase_f(int q, double t) {
    g.add_phase_f(t, ket[(size_t)q]);
    g.add_phase_f(-t, bra[(size_t)q]);
  }
  void rx(int q, double t) { H(q); phase_f(q, t); H(q); }
  // R_Y(t) = S R_X(t) S^dag (S X S^dag = Y); in time order S^dag first
  void ry(int q, double t) { phase(q, 6); rx(q, t); phase(q, 2); }
  void Xg(int q) { ket[(size_t)q].c ^= 1; bra[(size_t)q].c ^= 1; }
  void Zg(int q) { phase(q, 4); }
  void CX(int c, int t) { form_xor(ket[(size_t)t], ket[(size_t)c]); form_xor(bra[(size_t)t], bra[(size_t)c]); }
  void CZ(int a, int b) {
    g.add_sign(ket[(size_t)a], ket[(size_t)b]);
    g.add_sign(bra[(size_t)a], bra[(size_t)b]);
  }
  void trace(int q) {
    Form f = ket[(size_t)q];
    form_xor(f, bra[(size_t)q]);
    if (f.vars.empty() && !f.params.any() && f.c == 0) return;  // delta(0 = 0)
    g.hub(f);
  }
  void noise_x(int q, int bit) { ket[(size_t)q].params.flip((size_t)bit); bra[(size_t)q].params.flip((size_t)bit); }
  void noise_z(int q, int bit) {
    g.add_sign(form_param(np, bit), ket[(size_t)q]);
    g.add_sign(form_param(np, bit), bra[(size_t)q]);
  }
  void measure(int q, int flip_bit) {
    trace(q);  // the measurement ties both copies: delta(ket = bra)
    Form a = ket[(size_t)q], b = bra[(size_t)q];
    if (flip_bit >= 0) { a.params.flip((size_t)flip_bit); b.params.flip((size_t)flip_bit); }
    mk.push_back(a);
    mb.push_back(b);
  }
  void reset(int q) { ket[(size_t)q] = zero(); bra[(size_t)q] = zero(); }

  void build() {
    ket.assign((size_t)C.num_qubits, zero());
    bra.assign((size_t)C.num_qubits, zero());
    std::map<std::pair<int, int>, int> mflip;  // (instr, target pos) -> raw bit
    std::map<int, std::vector<const RawChannel*>> chans;
    for (const RawChannel& ch : C.channels) {
      if (ch.kind == Op::M) mflip[{ch.instr, ch.target_pos}] = ch.first_bit;
      else chans[ch.instr].push_back(&ch);
    }
    for (size_t idx = 0; idx < C.ins.size(); ++idx) {
      const Instr& in = C.ins[idx];
      auto tq = [&](size_t k) { return in.t[k].v; };
      switch (in.op) {
        case Op::I: case Op::DETECTOR: case Op::OBSERVABLE_INCLUDE: break;
        case Op::X: for (size_t k = 0; k < in.t.size(); ++k) Xg(tq(k)); break;
        case Op::Z: for (size_t k = 0; k < in.t.size(); ++k) Zg(tq(k)); break;
        case Op::Y:  // Y = i X Z; the i cancels between the two copies
          for (size_t k = 0; k < in.t.size(); ++k) { Zg(tq(k)); Xg(tq(k)); }
          break;
        case Op::H: for (size_t k = 0; k < in.t.size(); ++k) H(tq(k)); break;
        case Op::S: for (size_t k = 0; k < in.t.size(); ++k) phase(tq(k), 2); break;
        case Op::S_DAG: for (size_t k = 0; k < in.t.size(); ++k) phase(tq(k), 6); break;
        case Op::T: for (size_t k = 0; k < in.t.size(); ++k) phase(tq(k), 1); break;
        case Op::T_DAG: for (size_t k = 0; k < in.t.size(); ++k) phase(tq(k), 7); break;
        case Op::R_Z: for (size_t k = 0; k < in.t.size(); ++k) phase_f(tq(k), in.args[0]); break;
        case Op::R_X: for (size_t k = 0; k < in.t.size(); ++k) rx(tq(k), in.args[0]); break;
        case Op::R_Y: for (size_t k = 0; k < in.t.size(); ++k) ry(tq(k), in.args[0]); break;
        case Op::U3:  // U3(theta, phi, lambda) ~ R_Z(phi) R_Y(theta) R_Z(lambda)
          for (size_t k = 0; k < in.t.size(); ++k) {
            phase_f(tq(k), in.args[2]);
            ry(tq(k), in.args[0]);
            phase_f(tq(k), in.args[1]);
          }
          break;
        case Op::SQRT_X: case Op::SQRT_X_DAG:  // H S H, H S_DAG H
          for (size_t k = 0; k < in.t.size(); ++k) {
            H(tq(k));
            phase(tq(k), in.op == Op::SQRT_X ? 2 : 6);
            H(tq(k));
          }
          break;
        case Op::CX: case Op::CY: case Op::CZ: case Op::SWAP:
          for (size_t k = 0; k + 1 < in.t.size(); k += 2) {
            int b = in.t[k + 1].v;
            if (in.t[k].rec) {
              int j = (int)mk.size() + in.t[k].v;
              // classically controlled Pauli: X^m and/or Z^m on both copies
              if (in.op == Op::CX || in.op == Op::CY) {
                form_xor(ket[(size_t)b], mk[(size_t)j]);
                form_xor(bra[(size_t)b], mb[(size_t)j]);
              }
              if (in.op == Op::CZ || in.op == Op::CY) {
                g.add_sign(mk[(size_t)j], ket[(size_t)b]);
                g.add_sign(mb[(size_t)j], bra[(size_t)b]);
              }
              continue;
            }
            int a = in.t[k].v;
            if (in.op == Op::CX) CX(a, b);
            else if (in.op == Op::CZ) CZ(a, b);
            else if (in.op == Op::CY) { phase(b, 6); CX(a, b); phase(b, 2); }
            else { std::swap(ket[(size_t)a], ket[(size_t)b]); std::swap(bra[(size_t)a], bra[(size_t)b]); }
          }
          break;
        case Op::R: for (size_t k = 0; k < in.t.size(); ++k) { trace(tq(k)); reset(tq(k)); } break;
        case Op::RX:
          for (size_t k = 0; k < in.t.size(); ++k) { trace(tq(k)); reset(tq(k)); H(tq(k)); }
          break;
        case Op::M: case Op::MX: case Op::MR: case Op::MRX:
          for (size_t k = 0; k < in.t.size(); ++k) {
            int q = tq(k);
            auto it = mflip.find({(int)idx, (int)k});
            int fb = it == mflip.end() ? -1 : it->second;
            bool xb = in.op == Op::MX || in.op == Op::MRX;
            if (xb) H(q);
            measure(q, fb);
            if (in.op == Op::MR || in.op == Op::MRX) reset(q);
            if (xb) H(q);
          }
          break;
        default: {  // noise channels
          auto it = chans.find((int)idx);
          if (it == chans.end()) break;
          for (const RawChannel* ch : it->second) {
            int b0 = ch->first_bit;
            switch (ch->kind) {
              case Op::X_ERROR: noise_x(ch->q0, b0); break;
              case Op::Z_ERROR: noise_z(ch->q0, b0); break;
              case Op::Y_ERROR: noise_z(ch->q0, b0); noise_x(ch->q0, b0); break;
              case Op::DEPOLARIZE1: case Op::PAULI_CHANNEL_1:
                noise_z(ch->q0, b0 + 1);
                noise_x(ch->q0, b0);
                break;
              case Op::DEPOLARIZE2: case Op::PAULI_CHANNEL_2:
                noise_z(ch->q0, b0 + 1);
                noise_x(ch->q0, b0);
                noise_z(ch->q1, b0 + 3);
                noise_x(ch->q1, b0 + 2);
                break;
              default: fail(TSIM_ERR_INTERNAL, "unknown channel kind");
            }
          }
          break;
        }
      }
    }
    for (int q = 0; q < C.num_qubits; ++q) trace(q);
    // outputs that are parameters of this diagram: delta(o = XOR of records)
    for (int i = 0; i < nout; ++i) {
      if (!is_param[(size_t)i]) continue;
      Form f = form_param(np, E + i);
      if (mode == TSIM_MODE_MEASUREMENTS) {
        form_xor(f, mk[(size_t)i]);
      } else {
        const std::vector<int>& recs =
            i < (int)C.detectors.size() ? C.detectors[(size_t)i] : C.observables[(size_t)(i - (int)C.detectors.size())];
        for (int j : recs) form_xor(f, mk[(size_t)j]);
      }
      g.hub(f);
    }
  }
};

// GF(2) row used by the output elimination: parity v (over all params) = c
struct DeltaRow {
  Bits v;
  int c = 0;
  int piv = -1;
};

// Minimal f basis (Eq. detector_sampling): Gaussian elimination over GF(2)
// of the error-bit parities that the program needs.
struct FBasis {
  std::vector<Bits> orig, vec, comb;
  std::vector<int> piv;
  Bits express(const Bits& g) {
    Bits v = g, cm;
    for (size_t i = 0; i < vec.size(); ++i)
      if (v.get((size_t)piv[i])) { v ^= vec[i]; cm ^= comb[i]; }
    if (!v.any()) return cm;
    size_t k = orig.size();
    orig.push_back(g);
    Bits nc = cm;
    if (nc.nwords() * 64 <= k) nc.w.resize(k / 64 + 1, 0);
    nc.flip(k);
    vec.push_back(v);
    comb.push_back(nc);
    piv.push_back(v.first());
    Bits m;
    m.w.resize(k / 64 + 1, 0);
    m.flip(k);
    return m;
  }
};

Bits restrict_bits(const Bits& b, size_t lo, size_t hi) {  // bits [lo, hi) shifted to 0
  Bits r(hi - lo);
  b.for_each([&](int i) {
    if ((size_t)i >= lo && (size_t)i < hi) r.set((size_t)i - lo);
  });
  return r;
}

struct BitsHash {
  size_t operator()(const Bits& b) const {
    uint64_t h = 1469598103934665603ull;
    size_t n = b.w.size();
    while (n && !b.w[n - 1]) --n;  // equal Bits may differ in trailing zero words
    for (size_t i = 0; i < n; ++i) h = (h ^ b.w[i]) * 1099511628211ull;
    return (size_t)h;
  }
};

struct RChan {
  std::vector<Bits> cols;  // F-space columns, one per bit
  std::vector<double> p;   // 2^k
  int first_raw = 0;
};

// distribution over the remaining bits after summing out bit `b`
void marginalize_bit(RChan& ch, size_t b) {
  size_t k = ch.cols.size();
  std::vector<double> np_((size_t)1 << (k - 1), 0.0);
  for (size_t o = 0; o < ch.p.size(); ++o) {
    size_t lo = o & ((1ull << b) - 1), hi = o >> (b + 1);
    np_[lo | (hi << b)] += ch.p[o];
  }
  ch.p.swap(np_);
  ch.cols.erase(ch.cols.begin() + (long)b);
}

// merge bit j into bit i (identical columns): new bit i = b_i XOR b_j
void merge_bits(RChan& ch, size_t i, size_t j) {
  std::vector<double> q(ch.p.size(), 0.0);
  for (size_t o = 0; o < ch.p.size(); ++o) {
    size_t bi = (o >> i) & 1, bj = (o >> j) & 1;
    size_t o2 = (o & ~(1ull << i)) | ((bi ^ bj) << i);
    o2 &= ~(1ull << j);
    q[o2] += ch.p[o];
  }
  ch.p.swap(q);
  marginalize_bit(ch, j);  // bit j is now always 0: summing it out keeps the rest
}

void canonicalize(RChan& ch) {
  // sort bits by column and merge duplicates (Appendix "Channel reduction",
  // step 2, "channel normalization")
  for (;;) {
    bool again = false;
    for (size_t i = 0; i < ch.cols.size() && !again; ++i)
      for (size_t j = i + 1; j < ch.cols.size() && !again; ++j)
        if (ch.cols[i] == ch.cols[j]) { merge_bits(ch, i, j); again = true; }
    if (!again) break;
  }
  size_t k = ch.cols.size();
  std::vector<size_t> perm(k);
  std::iota(perm.begin(), perm.end(), 0);
  std::sort(perm.begin(), perm.end(), [&](size_t a, size_t b) { return ch.cols[a] < ch.cols[b]; });
  std::vector<Bits> nc(k);
  std::vector<double> q(ch.p.size(), 0.0);
  for (size_t i = 0; i < k; ++i) nc[i] = ch.cols[perm[i]];
  for (size_t o = 0; o < ch.p.size(); ++o) {
    size_t o2 = 0;
    for (size_t i = 0; i < k; ++i) o2 |= ((o >> perm[i]) & 1) << i;
    q[o2] += ch.p[o];
  }
  ch.cols.swap(nc);
  ch.p.swap(q);
}

// XOR convolution, P(o) = sum_{a ^ b = o} P_A(a) P_B(b) (step 3)
void xor_convolve(RChan& into, const std::vector<double>& pb) {
  std::vector<double> q(into.p.size(), 0.0);
  for (size_t a = 0; a < into.p.size(); ++a)
    for (size_t b = 0; b < pb.size(); ++b) q[a ^ b] += into.p[a] * pb[b];
  into.p.swap(q);
}

std::vector<uint64_t> to_words(const Bits& b, int W) {
  std::vector<uint64_t> w((size_t)W, 0);
  b.for_each([&](int i) { w[(size_t)i >> 6] |= 1ull << (i & 63); });
  return w;
}

}  // namespace

std::atomic<CutScorer> g_cut_scorer{nullptr};

// Spare host threads for decomposing marginals: the process shares
// hardware_concurrency - 1 helpers among concurrent compilations, so that
// compiling many programs on many threads does not oversubscribe the cores.
std::atomic<int> g_helpers_free{-1};
int acquire_helpers(int want) {
  if (want <= 0) return 0;
  int cur = g_helpers_free.load();
  if (cur < 0) {
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    g_helpers_free.compare_exchange_strong(cur, hw - 1);
    cur = g_helpers_free.load();
  }
  for (;;) {
    if (cur <= 0) return 0;
    const int take = std::min(cur, want);
    if (g_helpers_free.compare_exchange_weak(cur, cur - take)) return take;
  }
}
void release_helpers(int n) {
  if (n > 0) g_helpers_free.fetch_add(n);
}
std::atomic<uint64_t> g_cut_stats[4];

// Decompose one marginal diagram.  LEARNED: the spiders of the simplified
// diagram are scored by the cut-order network, cut units are ranked by their
// best member, and learned unit orders are tried against the heuristic order,
// which judges (a learned order is kept only with strictly fewer terms; every
// order gives the same exact sum).  Without a scorer LEARNED falls back to
// the heuristic.
// When set, compile_program records each marginal's diagram after the
// Clifford rewrites and stops before decomposing anything.
thread_local std::vector<Graph>* g_marginal_capture = nullptr;
struct CaptureDone {};

void decompose_marginal(Graph M, const tsim_compile_opts& opts, uint64_t budget, uint64_t* total,
                        std::vector<Term>& out, std::atomic<uint64_t>* shared_total) {
  if (g_marginal_capture) {
    M.simplify();
    M.compact();
    g_marginal_capture->push_back(std::move(M));
    return;
  }
  DecompStats st;
  st.budget = budget;
  st.total = total;
  st.total_budget = opts.total_budget;
  const CutScorer scorer = g_cut_scorer.load();
  if (opts.decomp != TSIM_DECOMP_LEARNED || !scorer) {
    // one decomposition per marginal: its terms count toward the program's
    // budget as they are made (LEARNED tries several and counts the kept one)
    st.shared_total = shared_total;
    decompose(M, opts.decomp == TSIM_DECOMP_LEARNED ? TSIM_DECOMP_HEURISTIC : opts.decomp, out, st);
    return;
  }
  M.simplify();
  M.compact();
  for (int v = 0; v < M.n; ++v) M.uid[(size_t)v] = v;
  std::vector<double> scores;
  g_cut_stats[0]++;
  if (!scorer(M, scores)) {
    decompose(M, TSIM_DECOMP_HEURISTIC, out, st);
    return;
  }
  // The network was trained to rank cut units (a cancelling ket/bra pair of
  // one T gate, or a single spider) by the terms when that unit is split
  // first and the rest follow the heuristic: decompose the heuristic order,
  // then the three best-ranked units first, then every unit in the
  // network's order, each with the fewest terms so far as its budget (a
  // worse order stops as soon as it exceeds it).  The heuristic is the
  // fallback and the judge: a learned order is kept only when it has
  // strictly fewer terms.
  std::vector<Term> heuristic;
  DecompStats s2 = st;
  uint64_t t2 = total ? *total : 0;
  s2.total = &t2;
  bool ok2 = true;
  try { decompose(M, TSIM_DECOMP_HEURISTIC, heuristic, s2); } catch (const Error& e) {
    if (e.code != TSIM_ERR_CHI_BUDGET) throw;
    ok2 = false;
  }
  // cut units (cancelling ket/bra pairs and single spiders), each scored by
  // its best member; the heuristic splits them in id order (unit 0 first)
  const std::vector<std::vector<int>> units = cut_units(M);
  std::vector<double> us(units.size(), 1e300);
  for (size_t u = 0; u < units.size(); ++u)
    for (int v : units[u]) us[u] = std::min(us[u], scores[(size_t)v]);
  std::vector<int> rank(units.size());
  for (size_t u = 0; u < rank.size(); ++u) rank[u] = (int)u;
  std::stable_sort(rank.begin(), rank.end(), [&](int a, int b) { return us[(size_t)a] < us[(size_t)b]; });
  std::vector<Term> learned;
  uint64_t t1 = t2;
  bool ok1 = false;
  auto trial_order = [&](const std::vector<int>& order) {
    std::vector<Term> trial;
    DecompStats s1 = st;
    uint64_t tt = total ? *total : 0;
    s1.total = &tt;
    const uint64_t best = ok1 ? learned.size() : (ok2 ? heuristic.size() : 0);
    if (best) s1.budget = std::min<uint64_t>(s1.budget ? s1.budget : best, best > 1 ? best - 1 : 1);
    const std::vector<double> sc = unit_order_scores(M, units, order);
    try {
      decompose(M, TSIM_DECOMP_LEARNED, trial, s1, &sc);
    } catch (const Error& e) {
      if (e.code != TSIM_ERR_CHI_BUDGET) throw;
      return;
    }
    if (!ok1 || trial.size() < learned.size()) {
      learned.swap(trial);
      t1 = tt;
      ok1 = true;
    }
  };
  // the three best-ranked units split first (the rest in the heuristic
  // order), then every unit in the network's order
  int tried = 0;
  for (size_t k = 0; k < rank.size() && tried < 3; ++k) {
    if (rank[k] == 0) continue;  // the heuristic's own first unit
    ++tried;
    std::vector<int> order{rank[k]};
    for (size_t u = 0; u < units.size(); ++u)
      if ((int)u != rank[k]) order.push_back((int)u);
    trial_order(order);
  }
  if (units.size() > 2) trial_order(rank);
  if (!ok1 && !ok2) fail(TSIM_ERR_CHI_BUDGET, "stabilizer terms exceed the budget");
  g_cut_stats[1]++;
  const bool use_learned = ok1 && (!ok2 || learned.size() < heuristic.size());
  g_cut_stats[use_learned ? 2 : 3]++;
  out = use_learned ? std::move(learned) : std::move(heuristic);
  if (total) *total = use_learned ? t1 : t2;
}

Program* compile_program(const std::string& text, const tsim_compile_opts& opts) {
  Circuit C = parse_circuit(text);
  auto prog = std::make_unique<Program>();
  Program& P = *prog;
  P.mode = opts.mode;
  P.nq = C.num_qubits;
  P.nmeas = C.num_measurements;
  P.ndet = (int)C.detectors.size();
  P.nobs = (int)C.observables.size();
  P.E = C.num_error_bits;
  const int E = P.E;
  const int nout = opts.mode == TSIM_MODE_MEASUREMENTS ? P.nmeas : P.ndet + P.nobs;
  const size_t np = (size_t)E + (size_t)nout;
  const uint64_t budget = opts.chi_budget ? opts.chi_budget : (1ull << 20);
  uint64_t total_terms = 0;

  // ---- 1-2: joint diagram, Clifford rewriting
  Builder J(C, opts.mode, std::vector<char>((size_t)nout, 1));
  J.build();
  Graph& G = J.g;
  G.simplify();
  G.compact();
  if (G.zero) fail(TSIM_ERR_INTERNAL, "joint distribution reduced to zero");

  // deterministic outputs: delta factors Node(0 or pi; a) whose parity names outputs
  std::vector<DeltaRow> rows;
  std::vector<Factor> rest;
  for (Factor& f : G.fac) {
    bool is_delta = f.kind == F_NODE && (f.alpha == 0 || f.alpha == 4) && f.a.last() >= E;
    if (!is_delta) { rest.push_back(f); continue; }
    DeltaRow r;
    r.v = f.a;
    r.c = f.alpha >> 2;
    for (const DeltaRow& o : rows)
      if (r.v.get((size_t)o.piv)) { r.v ^= o.v; r.c ^= o.c; }
    int p = r.v.last();
    if (p < E) {
      if (r.v.any() || r.c) fail(TSIM_ERR_INTERNAL, "output-free constraint in the joint distribution");
      continue;
    }
    r.piv = p;
    for (DeltaRow& o : rows)
      if (o.v.get((size_t)p)) { o.v ^= r.v; o.c ^= r.c; }
    rows.push_back(r);
  }
  std::vector<int> pivot_row((size_t)nout, -1);
  for (size_t i = 0; i < rows.size(); ++i) pivot_row[(size_t)(rows[i].piv - E)] = (int)i;

  // substitute the deterministic outputs everywhere else
  auto apply_rules = [&](Bits& a, int& c) {
    for (const DeltaRow& r : rows)
      if (a.get((size_t)r.piv)) { a ^= r.v; c ^= r.c; }
  };
  G.fac.clear();
  for (Factor f : rest) {
    int ca = 0, cb = 0;
    apply_rules(f.a, ca);
    apply_rules(f.b, cb);
    switch (f.kind) {
      case F_NODE: G.add_factor(F_NODE, f.alpha + 4 * ca, 0, f.a, f.b); break;
      case F_PHASE:
        if (ca) { G.ph = (G.ph + f.alpha) & 7; f.alpha = -f.alpha; }
        G.add_factor(F_PHASE, f.alpha, 0, f.a, f.b);
        break;
      case F_PHASE_F:
        if (ca) { G.fph = angle_mod2(G.fph + f.t); f.t = -f.t; }
        G.add_factor_f(f.t, f.a);
        break;
      case F_PI_PAIR:
        G.add_factor(F_PI_PAIR, 0, 0, f.a, f.b);
        if (cb) G.add_factor(F_PHASE, 4, 0, f.a, Bits());
        if (ca) G.add_factor(F_PHASE, 4, 0, f.b, Bits());
        if (ca && cb) G.ph = (G.ph + 4) & 7;
        break;
      default: G.add_factor(f.kind, f.alpha + 4 * ca, f.beta + 4 * cb, f.a, f.b); break;
    }
  }
  for (int v = 0; v < G.n; ++v) {
    if (!G.alive[(size_t)v]) continue;
    int c = 0;
    apply_rules(G.P[(size_t)v], c);
    if (c) G.lam[(size_t)v] = (G.lam[(size_t)v] + 4) & 7;
  }

  // ---- chains: connected components over free outputs and residual spiders
  std::vector<int> free_out;
  std::vector<int> free_index((size_t)nout, -1);
  for (int i = 0; i < nout; ++i)
    if (pivot_row[(size_t)i] < 0) {
      free_index[(size_t)i] = (int)free_out.size();
      free_out.push_back(i);
    }
  const int nr = (int)free_out.size();
  std::vector<int> parent((size_t)(G.n + nout));
  std::iota(parent.begin(), parent.end(), 0);
  std::function<int(int)> find = [&](int x) { return parent[(size_t)x] == x ? x : parent[(size_t)x] = find(parent[(size_t)x]); };
  auto unite = [&](int a, int b) { parent[(size_t)find(a)] = find(b); };
  auto out_node = [&](int o) { return G.n + o; };
  for (int v = 0; v < G.n; ++v) {
    if (!G.alive[(size_t)v]) continue;
    for (int u : G.nbrs(v)) unite(v, u);
    G.P[(size_t)v].for_each([&](int p) { if (p >= E) unite(v, out_node(p - E)); });
  }
  for (const Factor& f : G.fac) {
    int first = -1;
    auto touch = [&](int p) {
      if (p < E) return;
      if (first < 0) first = out_node(p - E);
      else unite(first, out_node(p - E));
    };
    f.a.for_each(touch);
    f.b.for_each(touch);
  }
  std::map<int, int> comp_chain;
  std::vector<std::vector<int>> chain_outputs;
  for (int o : free_out) {
    int r = find(out_node(o));
    auto it = comp_chain.find(r);
    if (it == comp_chain.end()) {
      comp_chain[r] = (int)chain_outputs.size();
      chain_outputs.push_back({o});
    } else {
      chain_outputs[(size_t)it->second].push_back(o);
    }
  }
  const int nchains = (int)chain_outputs.size();

  // ---- 3: marginal diagrams per chain, decomposed into Clifford terms
  struct RawTable { std::vector<Term> terms; };
  std::vector<RawTable> rtabs;
  std::vector<Graph> marg;  // marginal diagrams, decomposed after all are built
  // Parities of the chain sub-diagrams before decomposition: every parity a
  // decomposition produces is a sum of these (rewriting only adds parameter
  // sets), so an f basis built from them does not depend on the cut order.
  std::vector<Bits> span_gens;
  std::vector<int> out_table((size_t)nout, -1), out_chain((size_t)nout, -1);
  for (int c = 0; c < nchains; ++c) {
    // sub-diagram of the chain; constant scalars and factors of other
    // components cancel in every ratio P_1 / P_prev and are dropped
    Graph Gc(np);
    std::vector<int> vmap((size_t)G.n, -1);
    int root = find(out_node(chain_outputs[(size_t)c][0]));
    for (int v = 0; v < G.n; ++v)
      if (G.alive[(size_t)v] && find(v) == root) {
        vmap[(size_t)v] = Gc.add_var(G.lam[(size_t)v]);
        Gc.ang[(size_t)vmap[(size_t)v]] = G.ang[(size_t)v];
        Gc.P[(size_t)vmap[(size_t)v]] = G.P[(size_t)v];
      }
    for (int v = 0; v < G.n; ++v) {
      if (vmap[(size_t)v] < 0) continue;
      for (int u : G.nbrs(v))
        if (u > v && vmap[(size_t)u] >= 0) Gc.toggle(vmap[(size_t)v], vmap[(size_t)u]);
    }
    for (const Factor& f : G.fac) {
      int hit = -1;
      auto look = [&](int p) { if (p >= E && hit < 0) hit = p - E; };
      f.a.for_each(look);
      f.b.for_each(look);
      if (hit >= 0 && find(out_node(hit)) == root) Gc.fac.push_back(f);
    }
    for (int v = 0; v < Gc.n; ++v) span_gens.push_back(Gc.P[(size_t)v]);
    for (const Factor& f : Gc.fac) {
      span_gens.push_back(f.a);
      span_gens.push_back(f.b);
    }
    const std::vector<int>& outs = chain_outputs[(size_t)c];
    for (int i = -1; i < (int)outs.size(); ++i) {
      Graph M = Gc;
      // trace outputs after i: each becomes a summation variable
      std::vector<int> zvar((size_t)nout, -1);
      for (size_t j = (size_t)(i + 1); j < outs.size(); ++j) zvar[(size_t)outs[j]] = M.add_var(0);
      for (int v = 0; v < Gc.n; ++v) {
        for (size_t j = (size_t)(i + 1); j < outs.size(); ++j) {
          size_t p = (size_t)(E + outs[j]);
          if (M.P[(size_t)v].get(p)) { M.P[(size_t)v].reset(p); M.toggle(v, zvar[(size_t)outs[j]]); }
        }
      }
      std::vector<Factor> keep;
      std::vector<Factor> redo;
      for (Factor& f : M.fac) {
        bool touches = false;
        auto chk = [&](int p) { if (p >= E && zvar[(size_t)(p - E)] >= 0) touches = true; };
        f.a.for_each(chk);
        f.b.for_each(chk);
        (touches ? redo : keep).push_back(f);
      }
      M.fac = keep;
      auto to_form = [&](const Bits& a) {
        Form F = form_const(np, 0);
        a.for_each([&](int p) {
          if (p >= E && zvar[(size_t)(p - E)] >= 0) F.vars.push_back(zvar[(size_t)(p - E)]);
          else F.params.set((size_t)p);
        });
        std::sort(F.vars.begin(), F.vars.end());
        return F;
      };
      for (const Factor& f : redo) {
        Form A = to_form(f.a), B = to_form(f.b);
        switch (f.kind) {
          case F_NODE: { int z = M.add_var(f.alpha); M.add_sign(form_var(np, z), A); break; }
          case F_PHASE: M.add_phase(f.alpha, A); break;
          case F_PHASE_F: M.add_phase_f(f.t, A); break;
          case F_PI_PAIR: M.add_sign(A, B); break;
          case F_PHASE_PAIR: {
            int x = M.add_var(f.alpha), y = M.add_var(f.beta);
            M.toggle(x, y);
            M.add_sign(form_var(np, x), A);
            M.add_sign(form_var(np, y), B);
            break;
          }
        }
      }
      if (i < 0) P.chain_norm.push_back((int)(rtabs.size() + marg.size()));
      else {
        out_table[(size_t)outs[(size_t)i]] = (int)(rtabs.size() + marg.size());
        out_chain[(size_t)outs[(size_t)i]] = c;
      }
      marg.push_back(std::move(M));
    }
  }
  // ---- 3b: decompose the marginals (independent of one another), on spare
  // host cores when there are any
  {
    std::vector<RawTable> done(marg.size());
    std::vector<uint64_t> totals(marg.size(), 0);
    std::atomic<uint64_t> shared_total{0};
    std::atomic<size_t> next{0};
    std::exception_ptr err;
    std::mutex err_mu;
    auto work = [&]() {
      for (;;) {
        const size_t k = next.fetch_add(1);
        if (k >= marg.size()) return;
        try {
          decompose_marginal(std::move(marg[k]), opts, budget, &totals[k], done[k].terms, &shared_total);
        } catch (...) {
          std::lock_guard<std::mutex> lk(err_mu);
          if (!err) err = std::current_exception();
          next.store(marg.size());
        }
      }
    };
    // the capture mode records into a thread-local list: no helpers then.
    // Helpers score cuts (LEARNED) on the caller's CUDA device.
    const int helpers = g_marginal_capture ? 0 : acquire_helpers((int)marg.size() - 1);
    int dev = -1;
    if (helpers && opts.decomp == TSIM_DECOMP_LEARNED && g_cut_scorer.load() && cudaGetDevice(&dev) != cudaSuccess)
      dev = -1;
    std::vector<std::thread> pool;
    pool.reserve((size_t)helpers);
    for (int h = 0; h < helpers; ++h) {
      try {
        pool.emplace_back([&work, dev]() {
          if (dev >= 0) cudaSetDevice(dev);
          work();
        });
      } catch (...) {
        break;  // no more threads to be had: the ones started and this one share the work
      }
    }
    work();
    for (std::thread& t : pool) t.join();
    release_helpers(helpers);
    if (err) std::rethrow_exception(err);
    for (size_t k = 0; k < marg.size(); ++k) {
      total_terms += totals[k];
      rtabs.push_back(std::move(done[k]));
    }
    if (opts.total_budget && total_terms > opts.total_budget)
      fail(TSIM_ERR_CHI_BUDGET, "stabilizer terms of the program exceed the budget (" +
                                    std::to_string(opts.total_budget) + ")");
  }

  if (g_marginal_capture) throw CaptureDone{};

  // ---- 4a: minimal f basis; table parities first so they occupy low X bits
  FBasis fb;
  auto epart = [&](const Bits& a) { return restrict_bits(a, 0, (size_t)E); };
  // parities repeat across terms: express each distinct one once (the
  // first-occurrence order, and so the f numbering, is unchanged)
  std::unordered_map<Bits, Bits, BitsHash> fm_cache;
  auto fmask_of = [&](const Bits& a) -> const Bits& {
    auto it = fm_cache.find(a);
    if (it != fm_cache.end()) return it->second;
    Bits fm = fb.express(epart(a));
    return fm_cache.emplace(a, std::move(fm)).first->second;
  };
  for (const Bits& g : span_gens) fmask_of(g);
  const int nft = (int)fb.orig.size();
  for (size_t t = 0; t < rtabs.size(); ++t)
    for (size_t k = 0; k < rtabs[t].terms.size(); ++k)
      for (const Factor& f : rtabs[t].terms[k].fac) {
        fmask_of(f.a);
        fmask_of(f.b);
      }
  if ((int)fb.orig.size() != nft) fail(TSIM_ERR_INTERNAL, "a decomposition left the span of its diagram's parities");
  std::vector<Bits> rule_f((size_t)nout);
  for (int i = 0; i < nout; ++i)
    if (pivot_row[(size_t)i] >= 0) {
      Bits r = rows[(size_t)pivot_row[(size_t)i]].v;
      r.reset((size_t)(E + i));
      rule_f[(size_t)i] = fb.express(epart(r));
    }
  const int nf = (int)fb.orig.size();
  P.nf = nf;
  P.nr = nr;
  P.nft = nft;
  P.nx = nf + nr;
  P.W = std::max(1, (P.nx + 63) / 64);
  const int W = P.W;
  auto fbit = [&](int k) { return k < nft ? k : k + nr; };
  auto xmask = [&](const Bits& fm, const Bits& full) {
    Bits x((size_t)W * 64);
    fm.for_each([&](int k) { x.flip((size_t)fbit(k)); });
    full.for_each([&](int p) {
      if (p >= E) {
        int fi = free_index[(size_t)(p - E)];
        if (fi < 0) fail(TSIM_ERR_INTERNAL, "deterministic output left in a parity");
        x.flip((size_t)(nft + fi));
      }
    });
    return to_words(x, W);
  };

  std::unordered_map<Bits, std::vector<uint64_t>, BitsHash> xm_cache;
  auto xmask_of = [&](const Bits& full) -> const std::vector<uint64_t>& {
    auto it = xm_cache.find(full);
    if (it != xm_cache.end()) return it->second;
    return xm_cache.emplace(full, xmask(fm_cache.at(full), full)).first->second;
  };

  // ---- tables
  P.tables.resize(rtabs.size());
  for (size_t t = 0; t < rtabs.size(); ++t) {
    for (size_t k = 0; k < rtabs[t].terms.size(); ++k) {
      const Term& tm = rtabs[t].terms[k];
      ProgTerm pt;
      pt.s0 = tm.s2;
      pt.j0 = tm.ph & 7;
      pt.fph = tm.fph;
      for (size_t q = 0; q < tm.fac.size(); ++q) {
        const Factor& f = tm.fac[q];
        ProgFactor pf;
        pf.kind = f.kind;
        pf.alpha = f.alpha & 7;
        pf.beta = f.beta & 7;
        pf.t = f.t;
        pf.u = xmask_of(f.a);
        pf.v = xmask_of(f.b);
        pt.f.push_back(std::move(pf));
      }
      P.tables[t].terms.push_back(std::move(pt));
    }
  }

  // ---- outputs in autoregressive order
  P.outputs.resize((size_t)nout);
  for (int i = 0; i < nout; ++i) {
    ProgOutput& o = P.outputs[(size_t)i];
    if (pivot_row[(size_t)i] >= 0) {
      const DeltaRow& r = rows[(size_t)pivot_row[(size_t)i]];
      Bits full = r.v;
      full.reset((size_t)(E + i));
      o.mask = xmask(rule_f[(size_t)i], full);
      o.cst = r.c;
    } else {
      o.random = true;
      o.xbit = nft + free_index[(size_t)i];
      o.chain = out_chain[(size_t)i];
      o.table = out_table[(size_t)i];
      o.mask.assign((size_t)W, 0);
    }
  }
  if (opts.mode == TSIM_MODE_MEASUREMENTS) {
    P.detmap = C.detectors;
    P.obsmap = C.observables;
  }

  // ---- 4b: columns of T and channel reduction
  std::vector<Bits> fcol((size_t)E, Bits((size_t)std::max(nf, 1)));
  for (int k = 0; k < nf; ++k) fb.orig[(size_t)k].for_each([&](int j) { fcol[(size_t)j].set((size_t)k); });
  auto xcol = [&](const Bits& fc) {
    Bits x((size_t)W * 64);
    fc.for_each([&](int k) { x.set((size_t)fbit(k)); });
    return to_words(x, W);
  };
  for (const RawChannel& rc : C.channels) {
    RawInfo ri;
    ri.nbits = rc.nbits;
    ri.probs = rc.probs;
    for (int b = 0; b < rc.nbits; ++b) ri.cols.push_back(xcol(fcol[(size_t)(rc.first_bit + b)]));
    P.raw.push_back(std::move(ri));
  }
  std::vector<RChan> chans;
  for (size_t ci = 0; ci < C.channels.size(); ++ci) {
    const RawChannel& rc = C.channels[ci];
    RChan ch;
    ch.p = rc.probs;
    ch.first_raw = (int)ci;
    for (int b = 0; b < rc.nbits; ++b) ch.cols.push_back(fcol[(size_t)(rc.first_bit + b)]);
    if (opts.channel_reduction) {
      // step 1: null-column elimination
      for (size_t b = ch.cols.size(); b-- > 0;)
        if (!ch.cols[b].any()) marginalize_bit(ch, b);
      if (ch.cols.empty()) continue;
      canonicalize(ch);  // step 2
    }
    chans.push_back(std::move(ch));
  }
  if (opts.channel_reduction) {
    // step 3: identical-channel merging by XOR convolution
    std::vector<RChan> merged;
    std::map<std::vector<Bits>, size_t, bool (*)(const std::vector<Bits>&, const std::vector<Bits>&)> index(
        [](const std::vector<Bits>& a, const std::vector<Bits>& b) {
          if (a.size() != b.size()) return a.size() < b.size();
          for (size_t i = 0; i < a.size(); ++i)
            if (a[i] != b[i]) return a[i] < b[i];
          return false;
        });
    for (RChan& ch : chans) {
      auto it = index.find(ch.cols);
      if (it == index.end()) {
        index[ch.cols] = merged.size();
        merged.push_back(std::move(ch));
      } else {
        xor_convolve(merged[it->second], ch.p);
      }
    }
    // step 4: subset absorption, larger signatures absorb smaller ones
    std::vector<size_t> order(merged.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
      return merged[a].cols.size() > merged[b].cols.size();
    });
    std::vector<char> gone(merged.size(), 0);
    for (size_t oi = 0; oi < order.size(); ++oi) {
      size_t big = order[oi];
      if (gone[big]) continue;
      for (size_t oj = oi + 1; oj < order.size(); ++oj) {
        size_t sm = order[oj];
        if (gone[sm] || merged[sm].cols.size() >= merged[big].cols.size()) continue;
        std::vector<int> pos;
        for (const Bits& c : merged[sm].cols) {
          int at = -1;
          for (size_t q = 0; q < merged[big].cols.size(); ++q)
            if (merged[big].cols[q] == c) at = (int)q;
          if (at < 0) break;
          pos.push_back(at);
        }
        if (pos.size() != merged[sm].cols.size()) continue;
        std::vector<double> emb(merged[big].p.size(), 0.0);
        for (size_t o = 0; o < merged[sm].p.size(); ++o) {
          size_t o2 = 0;
          for (size_t q = 0; q < pos.size(); ++q) o2 |= ((o >> q) & 1) << pos[q];
          emb[o2] += merged[sm].p[o];
        }
        xor_convolve(merged[big], emb);
        merged[big].first_raw = std::min(merged[big].first_raw, merged[sm].first_raw);
        gone[sm] = 1;
      }
    }
    chans.clear();
    for (size_t i = 0; i < merged.size(); ++i)
      if (!gone[i]) chans.push_back(std::move(merged[i]));
    std::stable_sort(chans.begin(), chans.end(), [](const RChan& a, const RChan& b) { return a.first_raw < b.first_raw; });
  }
  for (const RChan& ch : chans) {
    // outcomes -> signatures; identical signatures merged, zero signature first
    std::vector<Bits> sigs;
    std::vector<double> probs;
    for (size_t o = 0; o < ch.p.size(); ++o) {
      Bits s((size_t)std::max(nf, 1));
      for (size_t b = 0; b < ch.cols.size(); ++b)
        if ((o >> b) & 1) s ^= ch.cols[b];
      size_t at = sigs.size();
      for (size_t q = 0; q < sigs.size(); ++q)
        if (sigs[q] == s) at = q;
      if (at == sigs.size()) { sigs.push_back(s); probs.push_back(0.0); }
      probs[at] += ch.p[o];
    }
    ProgChannel pc;
    std::vector<size_t> keep;
    for (size_t q = 0; q < sigs.size(); ++q)
      if (q == 0 || probs[q] > 0) keep.push_back(q);
    if (!opts.channel_reduction) keep.resize(sigs.size()), std::iota(keep.begin(), keep.end(), 0);
    if (opts.channel_reduction && keep.size() == 1) continue;
    double cdf = 0;
    for (size_t q = 0; q < keep.size(); ++q) {
      pc.sig.push_back(xcol(sigs[keep[q]]));
      pc.probs.push_back(probs[keep[q]]);
      if (q + 1 < keep.size()) {
        cdf += probs[keep[q]];
        double t = std::floor(cdf * 4294967296.0);
        if (t > 4294967295.0) t = 4294967295.0;
        if (t < 0) t = 0;
        pc.thr.push_back((uint32_t)t);
      }
    }
    P.channels.push_back(std::move(pc));
  }
  set_noise_sampling(P, -1);
  prepare_device_tables(P);
  return prog.release();
}

namespace {

// Groups for the geometric-gap noise rule.  Channels that can fire are sorted
// by their probability of firing f (2^32 - thr[0], in units of 2^-32),
// largest first, and cut into consecutive runs; a run's leader (its most
// likely channel) gives Q, so every member's outcome-0 threshold is >= Q and
// the rule is exact for any cut.  A run of n channels led by f costs about
// 1 + 2 n f random words per shot (a gap word, and per candidate its word and
// the next gap word); the cuts minimise the total by dynamic programming over
// the sorted list (O(channels^2)).  Members keep program order.  Channels
// that cannot fire (one outcome) join no group.
std::vector<NoiseGroup> noise_groups(const Program& p) {
  std::vector<int> order;
  for (size_t c = 0; c < p.channels.size(); ++c)
    if (!p.channels[c].thr.empty()) order.push_back((int)c);
  auto fire = [&](int c) { return (uint64_t(1) << 32) - p.channels[(size_t)c].thr[0]; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return fire(a) > fire(b); });
  const size_t n = order.size();
  // best[j]: fewest expected words for the first j channels; cut[j]: where
  // the last run of that optimum starts
  std::vector<double> best(n + 1, 0.0);
  std::vector<size_t> cut(n + 1, 0);
  for (size_t j = 1; j <= n; ++j) {
    best[j] = 1e300;
    for (size_t i = 0; i < j; ++i) {
      const double f = (double)fire(order[i]) / 4294967296.0;
      const double c = best[i] + 1.0 + 2.0 * (double)(j - i) * f;
      if (c < best[j]) {
        best[j] = c;
        cut[j] = i;
      }
    }
  }
  std::vector<NoiseGroup> out;
  for (size_t j = n; j > 0; j = cut[j]) {
    NoiseGroup g;
    g.Q = p.channels[(size_t)order[cut[j]]].thr[0];
    for (size_t k = cut[j]; k < j; ++k) g.member.push_back(order[k]);
    std::sort(g.member.begin(), g.member.end());
    out.push_back(std::move(g));
  }
  std::reverse(out.begin(), out.end());
  return out;
}

double geometric_words(const std::vector<NoiseGroup>& gs) {
  // per group one gap word, and per candidate its word and the next gap word
  double w = 0;
  for (const NoiseGroup& g : gs) w += 1.0 + 2.0 * (double)g.member.size() * (4294967296.0 - g.Q) / 4294967296.0;
  return w;
}

}  // namespace

void noise_word_estimate(const Program& p, double out[2]) {
  double pc = 0;
  for (const ProgChannel& c : p.channels) pc += c.thr.empty() ? 0.0 : 1.0;
  out[0] = pc;
  out[1] = geometric_words(noise_groups(p));
}

void set_noise_sampling(Program& p, int mode) {
  if (mode < -1 || mode > 1) fail(TSIM_ERR_ARG, "noise sampling mode must be -1, 0 or 1");
  std::vector<NoiseGroup> gs = noise_groups(p);
  if (mode < 0) {
    double est[2];
    noise_word_estimate(p, est);
    // a geometric word costs about twice a per-channel word (the gap search
    // and the serial dependence between words)
    mode = (!gs.empty() && 2.0 * est[1] < est[0]) ? 1 : 0;
  }
  p.noise_mode = mode;
  p.groups = mode ? std::move(gs) : std::vector<NoiseGroup>();
}

bool ProgTable::is_float() const {
  for (const ProgTerm& tm : terms) {
    if (tm.fph != 0.0) return true;
    for (const ProgFactor& f : tm.f)
      if (f.kind == F_PHASE_F) return true;
  }
  return false;
}

std::complex<double> eval_table_host_c(const Program& p, int t, const uint64_t* x) {
  if (t < 0 || t >= (int)p.tables.size()) fail(TSIM_ERR_ARG, "table index out of range");
  auto par = [&](const std::vector<uint64_t>& m) {
    uint64_t acc = 0;
    for (size_t w = 0; w < m.size(); ++w) acc ^= m[w] & x[w];
    return __builtin_parityll(acc);
  };
  std::complex<double> sum = 0.0;
  for (const ProgTerm& tm : p.tables[(size_t)t].terms) {
    ZW c = ZW::omega(tm.j0);
    c.k = tm.s0;
    std::complex<double> v = zw_to_complex(c) * std::polar(1.0, M_PI * tm.fph);
    for (const ProgFactor& f : tm.f) {
      Factor fc;
      fc.kind = f.kind;
      fc.alpha = f.alpha;
      fc.beta = f.beta;
      fc.t = f.t;
      v *= factor_value_c(fc, par(f.u), par(f.v));
    }
    sum += v;
  }
  return sum;
}

ZW eval_table_host(const Program& p, int t, const uint64_t* x) {
  if (t < 0 || t >= (int)p.tables.size()) fail(TSIM_ERR_ARG, "table index out of range");
  if (p.tables[(size_t)t].is_float()) fail(TSIM_ERR_ARG, "table has arbitrary phases: use the floating-point evaluation");
  auto par = [&](const std::vector<uint64_t>& m) {
    uint64_t acc = 0;
    for (size_t w = 0; w < m.size(); ++w) acc ^= m[w] & x[w];
    return __builtin_parityll(acc);
  };
  ZW sum;
  for (const ProgTerm& tm : p.tables[(size_t)t].terms) {
    ZW v = ZW::omega(tm.j0);
    v.k = tm.s0;
    for (const ProgFactor& f : tm.f) {
      Factor fc;
      fc.kind = f.kind;
      fc.alpha = f.alpha;
      fc.beta = f.beta;
      v = zw_mul(v, factor_value(fc, par(f.u), par(f.v)));
      if (v.zero()) break;
    }
    sum = zw_add(sum, v);
  }
  return sum;
}

std::vector<Graph> marginal_diagrams(const std::string& text, int mode) {
  std::vector<Graph> out;
  tsim_compile_opts opts{};
  opts.mode = mode;
  opts.decomp = TSIM_DECOMP_HEURISTIC;
  opts.channel_reduction = 1;
  g_marginal_capture = &out;
  try {
    delete compile_program(text, opts);
  } catch (const CaptureDone&) {
  } catch (...) {
    g_marginal_capture = nullptr;
    throw;
  }
  g_marginal_capture = nullptr;
  return out;
}

}  // namespace tsim
