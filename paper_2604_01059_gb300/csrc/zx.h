// Parameterised graph-like ZX diagram, stored as a sum over binary spider
// variables (a "path sum"):
//
//   value(p) = sqrt2^s2 * w^ph * prod_k factor_k(p)
//              * sum_{z in {0,1}^V} prod_v w^(lam_v z_v) (-1)^(z_v <P_v, p>)
//                                   prod_{(u,v) in E} (-1)^(z_u z_v)
//
// Every vertex is a Z spider with phase lam_v * pi/4 + pi * (parity of the
// parameters in P_v) (Appendix "ZX-Calculus": parameterised Pauli phases a*pi);
// every edge is a Hadamard edge.  Parameters are the raw error bits e and the
// output bits of the diagram.  The scalar factors are the parameter-dependent
// phase terms of Table "Types of parameterized phase terms" (Appendix
// "Parameterized evaluation of Clifford ZX diagrams").
//
// Clifford rewriting (local complementation, pivoting, fusion, removal of
// isolated spiders) is implemented as exact elimination of one summation
// variable at a time; stabilizer decomposition (Appendix "Stabilizer
// decompositions") as splitting a sum into Clifford branches.
#pragma once
#include <atomic>
#include <complex>
#include <vector>

#include "common.h"

namespace tsim {

// Factor kinds, values with angles in units of pi/4 and w = e^{i pi/4}:
enum FactorKind {
  F_PHASE_PAIR = 0,  // 1 + w^(al+4a) + w^(be+4b) - w^(al+be+4a+4b)     Eq. phase_pair
  F_NODE = 1,        // 1 + w^(al+4a)                                    "Node"
  F_PHASE = 2,       // w^(al*a)  (al = +-2: "Half-pi"; al = 4: a sign)
  F_PI_PAIR = 3,     // (-1)^(a b)                                       "pi-pair"
  F_PHASE_F = 4      // e^(i pi t a) for an arbitrary angle t (rotation gates)
};

struct Factor {
  int kind = 0;
  int alpha = 0, beta = 0;
  double t = 0;  // F_PHASE_F: the angle, in units of pi
  Bits a, b;     // parities over the diagram's parameters
};

// Angles of arbitrary rotations, in units of pi, reduced to [0, 2); an angle
// within kAngleTol of a multiple of 1/4 is that multiple (it joins the exact
// phases in units of pi/4).
constexpr double kAngleTol = 1e-12;
double angle_mod2(double t);
// k in 0..7 when t is k/4 (mod 2) within kAngleTol, else -1
int angle_eighths(double t);

// Affine GF(2) form: XOR of variables, parameters and a constant bit.
struct Form {
  std::vector<int> vars;  // sorted, unique
  Bits params;
  int c = 0;
};

Form form_const(size_t np, int c);
Form form_var(size_t np, int v);
Form form_param(size_t np, int p);
Form form_params(const Bits& ps);
void form_xor(Form& a, const Form& b);

struct Term {
  int s2 = 0, ph = 0;
  double fph = 0;  // a further constant phase e^(i pi fph) from arbitrary rotations
  std::vector<Factor> fac;
  bool is_float() const;
};

struct Graph {
  size_t np = 0;
  int n = 0, cap = 0;
  std::vector<int> lam;
  std::vector<double> ang;  // arbitrary part of each spider's phase: e^(i pi ang z), 0 for Clifford+T
  double fph = 0;           // constant phase e^(i pi fph)
  std::vector<Bits> P;
  std::vector<std::vector<uint64_t>> adj;
  std::vector<char> alive;
  std::vector<int> uid;  // stable vertex id through copies and compaction (-1: created later)
  int s2 = 0, ph = 0;
  bool zero = false;
  std::vector<Factor> fac;

  explicit Graph(size_t nparams = 0) : np(nparams) {}

  int add_var(int l = 0);
  void kill(int v);
  bool edge(int u, int v) const { return (adj[(size_t)u][(size_t)v >> 6] >> (v & 63)) & 1; }
  void toggle(int u, int v);
  std::vector<int> nbrs(int v) const;
  int degree(int v) const;
  int num_alive() const;

  // multiply the diagram by w^(theta * L)
  void add_phase(int theta, Form L);
  // multiply the diagram by e^(i pi t L) for an arbitrary angle t
  void add_phase_f(double t, Form L);
  // the spider is not Clifford: odd phase or an arbitrary angle
  bool non_clifford(int v) const { return (lam[(size_t)v] & 1) || ang[(size_t)v] != 0.0; }
  // multiply by (-1)^(F * G)
  void add_sign(const Form& F, const Form& G);
  void add_factor(int kind, int alpha, int beta, const Bits& a, const Bits& b);
  // multiply by e^(i pi t a) (a multiple of pi/4 becomes an exact factor)
  void add_factor_f(double t, const Bits& a);
  // set a spider's arbitrary angle (a multiple of pi/4 joins lam)
  void set_angle(int v, double t);
  // multiply by delta(L = 0), as (1/2) sum_w (-1)^(w L)
  void hub(const Form& L);
  bool can_substitute(int y, const Form& L) const;
  // replace variable y by the affine form L (valid only if can_substitute)
  void substitute(int y, const Form& L);

  // rewrite steps
  void remove_isolated(int v);
  void lcomp(int v);
  void eliminate(int v, int u);
  void simplify();
  void compact();
  void fold_phase_factors();
  Term as_term() const;
};

// value of one factor for parity values a, b (exact kinds only)
ZW factor_value(const Factor& f, int a, int b);
// value of any factor, in complex double
std::complex<double> factor_value_c(const Factor& f, int a, int b);
std::complex<double> zw_to_complex(const ZW& z);

struct DecompStats {
  uint64_t terms = 0;
  uint64_t budget = 0;         // per decomposition
  uint64_t leaves = 0;
  uint64_t nodes = 0;          // branches explored
  uint64_t* total = nullptr;   // running count over all decompositions of a program
  uint64_t total_budget = 0;
  // the same count shared by marginals decomposed on several threads (the
  // program-wide budget then stops every thread early)
  std::atomic<uint64_t>* shared_total = nullptr;
};

// Decompose into Clifford terms (Appendix "Stabilizer decompositions").
// policy: 0 = the heuristic: odd spiders in ascending id; the first two are
// split as a BSS pair (2 terms) while some two consecutive ones have phases
// that cancel (lam sum = 0 mod 8), otherwise Cat5 takes the first five (3
// terms, one odd spider left per term); pairs for two to four, a single cut
// for the last; 4 = Cat5 on the first five whenever five remain; 3 = pairs
// only; 2 = single cuts; 1 = as 0 with the spiders in ascending
// `scores[uid]` (a learned cut order; spiders without a score go last).
// `first` >= 0 forces the spider with that uid into the first cut.  Every
// order and policy gives the same sum.
void decompose(Graph g, int policy, std::vector<Term>& out, DecompStats& st,
               const std::vector<double>* scores = nullptr, int first = -1);

// Units of a cut order: the non-Clifford spiders in ascending id, two
// consecutive ones whose phases cancel (a T gate's ket and bra copies) forming
// one pair unit, every other spider a unit of its own.  The heuristic splits
// the pair units in id order; a cut order that keeps them together only
// reorders units.
std::vector<std::vector<int>> cut_units(const Graph& g);
// Scores for decompose(policy 1) that put the units in the given order
// (members of one unit in ascending id); spiders in no listed unit go last.
std::vector<double> unit_order_scores(const Graph& g, const std::vector<std::vector<int>>& units,
                                      const std::vector<int>& order);

// Node features of the alive spiders for the cut-order network, row-major
// [nodes][kCutFeatures], with the adjacency in CSR form and each node's uid.
constexpr int kCutFeatures = 14;
void cut_features(const Graph& g, std::vector<float>& X, std::vector<int>& rowptr,
                  std::vector<int>& col, std::vector<int>& uids);

// A seeded random Clifford+T ZX diagram: t non-Clifford spiders and c
// Clifford spiders, each joined by Hadamard edges to three random others.
Graph random_zx_diagram(uint64_t seed, int t, int c);

// Brute-force value of a small graph for one parameter assignment (tests).
ZW brute_value(const Graph& g, const Bits& pv);
ZW term_value(const Term& t, const Bits& pv);
// the same in complex double, for graphs with arbitrary angles
std::complex<double> brute_value_c(const Graph& g, const Bits& pv);
std::complex<double> term_value_c(const Term& t, const Bits& pv);

}  // namespace tsim
