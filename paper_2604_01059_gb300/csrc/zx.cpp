// Rewrite rules of the parameterised graph-like diagram (see zx.h).
//
// Each rule removes summation variables exactly:
//   * isolated spider v:      sum_z w^(lam z)(-1)^(z a) = 1 + w^(lam + 4a)      -> Node factor
//   * local complementation:  lam_v = +-pi/2:  1 + (+-i)(-1)^K = sqrt2 w^(+-1) w^(-+2K),
//                             K = P_v + sum_{N(v)} z  (Eq. local_comp)
//   * pivot / fusion:         lam_v in {0, pi}: sum_{z_v} (-1)^(z_v (c + P_v + sum_N z)) =
//                             2 delta(...), solved for one neighbour u and substituted
//                             (Eq. pivoting when u is also a Pauli spider)
// Parameter-dependent phases produced on the way are kept as factors (Table
// "Types of parameterized phase terms").  The pi-commutation rule is never
// applied to non-Clifford spiders (Appendix "ZX-Calculus"): an odd-phase
// variable is only ever replaced by a single variable (fusion) or by a
// parameter parity.
#include "zx.h"

#include <algorithm>
#include <cmath>

namespace tsim {

double angle_mod2(double t) {
  t = std::fmod(t, 2.0);
  if (t < 0) t += 2.0;
  if (t >= 2.0 - kAngleTol) t = 0.0;
  return t;
}

int angle_eighths(double t) {
  const double q = angle_mod2(t) * 4.0;
  const double r = std::nearbyint(q);
  if (std::fabs(q - r) > 4.0 * kAngleTol) return -1;
  return ((int)r) & 7;
}

bool Term::is_float() const {
  if (fph != 0.0) return true;
  for (const Factor& f : fac)
    if (f.kind == F_PHASE_F) return true;
  return false;
}

Form form_const(size_t np, int c) {
  Form f;
  f.params = Bits(np);
  f.c = c & 1;
  return f;
}
Form form_var(size_t np, int v) {
  Form f = form_const(np, 0);
  f.vars.push_back(v);
  return f;
}
Form form_param(size_t np, int p) {
  Form f = form_const(np, 0);
  f.params.set((size_t)p);
  return f;
}
Form form_params(const Bits& ps) {
  Form f;
  f.params = ps;
  return f;
}
void form_xor(Form& a, const Form& b) {
  std::vector<int> out;
  out.reserve(a.vars.size() + b.vars.size());
  size_t i = 0, j = 0;
  while (i < a.vars.size() || j < b.vars.size()) {
    if (j >= b.vars.size() || (i < a.vars.size() && a.vars[i] < b.vars[j])) out.push_back(a.vars[i++]);
    else if (i >= a.vars.size() || b.vars[j] < a.vars[i]) out.push_back(b.vars[j++]);
    else { ++i; ++j; }
  }
  a.vars.swap(out);
  a.params ^= b.params;
  a.c ^= b.c;
}

int Graph::add_var(int l) {
  if (n == cap) {
    int nc = cap ? cap * 2 : 64;
    size_t words = (size_t)(nc + 63) / 64;
    for (auto& row : adj) row.resize(words, 0);
    adj.resize((size_t)nc, std::vector<uint64_t>(words, 0));
    cap = nc;
  }
  lam.push_back(l & 7);
  ang.push_back(0.0);
  P.push_back(Bits(np));
  alive.push_back(1);
  uid.push_back(-1);
  return n++;
}

void Graph::kill(int v) {
  for (int u : nbrs(v)) adj[(size_t)u][(size_t)v >> 6] &= ~(1ull << (v & 63));
  std::fill(adj[(size_t)v].begin(), adj[(size_t)v].end(), 0ull);
  alive[(size_t)v] = 0;
}

void Graph::toggle(int u, int v) {
  if (u == v) {
    lam[(size_t)u] = (lam[(size_t)u] + 4) & 7;
    return;
  }
  adj[(size_t)u][(size_t)v >> 6] ^= 1ull << (v & 63);
  adj[(size_t)v][(size_t)u >> 6] ^= 1ull << (u & 63);
}

std::vector<int> Graph::nbrs(int v) const {
  std::vector<int> out;
  const auto& row = adj[(size_t)v];
  for (size_t i = 0; i < row.size(); ++i) {
    uint64_t x = row[i];
    while (x) {
      out.push_back((int)(i * 64 + (size_t)__builtin_ctzll(x)));
      x &= x - 1;
    }
  }
  return out;
}

int Graph::degree(int v) const {
  int d = 0;
  for (uint64_t x : adj[(size_t)v]) d += __builtin_popcountll(x);
  return d;
}

int Graph::num_alive() const {
  int c = 0;
  for (char a : alive) c += a ? 1 : 0;
  return c;
}

void Graph::add_factor(int kind, int alpha, int beta, const Bits& a, const Bits& b) {
  alpha &= 7;
  beta &= 7;
  switch (kind) {
    case F_PHASE:
      if (!alpha || !a.any()) return;
      break;
    case F_PHASE_F:
      fail(TSIM_ERR_INTERNAL, "arbitrary phase factors are added by add_factor_f");
    case F_NODE:
      if (!a.any()) {
        switch (alpha) {  // 1 + w^alpha
          case 0: s2 += 2; return;
          case 4: zero = true; return;
          case 2: s2 += 1; ph = (ph + 1) & 7; return;
          case 6: s2 += 1; ph = (ph + 7) & 7; return;
          default: fail(TSIM_ERR_INTERNAL, "constant non-Clifford node factor");
        }
      }
      break;
    case F_PI_PAIR:
      if (!a.any() || !b.any()) return;
      if (a == b) {  // (-1)^(a a) = (-1)^a
        add_factor(F_PHASE, 4, 0, a, Bits());
        return;
      }
      break;
    default:
      fail(TSIM_ERR_INTERNAL, "factor kind not produced by the rewriter");
  }
  Factor f;
  f.kind = kind;
  f.alpha = alpha;
  f.beta = beta;
  f.a = a;
  f.b = (kind == F_PI_PAIR || kind == F_PHASE_PAIR) ? b : Bits(np);
  if (f.b.nwords() < f.a.nwords()) f.b.w.resize(f.a.nwords(), 0);
  fac.push_back(std::move(f));
}

void Graph::add_factor_f(double t, const Bits& a) {
  t = angle_mod2(t);
  const int k = angle_eighths(t);
  if (k >= 0) {
    add_factor(F_PHASE, k, 0, a, Bits());
    return;
  }
  if (!a.any()) return;
  Factor f;
  f.kind = F_PHASE_F;
  f.t = t;
  f.a = a;
  f.b = Bits(np);
  if (f.b.nwords() < f.a.nwords()) f.b.w.resize(f.a.nwords(), 0);
  fac.push_back(std::move(f));
}

void Graph::set_angle(int v, double t) {
  t = angle_mod2(t);
  const int k = angle_eighths(t);
  if (k >= 0) {
    lam[(size_t)v] = (lam[(size_t)v] + k) & 7;
    ang[(size_t)v] = 0.0;
  } else {
    ang[(size_t)v] = t;
  }
}

void Graph::add_phase_f(double t, Form L) {
  t = angle_mod2(t);
  const int k = angle_eighths(t);
  if (k >= 0) {  // a multiple of pi/4: exact
    add_phase(k, L);
    return;
  }
  if (L.c) {  // e^(i pi t (1 + g)) = e^(i pi t) e^(-i pi t g)
    fph = angle_mod2(fph + t);
    t = angle_mod2(-t);
    L.c = 0;
  }
  if (L.vars.empty()) {
    if (L.params.any()) add_factor_f(t, L.params);
    return;
  }
  if (L.vars.size() == 1 && !L.params.any()) {
    set_angle(L.vars[0], ang[(size_t)L.vars[0]] + t);
    return;
  }
  // phase gadget: new variable y = L, carrying the angle
  int y = add_var(0);
  Form h = L;
  form_xor(h, form_var(np, y));
  hub(h);
  ang[(size_t)y] = t;
}

void Graph::add_phase(int theta, Form L) {
  theta &= 7;
  if (!theta) return;
  if (L.c) {  // w^(theta (1 + g)) = w^theta w^(-theta g)
    ph = (ph + theta) & 7;
    theta = (8 - theta) & 7;
    L.c = 0;
  }
  if (L.vars.empty()) {
    if (L.params.any()) add_factor(F_PHASE, theta, 0, L.params, Bits());
    return;
  }
  if ((theta & 1) == 0) {
    // i^(t XOR b) = prod i^(t b_k) prod_{k<l} (-1)^(t b_k b_l)
    bool odd_t = (theta == 2 || theta == 6);
    for (int v : L.vars) lam[(size_t)v] = (lam[(size_t)v] + theta) & 7;
    if (odd_t)
      for (size_t i = 0; i < L.vars.size(); ++i)
        for (size_t j = i + 1; j < L.vars.size(); ++j) toggle(L.vars[i], L.vars[j]);
    if (L.params.any()) {
      add_factor(F_PHASE, theta, 0, L.params, Bits());
      if (odd_t)
        for (int v : L.vars) P[(size_t)v] ^= L.params;
    }
    return;
  }
  if (L.vars.size() == 1 && !L.params.any()) {
    lam[(size_t)L.vars[0]] = (lam[(size_t)L.vars[0]] + theta) & 7;
    return;
  }
  // phase gadget: new variable y = L, carrying the odd phase
  int y = add_var(0);
  Form h = L;
  form_xor(h, form_var(np, y));
  hub(h);
  lam[(size_t)y] = theta;
}

void Graph::add_sign(const Form& F, const Form& G) {
  for (int x : F.vars)
    for (int y : G.vars) toggle(x, y);
  if (G.params.any())
    for (int x : F.vars) P[(size_t)x] ^= G.params;
  if (G.c)
    for (int x : F.vars) lam[(size_t)x] = (lam[(size_t)x] + 4) & 7;
  if (F.params.any())
    for (int y : G.vars) P[(size_t)y] ^= F.params;
  if (F.c)
    for (int y : G.vars) lam[(size_t)y] = (lam[(size_t)y] + 4) & 7;
  if (F.params.any() && G.params.any()) add_factor(F_PI_PAIR, 0, 0, F.params, G.params);
  if (G.c && F.params.any()) add_factor(F_PHASE, 4, 0, F.params, Bits());
  if (F.c && G.params.any()) add_factor(F_PHASE, 4, 0, G.params, Bits());
  if (F.c && G.c) ph = (ph + 4) & 7;
}

void Graph::hub(const Form& L) {
  int w = add_var(0);
  add_sign(form_var(np, w), L);
  s2 -= 2;
}

bool Graph::can_substitute(int y, const Form& L) const {
  if (std::binary_search(L.vars.begin(), L.vars.end(), y)) return false;
  if (!non_clifford(y)) return true;
  return L.vars.empty() || (L.vars.size() == 1 && !L.params.any());
}

void Graph::substitute(int y, const Form& L) {
  if (!can_substitute(y, L)) fail(TSIM_ERR_INTERNAL, "invalid substitution");
  int th = lam[(size_t)y];
  const double ty = ang[(size_t)y];
  Bits py = P[(size_t)y];
  std::vector<int> nb = nbrs(y);
  kill(y);
  add_phase(th, L);
  if (ty != 0.0) add_phase_f(ty, L);
  if (py.any()) add_sign(form_params(py), L);
  for (int t : nb) add_sign(form_var(np, t), L);
}

void Graph::remove_isolated(int v) {
  int l = lam[(size_t)v];
  Bits a = P[(size_t)v];
  kill(v);
  add_factor(F_NODE, l, 0, a, Bits());
}

void Graph::lcomp(int v) {
  int l = lam[(size_t)v];
  int s = (l == 2) ? 1 : -1;
  Form K = form_params(P[(size_t)v]);
  K.vars = nbrs(v);
  kill(v);
  s2 += 1;
  ph = (ph + s + 8) & 7;
  add_phase(-2 * s, K);
}

void Graph::eliminate(int v, int u) {
  Form L = form_params(P[(size_t)v]);
  L.c = lam[(size_t)v] >> 2;
  for (int t : nbrs(v))
    if (t != u) L.vars.push_back(t);
  kill(v);
  s2 += 2;
  substitute(u, L);
}

void Graph::simplify() {
  bool changed = true;
  while (changed && !zero) {
    changed = false;
    for (int v = 0; v < n; ++v) {
      if (!alive[(size_t)v] || ang[(size_t)v] != 0.0) continue;
      int l = lam[(size_t)v];
      if (l == 2 || l == 6) {
        lcomp(v);
        changed = true;
        continue;
      }
      if (l != 0 && l != 4) continue;
      std::vector<int> nb = nbrs(v);
      if (nb.empty()) {
        remove_isolated(v);
        changed = true;
        continue;
      }
      int best = -1, cliff = -1;
      for (int u : nb) {
        if (ang[(size_t)u] != 0.0) continue;
        int lu = lam[(size_t)u];
        if (lu == 0 || lu == 4) { best = u; break; }
        if ((lu == 2 || lu == 6) && cliff < 0) cliff = u;
      }
      if (best < 0) best = cliff;
      if (best < 0 && (nb.size() == 1 || (nb.size() == 2 && !P[(size_t)v].any()))) best = nb[0];
      if (best >= 0) {
        eliminate(v, best);
        changed = true;
      }
    }
  }
}

void Graph::compact() {
  std::vector<int> map((size_t)n, -1);
  int m = 0;
  for (int v = 0; v < n; ++v)
    if (alive[(size_t)v]) map[(size_t)v] = m++;
  Graph h(np);
  for (int v = 0; v < n; ++v)
    if (alive[(size_t)v]) {
      int nv = h.add_var(lam[(size_t)v]);
      h.ang[(size_t)nv] = ang[(size_t)v];
      h.P[(size_t)nv] = P[(size_t)v];
      h.uid[(size_t)nv] = uid[(size_t)v];
    }
  for (int v = 0; v < n; ++v) {
    if (!alive[(size_t)v]) continue;
    for (int u : nbrs(v))
      if (u > v) h.toggle(map[(size_t)v], map[(size_t)u]);
  }
  h.s2 = s2;
  h.ph = ph;
  h.fph = fph;
  h.zero = zero;
  h.fac = std::move(fac);
  *this = std::move(h);
}

void Graph::fold_phase_factors() {
  // merge w^(al1 a) w^(al2 a) into one factor per parity, and the arbitrary
  // phases e^(i pi t1 a) e^(i pi t2 a) likewise (an arbitrary sum that
  // reaches a multiple of pi/4 joins the exact factor); drop trivial ones
  std::vector<Factor> out;
  for (int pass = 0; pass < 2; ++pass) {
    out.clear();
    for (auto& f : fac) {
      if (f.kind == F_PHASE || f.kind == F_PHASE_F) {
        bool merged = false;
        for (auto& g : out)
          if (g.kind == f.kind && g.a == f.a) {
            if (f.kind == F_PHASE) g.alpha = (g.alpha + f.alpha) & 7;
            else g.t = angle_mod2(g.t + f.t);
            merged = true;
            break;
          }
        if (!merged) out.push_back(f);
      } else {
        out.push_back(f);
      }
    }
    fac.clear();
    for (auto& f : out) {
      if (f.kind == F_PHASE_F) {
        const int k = angle_eighths(f.t);
        if (k >= 0) {
          f.kind = F_PHASE;
          f.alpha = k;
          f.t = 0;
        }
      }
      if (!(f.kind == F_PHASE && f.alpha == 0)) fac.push_back(std::move(f));
    }
  }
}

Term Graph::as_term() const {
  Term t;
  t.s2 = s2;
  t.ph = ph;
  t.fph = fph;
  t.fac = fac;
  return t;
}

ZW factor_value(const Factor& f, int a, int b) {
  ZW one = ZW::omega(0);
  switch (f.kind) {
    case F_PHASE_PAIR: {
      ZW r = zw_add(one, ZW::omega(f.alpha + 4 * a));
      r = zw_add(r, ZW::omega(f.beta + 4 * b));
      return zw_add(r, ZW::omega(f.alpha + f.beta + 4 * a + 4 * b + 4));
    }
    case F_NODE: return zw_add(one, ZW::omega(f.alpha + 4 * a));
    case F_PHASE: return ZW::omega(f.alpha * a);
    case F_PI_PAIR: return ZW::omega(4 * (a & b));
  }
  fail(TSIM_ERR_INTERNAL, "bad factor kind");
}

std::complex<double> zw_to_complex(const ZW& z) {
  const double r = std::sqrt(0.5);
  std::complex<double> v((double)z.c[0] + r * ((double)z.c[1] - (double)z.c[3]),
                         r * ((double)z.c[1] + (double)z.c[3]) + (double)z.c[2]);
  return v * std::pow(std::sqrt(2.0), z.k);
}

std::complex<double> factor_value_c(const Factor& f, int a, int b) {
  if (f.kind == F_PHASE_F) return a ? std::polar(1.0, M_PI * f.t) : std::complex<double>(1.0, 0.0);
  return zw_to_complex(factor_value(f, a, b));
}

static ZW scalar_value(int s2, int ph, const std::vector<Factor>& fac, const Bits& pv) {
  ZW v = ZW::omega(ph);
  v.k = s2;
  for (const Factor& f : fac) {
    v = zw_mul(v, factor_value(f, f.a.dot(pv), f.b.dot(pv)));
    if (v.zero()) break;
  }
  return v;
}

ZW term_value(const Term& t, const Bits& pv) {
  if (t.is_float()) fail(TSIM_ERR_INTERNAL, "exact value of a term with an arbitrary phase");
  return scalar_value(t.s2, t.ph, t.fac, pv);
}

static std::complex<double> scalar_value_c(int s2, int ph, double fph, const std::vector<Factor>& fac,
                                           const Bits& pv) {
  ZW c = ZW::omega(ph);
  c.k = s2;
  std::complex<double> v = zw_to_complex(c) * std::polar(1.0, M_PI * fph);
  for (const Factor& f : fac) v *= factor_value_c(f, f.a.dot(pv), f.b.dot(pv));
  return v;
}

std::complex<double> term_value_c(const Term& t, const Bits& pv) { return scalar_value_c(t.s2, t.ph, t.fph, t.fac, pv); }

std::complex<double> brute_value_c(const Graph& g, const Bits& pv) {
  if (g.zero) return 0.0;
  std::vector<int> vs;
  for (int v = 0; v < g.n; ++v)
    if (g.alive[(size_t)v]) vs.push_back(v);
  if (vs.size() > 20) fail(TSIM_ERR_INTERNAL, "brute force on a large graph");
  std::complex<double> sum = 0.0;
  for (uint64_t z = 0; z < (1ull << vs.size()); ++z) {
    int phase = 0;
    double fl = 0.0;
    for (size_t i = 0; i < vs.size(); ++i) {
      if (!((z >> i) & 1)) continue;
      int v = vs[i];
      phase += g.lam[(size_t)v] + 4 * g.P[(size_t)v].dot(pv);
      fl += g.ang[(size_t)v];
      for (size_t j = i + 1; j < vs.size(); ++j)
        if (((z >> j) & 1) && g.edge(v, vs[j])) phase += 4;
    }
    sum += std::polar(1.0, M_PI * (phase / 4.0 + fl));
  }
  return sum * scalar_value_c(g.s2, g.ph, g.fph, g.fac, pv);
}

ZW brute_value(const Graph& g, const Bits& pv) {
  if (g.zero) return ZW();
  std::vector<int> vs;
  for (int v = 0; v < g.n; ++v)
    if (g.alive[(size_t)v]) vs.push_back(v);
  if (vs.size() > 20) fail(TSIM_ERR_INTERNAL, "brute force on a large graph");
  ZW sum;
  for (uint64_t z = 0; z < (1ull << vs.size()); ++z) {
    int phase = 0;
    for (size_t i = 0; i < vs.size(); ++i) {
      if (!((z >> i) & 1)) continue;
      int v = vs[i];
      phase += g.lam[(size_t)v] + 4 * g.P[(size_t)v].dot(pv);
      for (size_t j = i + 1; j < vs.size(); ++j)
        if (((z >> j) & 1) && g.edge(v, vs[j])) phase += 4;
    }
    sum = zw_add(sum, ZW::omega(phase));
  }
  return zw_mul(sum, scalar_value(g.s2, g.ph, g.fac, pv));
}

namespace {

struct Decomposer {
  int policy;
  std::vector<Term>* out;
  DecompStats* st;
  const std::vector<double>* scores;
  int first;

  void emit(Graph& g) {
    if (g.zero) return;
    g.fold_phase_factors();
    if (st->budget && out->size() >= st->budget)
      fail(TSIM_ERR_CHI_BUDGET, "stabilizer terms exceed the budget (" + std::to_string(st->budget) + ")");
    if (st->total && st->total_budget && ++*st->total > st->total_budget)
      fail(TSIM_ERR_CHI_BUDGET, "stabilizer terms of the program exceed the budget (" +
                                    std::to_string(st->total_budget) + ")");
    if (st->shared_total && st->total_budget && st->shared_total->fetch_add(1) + 1 > st->total_budget)
      fail(TSIM_ERR_CHI_BUDGET, "stabilizer terms of the program exceed the budget (" +
                                    std::to_string(st->total_budget) + ")");
    out->push_back(g.as_term());
  }

  // Partial Cat5 decomposition (Appendix "Stabilizer decompositions", Eq.
  // cat5) of five odd spiders z_0..z_4, at theta = pi/4, in path-sum form.
  // Each spider's weight is w^(lam_k z_k) = w^(z_k) w^((lam_k - 1) z_k); the
  // product of the five w^(z_k), a function of the Hamming weight k = |z|,
  // equals  2 A + (w^3 / sqrt2^3) B + (w^5 / sqrt2^3) C  with
  //   A = [k = 0] + w^5 [k = 5]                  (the five spiders fused),
  //   B = sum_{c,y} (-1)^(c k + c y) w^(-y)      (= 2 for even k, 2 w^-1 odd),
  //   C = i^k sum_{c,y} (-1)^(c k + c y) w^(y)   (= 2 i^k for even k, 2 w i^k odd),
  // i.e. the paper's three terms with coefficients 1 - e^(4i theta) = 2,
  // 2 e^(3i theta) cos(theta) and 2 e^(3i theta) i sin(theta) up to the
  // normalisation of its Hadamard edges.  Every branch keeps one odd spider
  // (the fused z_0, or y), so five become one at three terms: growth
  // 2^(alpha T) with alpha = log2(3) / 4.
  void cat5(Graph& g, const int* v, int depth) {
    {  // 2 A: z_1..z_4 fused into z_0, whose phase becomes the sum of the five
      Graph h = g;
      for (int k = 1; k < 5; ++k) h.substitute(v[k], form_var(g.np, v[0]));
      h.s2 += 2;
      run(h, depth + 1);
    }
    for (int br = 0; br < 2; ++br) {
      // B: lam_k - 1, new c (phase 0) joined to every z_k and to y (phase -pi/4);
      // C: lam_k + 1 (the i^(z_k)), y with phase +pi/4
      Graph h = g;
      const int dl = br == 0 ? 7 : 1;
      for (int k = 0; k < 5; ++k) h.lam[(size_t)v[k]] = (h.lam[(size_t)v[k]] + dl) & 7;
      const int c = h.add_var(0);
      const int y = h.add_var(br == 0 ? 7 : 1);
      for (int k = 0; k < 5; ++k) h.toggle(c, v[k]);
      h.toggle(c, y);
      h.s2 -= 3;
      h.ph = (h.ph + (br == 0 ? 3 : 5)) & 7;
      run(h, depth + 1);
    }
  }

  void run(Graph& g, int depth) {
    // branches that vanish are pruned without a term; bound the search too
    if (st->budget && ++st->nodes > 64 * st->budget)
      fail(TSIM_ERR_CHI_BUDGET, "stabilizer decomposition search exceeds 64x the term budget");
    g.simplify();
    if (g.zero) return;
    std::vector<int> odd;
    for (int v = 0; v < g.n; ++v)
      if (g.alive[(size_t)v] && g.non_clifford(v)) odd.push_back(v);
    if (odd.empty()) {
      if (g.num_alive() != 0) fail(TSIM_ERR_INTERNAL, "Clifford diagram did not reduce to a scalar");
      st->leaves++;
      emit(g);
      return;
    }
    if (depth == 0 || g.num_alive() * 2 < g.n) g.compact();
    odd.clear();
    for (int v = 0; v < g.n; ++v)
      if (g.alive[(size_t)v] && g.non_clifford(v)) odd.push_back(v);
    auto score = [&](int v) {
      const int u = g.uid[(size_t)v];
      if (u >= 0 && u == first) return -1e300;
      if (policy == 1 && scores && u >= 0 && (size_t)u < scores->size()) return (*scores)[(size_t)u];
      return policy == 1 ? 1e300 : 0.0;
    };
    if (first >= 0 || (policy == 1 && scores)) {
      std::stable_sort(odd.begin(), odd.end(), [&](int a, int b) { return score(a) < score(b); });
    }
    // Cat5 (policy 4 always; the heuristic only when no pair of consecutive
    // odd spiders has phases that cancel, lam_x + lam_y = 0 mod 8: such a
    // pair -- typically a T gate's ket and bra copies in the doubled diagram
    // -- fuses away in the pair split, which then beats Cat5 by far)
    // (Cat5 at theta = pi/4 only: a group with an arbitrary angle is split in pairs)
    if ((policy == 0 || policy == 1 || policy == 4) && odd.size() >= 5 && g.ang[(size_t)odd[0]] == 0.0 &&
        g.ang[(size_t)odd[1]] == 0.0 && g.ang[(size_t)odd[2]] == 0.0 && g.ang[(size_t)odd[3]] == 0.0 &&
        g.ang[(size_t)odd[4]] == 0.0) {
      bool cancelling = false;
      for (size_t i = 0; policy != 4 && i + 1 < odd.size() && !cancelling; ++i)
        cancelling = ((g.lam[(size_t)odd[i]] + g.lam[(size_t)odd[i + 1]]) & 7) == 0 &&
                     angle_eighths(g.ang[(size_t)odd[i]] + g.ang[(size_t)odd[i + 1]]) == 0;
      if (!cancelling) {
        cat5(g, odd.data(), depth);
        return;
      }
    }
    if (policy == 2 || odd.size() == 1) {
      int v = odd[0];
      for (int c = 0; c < 2; ++c) {
        Graph h = g;
        h.substitute(v, form_const(g.np, c));
        run(h, depth + 1);
      }
      return;
    }
    // a pair of odd spiders x, y: sum_{z_y} = [z_y = z_x] + [z_y = z_x + 1];
    // both branches leave x with an even (Clifford) phase
    int x = odd[0], y = odd[1];
    for (int c = 0; c < 2; ++c) {
      Graph h = g;
      Form L = form_var(g.np, x);
      L.c = c;
      h.substitute(y, L);
      run(h, depth + 1);
    }
  }
};

}  // namespace

void decompose(Graph g, int policy, std::vector<Term>& out, DecompStats& st,
               const std::vector<double>* scores, int first) {
  Decomposer d{policy, &out, &st, scores, first};
  d.run(g, 0);
  st.terms = out.size();
}

}  // namespace tsim

namespace tsim {

std::vector<std::vector<int>> cut_units(const Graph& g) {
  std::vector<int> odd;
  for (int v = 0; v < g.n; ++v)
    if (g.alive[(size_t)v] && g.non_clifford(v)) odd.push_back(v);
  std::vector<std::vector<int>> units;
  for (size_t i = 0; i < odd.size();) {
    const int a = odd[i];
    if (i + 1 < odd.size()) {
      const int b = odd[i + 1];
      if (((g.lam[(size_t)a] + g.lam[(size_t)b]) & 7) == 0 && angle_eighths(g.ang[(size_t)a] + g.ang[(size_t)b]) == 0) {
        units.push_back({a, b});
        i += 2;
        continue;
      }
    }
    units.push_back({a});
    i += 1;
  }
  return units;
}

std::vector<double> unit_order_scores(const Graph& g, const std::vector<std::vector<int>>& units,
                                      const std::vector<int>& order) {
  std::vector<double> sc((size_t)g.n, 1e300);
  double r = 0;
  for (int u : order)
    for (int v : units[(size_t)u]) {
      const int id = g.uid[(size_t)v] >= 0 ? g.uid[(size_t)v] : v;
      if ((size_t)id >= sc.size()) sc.resize((size_t)id + 1, 1e300);
      sc[(size_t)id] = r;
      r += 1;
    }
  return sc;
}

void cut_features(const Graph& g, std::vector<float>& X, std::vector<int>& rowptr, std::vector<int>& col,
                  std::vector<int>& uids) {
  std::vector<int> idx((size_t)g.n, -1);
  int m = 0;
  for (int v = 0; v < g.n; ++v)
    if (g.alive[(size_t)v]) idx[(size_t)v] = m++;
  X.assign((size_t)m * kCutFeatures, 0.0f);
  rowptr.assign((size_t)m + 1, 0);
  col.clear();
  uids.assign((size_t)m, -1);
  for (int v = 0; v < g.n; ++v) {
    if (!g.alive[(size_t)v]) continue;
    const int i = idx[(size_t)v];
    const int l = g.lam[(size_t)v];
    float* x = &X[(size_t)i * kCutFeatures];
    const std::vector<int> nb = g.nbrs(v);
    int odd_nb = 0;
    for (int u : nb) {
      col.push_back(idx[(size_t)u]);
      odd_nb += g.non_clifford(u);
    }
    rowptr[(size_t)i + 1] = (int)col.size();
    x[0] = (float)g.non_clifford(v);            // non-Clifford
    x[1] = (float)(l == 0 || l == 4);            // Pauli
    x[2] = (float)(l == 2 || l == 6);            // proper Clifford
    x[3 + l] = 1.0f;                             // phase mod 2pi in units of pi/4
    x[11] = std::log1p((float)nb.size());        // degree
    x[12] = g.P[(size_t)v].any() ? 1.0f : 0.0f;  // parameter-dependent phase
    x[13] = nb.empty() ? 0.0f : (float)odd_nb / (float)nb.size();
    uids[(size_t)i] = g.uid[(size_t)v];
  }
}

Graph random_zx_diagram(uint64_t seed, int t, int c) {
  uint64_t s = seed * 0x9E3779B97F4A7C15ull + 0xD1B54A32D192ED03ull;
  auto next = [&]() {  // splitmix64
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  Graph g(1);
  const int n = t + c;
  for (int v = 0; v < n; ++v) {
    const int l = v < t ? (int)(1 + 2 * (next() % 4)) : (int)(2 * (next() % 4));
    g.add_var(l);
  }
  for (int v = 0; v < n; ++v)
    for (int k = 0; k < 3; ++k) {
      const int u = (int)(next() % (uint64_t)n);
      if (u != v && !g.edge(u, v)) g.toggle(u, v);
    }
  return g;
}

}  // namespace tsim
