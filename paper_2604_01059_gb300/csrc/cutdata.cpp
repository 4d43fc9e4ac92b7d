// Training data for the learned cut order: ZX diagrams of the marginals of
// seeded random Clifford+T circuits, each reduced by the Clifford rewrites
// exactly as the compiler reduces it, with every candidate cut unit (a
// cancelling ket/bra pair of one T gate, or a single non-Clifford spider)
// labelled, on its members, by the exact number of stabilizer terms the
// compiler produces when that unit is split first (the rest in the heuristic
// order).  The labels are measured, not estimated: they are the term counts
// of real decompositions, capped by a budget.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <thread>

#include <cuda_runtime.h>

#include "cutnet.h"
#include "program.h"
#include "zx.h"

namespace tsim {
namespace {

struct CutGraph {
  std::vector<float> X, y;
  std::vector<int> rowptr, col;
};

uint64_t mix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// A seeded random Clifford+T circuit: q qubits, layers of CX pairs on random
// partners (density 0.4) and single-qubit gates (T or T_DAG with probability
// 1/4, else H, S, S_DAG or SQRT_X) until t T/T_DAG gates are placed,
// DEPOLARIZE1(1e-3) after every layer, Z measurement of every qubit.
std::string random_circuit(uint64_t r, int q, int t) {
  std::string c = "R";
  for (int i = 0; i < q; ++i) c += " " + std::to_string(i);
  c += "\n";
  static const char* one[] = {"H", "S", "S_DAG", "SQRT_X"};
  int placed = 0;
  std::vector<int> qs((size_t)q);
  while (placed < t) {
    for (int i = 0; i < q; ++i) qs[(size_t)i] = i;
    for (size_t i = qs.size(); i > 1; --i) {
      r = mix(r);
      std::swap(qs[i - 1], qs[(size_t)(r % i)]);
    }
    const int pairs = (int)(0.4 * q / 2 + 0.5);
    for (int k = 0; k < pairs; ++k)
      c += "CX " + std::to_string(qs[(size_t)(2 * k)]) + " " + std::to_string(qs[(size_t)(2 * k + 1)]) + "\n";
    for (size_t k = (size_t)(2 * pairs); k < qs.size(); ++k) {
      r = mix(r);
      const int qb = qs[k];
      if ((r & 3) == 0 && placed < t) {
        c += ((r >> 2) & 1 ? "T_DAG " : "T ") + std::to_string(qb) + "\n";
        ++placed;
      } else {
        c += std::string(one[(r >> 3) % 4]) + " " + std::to_string(qb) + "\n";
      }
    }
    c += "DEPOLARIZE1(0.001)";
    for (int i = 0; i < q; ++i) c += " " + std::to_string(i);
    c += "\n";
  }
  c += "M";
  for (int i = 0; i < q; ++i) c += " " + std::to_string(i);
  return c + "\n";
}

int odd_count(const Graph& g) {
  int k = 0;
  for (int v = 0; v < g.n; ++v) k += g.alive[(size_t)v] && g.non_clifford(v);
  return k;
}

// Training graph gi: one marginal diagram (chosen at random among those with
// two or more non-Clifford spiders) of a random circuit with t_min..t_max
// T/T_DAG gates on 3..10 qubits.
// The marginal diagram of training graph gi (see make_graph), compacted,
// with uid = vertex index; r receives the generator state after it.
Graph pick_graph(uint64_t seed, int gi, int t_min, int t_max, uint64_t& r) {
  r = mix(seed * 1000003ull + (uint64_t)gi);
  Graph g;
  for (int attempt = 0; attempt < 8; ++attempt) {
    r = mix(r);
    const int t = t_min + (int)(r % (uint64_t)(t_max - t_min + 1));
    r = mix(r);
    const int q = 3 + (int)(r % 8);
    std::vector<Graph> ms = marginal_diagrams(random_circuit(mix(r), q, t), TSIM_MODE_MEASUREMENTS);
    std::vector<size_t> ok;
    for (size_t i = 0; i < ms.size(); ++i)
      if (!ms[i].zero && odd_count(ms[i]) >= 2) ok.push_back(i);
    if (ok.empty()) continue;
    r = mix(r);
    g = std::move(ms[ok[(size_t)(r % ok.size())]]);
    break;
  }
  g.compact();
  for (int v = 0; v < g.n; ++v) g.uid[(size_t)v] = v;
  return g;
}

// terms when unit u is split first and the rest follow the heuristic order
// (2 budget when they exceed the budget)
double unit_first_terms(const Graph& g, const std::vector<std::vector<int>>& units, int u, uint64_t budget) {
  std::vector<int> order{u};
  for (size_t k = 0; k < units.size(); ++k)
    if ((int)k != u) order.push_back((int)k);
  const std::vector<double> sc = unit_order_scores(g, units, order);
  std::vector<Term> terms;
  DecompStats st;
  st.budget = budget;
  try {
    decompose(g, TSIM_DECOMP_LEARNED, terms, st, &sc);
  } catch (const Error& e) {
    if (e.code != TSIM_ERR_CHI_BUDGET) throw;
    return 2.0 * (double)budget;
  }
  return (double)std::max<size_t>(1, terms.size());
}

// terms of one decomposition, 2 budget when it exceeds the budget
double count_terms(const Graph& g, int policy, uint64_t budget, int first) {
  std::vector<Term> terms;
  DecompStats st;
  st.budget = budget;
  try {
    decompose(g, policy, terms, st, nullptr, first);
  } catch (const Error& e) {
    if (e.code != TSIM_ERR_CHI_BUDGET) throw;
    return 2.0 * (double)budget;
  }
  return (double)std::max<size_t>(1, terms.size());
}

void make_graph(uint64_t seed, int gi, int t_min, int t_max, uint64_t budget, int max_cand, CutGraph& out) {
  uint64_t r = 0;
  Graph g = pick_graph(seed, gi, t_min, t_max, r);
  std::vector<int> uids;
  cut_features(g, out.X, out.rowptr, out.col, uids);
  out.y.assign(uids.size(), NAN);
  // candidates: a seeded shuffle of the cut units (cancelling pairs and
  // single spiders), at most max_cand; each is labelled, on every member,
  // with the terms when it is split first and the rest follow the heuristic
  const std::vector<std::vector<int>> units = cut_units(g);
  size_t n_odd = 0;
  for (const auto& u : units) n_odd += u.size();
  if (n_odd < 2) return;
  std::vector<int> order(units.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  for (size_t i = order.size(); i > 1; --i) {
    r = mix(r);
    std::swap(order[i - 1], order[(size_t)(r % i)]);
  }
  if ((int)order.size() > max_cand) order.resize((size_t)max_cand);
  for (int u : order) {
    const double count = unit_first_terms(g, units, u, budget);
    // after compact() every vertex is alive, so node index = vertex index
    for (int v : units[(size_t)u]) out.y[(size_t)v] = (float)std::log2(count);
  }
}

}  // namespace

// compile.cpp: one marginal decomposed by the policy of opts (LEARNED: the
// heuristic against the network's orders)
void decompose_marginal(Graph M, const tsim_compile_opts& opts, uint64_t budget, uint64_t* total,
                        std::vector<Term>& out, std::atomic<uint64_t>* shared_total = nullptr);

}  // namespace tsim

namespace tsim {
namespace cutnet {

void evaluate_one(uint64_t seed, int gi, int t_min, int t_max, uint64_t budget, double* row);

void evaluate_policy(uint64_t seed, int n_graphs, int t_min, int t_max, uint64_t budget, double* out) {
  if (n_graphs < 0 || t_min < 1 || t_max < t_min || !budget || !out) fail(TSIM_ERR_ARG, "bad evaluation parameters");
  // graphs in parallel host threads; the network's scorer serialises itself
  int dev = 0;
  cudaGetDevice(&dev);
  std::atomic<int> next{0}, failed{0};
  const unsigned nt = std::max(1u, std::thread::hardware_concurrency());
  std::vector<std::thread> pool;
  for (unsigned k = 0; k < nt; ++k)
    pool.emplace_back([&] {
      cudaSetDevice(dev);
      for (;;) {
        const int gi = next++;
        if (gi >= n_graphs) return;
        try {
          evaluate_one(seed, gi, t_min, t_max, budget, out + 5 * (size_t)gi);
        } catch (...) {
          failed++;
        }
      }
    });
  for (auto& th : pool) th.join();
  if (failed) fail(TSIM_ERR_INTERNAL, "a held-out graph could not be decomposed");
}

void evaluate_one(uint64_t seed, int gi, int t_min, int t_max, uint64_t budget, double* row) {
  {
    uint64_t r = 0;
    const Graph g = pick_graph(seed, gi, t_min, t_max, r);
    std::vector<int> odd;
    for (int v = 0; v < g.n; ++v)
      if (g.alive[(size_t)v] && g.non_clifford(v)) odd.push_back(v);
    row[0] = (double)odd.size();
    row[1] = count_terms(g, TSIM_DECOMP_HEURISTIC, budget, -1);
    {
      tsim_compile_opts o{};
      o.decomp = TSIM_DECOMP_LEARNED;
      std::vector<Term> terms;
      try {
        decompose_marginal(g, o, budget, nullptr, terms);
        row[2] = (double)std::max<size_t>(1, terms.size());
      } catch (const Error& e) {
        if (e.code != TSIM_ERR_CHI_BUDGET) throw;
        row[2] = 2.0 * (double)budget;
      }
    }
    const std::vector<std::vector<int>> units = cut_units(g);
    double sum = 0, best = row[1];
    int n = 0;
    for (size_t k = 0; k < units.size() && k < 16; ++k) {
      const double c = unit_first_terms(g, units, (int)k, budget);
      sum += std::log2(c);
      best = std::min(best, c);
      ++n;
    }
    row[3] = n ? std::exp2(sum / n) : row[1];  // geometric mean over first units: a random first unit
    row[4] = best;
  }
}

void write_dataset(uint64_t seed, int n_graphs, int t_min, int t_max, uint64_t budget, int max_candidates,
                   const std::string& path) {
  if (n_graphs < 0 || t_min < 1 || t_max < t_min || !budget || max_candidates < 1)
    fail(TSIM_ERR_ARG, "bad dataset parameters");
  std::vector<CutGraph> gs((size_t)n_graphs);
  std::atomic<int> next{0};
  std::atomic<int> failed{0};
  const unsigned nt = std::max(1u, std::thread::hardware_concurrency());
  std::vector<std::thread> pool;
  for (unsigned k = 0; k < nt; ++k)
    pool.emplace_back([&] {
      for (;;) {
        const int i = next++;
        if (i >= n_graphs) return;
        try {
          make_graph(seed, i, t_min, t_max, budget, max_candidates, gs[(size_t)i]);
        } catch (...) {
          failed++;
        }
      }
    });
  for (auto& th : pool) th.join();
  if (failed) fail(TSIM_ERR_INTERNAL, "a training graph could not be decomposed");
  FILE* f = std::fopen(path.c_str(), "wb");
  if (!f) fail(TSIM_ERR_ARG, "cannot open the dataset file for writing");
  auto w32 = [&](int32_t v) { std::fwrite(&v, 4, 1, f); };
  std::fwrite("TSIMCUTD", 1, 8, f);
  w32(n_graphs);
  w32(kCutFeatures);
  for (const CutGraph& g : gs) {
    const int n = (int)g.y.size();
    w32(n);
    w32((int32_t)g.col.size());
    if (n) {
      std::fwrite(g.X.data(), 4, g.X.size(), f);
      std::fwrite(g.rowptr.data(), 4, g.rowptr.size(), f);
      if (!g.col.empty()) std::fwrite(g.col.data(), 4, g.col.size(), f);
      std::fwrite(g.y.data(), 4, g.y.size(), f);
    }
  }
  if (std::fclose(f) != 0) fail(TSIM_ERR_ARG, "writing the dataset file failed");
}

Batch read_dataset(const std::string& path) {
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) fail(TSIM_ERR_ARG, "cannot open the dataset file");
  Batch b;
  auto bad = [&](const char* m) {
    std::fclose(f);
    fail(TSIM_ERR_PARSE, std::string("dataset file: ") + m);
  };
  char magic[8];
  int32_t hdr[2];
  if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, "TSIMCUTD", 8) || std::fread(hdr, 4, 2, f) != 2)
    bad("bad header");
  if (hdr[0] < 0 || hdr[1] != kCutFeatures) bad("feature count differs from the compiler's");
  b.goff.push_back(0);
  b.rowptr.push_back(0);
  for (int g = 0; g < hdr[0]; ++g) {
    int32_t nm[2];
    if (std::fread(nm, 4, 2, f) != 2 || nm[0] < 0 || nm[1] < 0) bad("truncated graph header");
    const int n = nm[0], nnz = nm[1];
    const int base = b.n;
    if (n) {
      std::vector<float> X((size_t)n * kCutFeatures), y((size_t)n);
      std::vector<int> rp((size_t)n + 1), col((size_t)nnz);
      if (std::fread(X.data(), 4, X.size(), f) != X.size() || std::fread(rp.data(), 4, rp.size(), f) != rp.size() ||
          (nnz && std::fread(col.data(), 4, col.size(), f) != col.size()) ||
          std::fread(y.data(), 4, y.size(), f) != y.size())
        bad("truncated graph");
      if (rp[0] != 0 || rp[(size_t)n] != nnz) bad("bad adjacency");
      for (int i = 0; i < n; ++i)
        if (rp[(size_t)i + 1] < rp[(size_t)i]) bad("bad adjacency");
      for (int c : col)
        if (c < 0 || c >= n) bad("neighbour out of range");
      b.X.insert(b.X.end(), X.begin(), X.end());
      b.y.insert(b.y.end(), y.begin(), y.end());
      const int e0 = (int)b.col.size();
      for (int i = 1; i <= n; ++i) b.rowptr.push_back(e0 + rp[(size_t)i]);
      for (int c : col) b.col.push_back(base + c);
      b.n += n;
    }
    b.goff.push_back(b.n);
  }
  std::fclose(f);
  return b;
}

}  // namespace cutnet
}  // namespace tsim
