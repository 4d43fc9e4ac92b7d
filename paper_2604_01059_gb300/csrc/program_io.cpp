// Program text format (save / load).  Line-oriented, whitespace separated;
// masks are W words of 16 hex digits (word 0 first), thresholds decimal:
//
//   TSIMPROG 2
//   mode detectors|measurements
//   nx <n_x>  words <W>  nf <n_f>  nr <n_random>
//   nmeas <N_m>  ndet <N_d>  nobs <N_o>
//   outputs <n>          then per output, in autoregressive order:
//     D <mask words> <const>          deterministic: bit = <mask, X> ^ const
//     R <xbit> <chain> <table>        drawn by Algorithm 1 from `table`
//   chains <n>           then  C <normalisation table>  per chain
//   channels <n>         then per channel:
//     K <n_outcomes> <thr_0> .. <thr_{n-2}>    outcome o iff U < thr[o] (first)
//     S <signature words>                      one line per outcome: X ^= sig
//   noise <mode> <groups>  mode 0: one word per channel; mode 1: geometric
//                        gaps, then per group  G <Q> <n> <channel indices>
//   tables <n>           then per table  T <terms> <float>, per term
//     t <s0> <j0> <m> [<phase>]   (c^t = w^j0 sqrt2^s0 e^(i pi phase); the
//                                   phase only in tables with float = 1)
//     and per factor  f <kind> <alpha> <beta> <u words> <v words> [<t>]
//     (kind 4, e^(i pi t a), carries its angle t in units of pi)
//   detmap <n> / obsmap <n>   then  M <count> <measurement indices>
//                             (measurement mode; 0 otherwise)
//   meta nq <qubits> E <raw bits> nft <table f bits>
//   raw <channels> <bits>     then per raw channel  Q <nbits> <probs 2^nbits>
//                             and one  B <column words>  line per bit
//   end
#include <cstdio>
#include <fstream>
#include <memory>
#include <sstream>

#include "device.h"
#include "program.h"

namespace tsim {
namespace {

void put_words(std::ostream& os, const std::vector<uint64_t>& w) {
  char buf[24];
  for (uint64_t x : w) {
    std::snprintf(buf, sizeof buf, " %016llx", (unsigned long long)x);
    os << buf;
  }
}

struct Reader {
  std::istream& is;
  int W = 1;
  std::string tok() {
    std::string t;
    if (!(is >> t)) fail(TSIM_ERR_PARSE, "program file truncated");
    return t;
  }
  void expect(const char* w) {
    std::string t = tok();
    if (t != w) fail(TSIM_ERR_PARSE, std::string("program file: expected '") + w + "', got '" + t + "'");
  }
  long long integer() {
    std::string t = tok();
    char* end = nullptr;
    long long v = std::strtoll(t.c_str(), &end, 10);
    if (!end || *end) fail(TSIM_ERR_PARSE, "program file: bad integer '" + t + "'");
    return v;
  }
  double real() {
    std::string t = tok();
    char* end = nullptr;
    double v = std::strtod(t.c_str(), &end);
    if (!end || *end) fail(TSIM_ERR_PARSE, "program file: bad number '" + t + "'");
    return v;
  }
  std::vector<uint64_t> words() {
    std::vector<uint64_t> w((size_t)W);
    for (int i = 0; i < W; ++i) {
      std::string t = tok();
      char* end = nullptr;
      w[(size_t)i] = std::strtoull(t.c_str(), &end, 16);
      if (!end || *end) fail(TSIM_ERR_PARSE, "program file: bad mask word '" + t + "'");
    }
    return w;
  }
};

}  // namespace

void save_program(const Program& p, const std::string& path) {
  std::ofstream os(path);
  if (!os) fail(TSIM_ERR_ARG, "cannot open " + path + " for writing");
  os << "TSIMPROG 2\nmode " << (p.mode == TSIM_MODE_MEASUREMENTS ? "measurements" : "detectors") << "\n";
  os << "nx " << p.nx << "\nwords " << p.W << "\nnf " << p.nf << "\nnr " << p.nr << "\n";
  os << "nmeas " << p.nmeas << "\nndet " << p.ndet << "\nnobs " << p.nobs << "\n";
  os << "outputs " << p.outputs.size() << "\n";
  for (const ProgOutput& o : p.outputs) {
    if (o.random) {
      os << "R " << o.xbit << " " << o.chain << " " << o.table << "\n";
    } else {
      os << "D";
      put_words(os, o.mask);
      os << " " << o.cst << "\n";
    }
  }
  os << "chains " << p.chain_norm.size() << "\n";
  for (int t : p.chain_norm) os << "C " << t << "\n";
  os << "channels " << p.channels.size() << "\n";
  for (const ProgChannel& c : p.channels) {
    os << "K " << c.sig.size();
    for (uint32_t t : c.thr) os << " " << t;
    os << "\n";
    for (const auto& s : c.sig) {
      os << "S";
      put_words(os, s);
      os << "\n";
    }
  }
  os << "noise " << p.noise_mode << " " << p.groups.size() << "\n";
  for (const NoiseGroup& g : p.groups) {
    os << "G " << g.Q << " " << g.member.size();
    for (int c : g.member) os << " " << c;
    os << "\n";
  }
  os << "tables " << p.tables.size() << "\n";
  for (const ProgTable& tb : p.tables) {
    const bool fl = tb.is_float();
    os << "T " << tb.terms.size() << " " << (fl ? 1 : 0) << "\n";
    char num[40];
    for (const ProgTerm& tm : tb.terms) {
      os << "t " << tm.s0 << " " << tm.j0 << " " << tm.f.size();
      if (fl) {
        std::snprintf(num, sizeof num, " %.17g", tm.fph);
        os << num;
      }
      os << "\n";
      for (const ProgFactor& f : tm.f) {
        os << "f " << f.kind << " " << f.alpha << " " << f.beta;
        put_words(os, f.u);
        put_words(os, f.v);
        if (f.kind == 4) {
          std::snprintf(num, sizeof num, " %.17g", f.t);
          os << num;
        }
        os << "\n";
      }
    }
  }
  auto maps = [&](const char* name, const std::vector<std::vector<int>>& m) {
    os << name << " " << m.size() << "\n";
    for (const auto& d : m) {
      os << "M " << d.size();
      for (int j : d) os << " " << j;
      os << "\n";
    }
  };
  maps("detmap", p.detmap);
  maps("obsmap", p.obsmap);
  os << "meta nq " << p.nq << " E " << p.E << " nft " << p.nft << "\n";
  int nbits = 0;
  for (const RawInfo& r : p.raw) nbits += r.nbits;
  os << "raw " << p.raw.size() << " " << nbits << "\n";
  char buf[40];
  for (const RawInfo& r : p.raw) {
    os << "Q " << r.nbits;
    for (double q : r.probs) {
      std::snprintf(buf, sizeof buf, " %.17g", q);
      os << buf;
    }
    os << "\n";
    for (const auto& c : r.cols) {
      os << "B";
      put_words(os, c);
      os << "\n";
    }
  }
  os << "end\n";
  if (!os) fail(TSIM_ERR_ARG, "write failed: " + path);
}

Program* load_program(const std::string& path) {
  std::ifstream is(path);
  if (!is) fail(TSIM_ERR_ARG, "cannot open " + path);
  Reader R{is};
  auto p = std::make_unique<Program>();
  R.expect("TSIMPROG");
  if (R.integer() != 2) fail(TSIM_ERR_PARSE, "unknown program version");
  R.expect("mode");
  std::string m = R.tok();
  if (m != "detectors" && m != "measurements") fail(TSIM_ERR_PARSE, "bad mode");
  p->mode = m == "measurements" ? TSIM_MODE_MEASUREMENTS : TSIM_MODE_DETECTORS;
  R.expect("nx"); p->nx = (int)R.integer();
  R.expect("words"); p->W = (int)R.integer();
  R.expect("nf"); p->nf = (int)R.integer();
  R.expect("nr"); p->nr = (int)R.integer();
  R.expect("nmeas"); p->nmeas = (int)R.integer();
  R.expect("ndet"); p->ndet = (int)R.integer();
  R.expect("nobs"); p->nobs = (int)R.integer();
  if (p->W < 1 || p->W > 1024 || p->nx > p->W * 64) fail(TSIM_ERR_PARSE, "bad word count");
  R.W = p->W;
  R.expect("outputs");
  long long n = R.integer();
  p->outputs.resize((size_t)n);
  for (auto& o : p->outputs) {
    std::string t = R.tok();
    if (t == "D") {
      o.mask = R.words();
      o.cst = (int)R.integer() & 1;
    } else if (t == "R") {
      o.random = true;
      o.xbit = (int)R.integer();
      o.chain = (int)R.integer();
      o.table = (int)R.integer();
      o.mask.assign((size_t)p->W, 0);
    } else {
      fail(TSIM_ERR_PARSE, "bad output line");
    }
  }
  R.expect("chains");
  n = R.integer();
  for (long long i = 0; i < n; ++i) { R.expect("C"); p->chain_norm.push_back((int)R.integer()); }
  R.expect("channels");
  n = R.integer();
  p->channels.resize((size_t)n);
  for (auto& c : p->channels) {
    R.expect("K");
    long long k = R.integer();
    if (k < 1 || k > 64) fail(TSIM_ERR_PARSE, "bad outcome count");
    for (long long i = 0; i + 1 < k; ++i) c.thr.push_back((uint32_t)R.integer());
    for (long long i = 0; i < k; ++i) { R.expect("S"); c.sig.push_back(R.words()); }
  }
  R.expect("noise");
  p->noise_mode = (int)R.integer();
  n = R.integer();
  if (p->noise_mode < 0 || p->noise_mode > 1 || n < 0 || (p->noise_mode == 0 && n != 0))
    fail(TSIM_ERR_PARSE, "bad noise section");
  {
    std::vector<char> seen(p->channels.size(), 0);
    for (long long g = 0; g < n; ++g) {
      R.expect("G");
      NoiseGroup G;
      long long q = R.integer();
      long long m = R.integer();
      if (q < 0 || q > 0xFFFFFFFFll || m < 1) fail(TSIM_ERR_PARSE, "bad noise group");
      G.Q = (uint32_t)q;
      for (long long k = 0; k < m; ++k) {
        long long c = R.integer();
        if (c < 0 || c >= (long long)p->channels.size() || seen[(size_t)c]) fail(TSIM_ERR_PARSE, "bad noise group member");
        const ProgChannel& ch = p->channels[(size_t)c];
        if (ch.thr.empty() || ch.thr[0] < G.Q) fail(TSIM_ERR_PARSE, "noise group Q above a member's outcome-0 threshold");
        seen[(size_t)c] = 1;
        G.member.push_back((int)c);
      }
      p->groups.push_back(std::move(G));
    }
    if (p->noise_mode == 1)
      for (size_t c = 0; c < p->channels.size(); ++c)
        if (!p->channels[c].thr.empty() && !seen[c]) fail(TSIM_ERR_PARSE, "a channel is in no noise group");
  }
  R.expect("tables");
  n = R.integer();
  p->tables.resize((size_t)n);
  for (auto& tb : p->tables) {
    R.expect("T");
    long long nt = R.integer();
    const long long fl = R.integer();
    if (fl != 0 && fl != 1) fail(TSIM_ERR_PARSE, "bad table float flag");
    tb.terms.resize((size_t)nt);
    for (auto& tm : tb.terms) {
      R.expect("t");
      tm.s0 = (int)R.integer();
      tm.j0 = (int)R.integer();
      long long nf = R.integer();
      if (fl) tm.fph = R.real();
      tm.f.resize((size_t)nf);
      for (auto& f : tm.f) {
        R.expect("f");
        f.kind = (int)R.integer();
        f.alpha = (int)R.integer();
        f.beta = (int)R.integer();
        f.u = R.words();
        f.v = R.words();
        if (f.kind < 0 || f.kind > 4) fail(TSIM_ERR_PARSE, "bad factor kind");
        if (f.kind == 4) {
          if (!fl) fail(TSIM_ERR_PARSE, "arbitrary phase factor in an exact table");
          f.t = R.real();
        }
      }
    }
  }
  auto maps = [&](const char* name, std::vector<std::vector<int>>& mm) {
    R.expect(name);
    long long k = R.integer();
    mm.resize((size_t)k);
    for (auto& d : mm) {
      R.expect("M");
      long long c = R.integer();
      for (long long i = 0; i < c; ++i) d.push_back((int)R.integer());
    }
  };
  maps("detmap", p->detmap);
  maps("obsmap", p->obsmap);
  R.expect("meta");
  R.expect("nq"); p->nq = (int)R.integer();
  R.expect("E"); p->E = (int)R.integer();
  R.expect("nft"); p->nft = (int)R.integer();
  R.expect("raw");
  n = R.integer();
  R.integer();
  p->raw.resize((size_t)n);
  for (auto& r : p->raw) {
    R.expect("Q");
    r.nbits = (int)R.integer();
    if (r.nbits < 0 || r.nbits > 8) fail(TSIM_ERR_PARSE, "bad raw channel");
    for (int i = 0; i < (1 << r.nbits); ++i) r.probs.push_back(R.real());
    for (int b = 0; b < r.nbits; ++b) { R.expect("B"); r.cols.push_back(R.words()); }
  }
  R.expect("end");
  // structural validation
  for (const auto& o : p->outputs)
    if (o.random && (o.xbit < 0 || o.xbit >= p->nx || o.chain < 0 || o.chain >= (int)p->chain_norm.size() ||
                     o.table < 0 || o.table >= (int)p->tables.size()))
      fail(TSIM_ERR_PARSE, "output refers outside the program");
  for (int t : p->chain_norm)
    if (t < 0 || t >= (int)p->tables.size()) fail(TSIM_ERR_PARSE, "chain refers to a missing table");
  if (p->mode == TSIM_MODE_DETECTORS && (int)p->outputs.size() != p->ndet + p->nobs)
    fail(TSIM_ERR_PARSE, "output count mismatch");
  if (p->mode == TSIM_MODE_MEASUREMENTS && (int)p->outputs.size() != p->nmeas)
    fail(TSIM_ERR_PARSE, "output count mismatch");
  prepare_device_tables(*p);
  return p.release();
}

}  // namespace tsim
