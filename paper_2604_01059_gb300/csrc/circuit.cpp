// Stim-subset parser and raw noise-channel enumeration.
//
// Raw channels are numbered in circuit order (instruction, then target) and
// raw error bits channel after channel.  Bit encodings follow Appendix "Pauli
// noise channels": two bits (e_x, e_z) per qubit, (1,0) = X, (1,1) = Y,
// (0,1) = Z; a two-qubit channel uses (x_a, z_a, x_b, z_b).  PAULI_CHANNEL_2
// lists its 15 probabilities in the order IX IY IZ XI XX XY XZ YI YX YY YZ ZI
// ZX ZY ZZ (first letter = first target).  A noisy measurement M(p) owns one
// bit that flips its recorded outcome.
#include "circuit.h"

#include <cctype>
#include <cmath>
#include <cstdlib>
#include <map>
#include <sstream>

namespace tsim {
namespace {

const std::map<std::string, Op>& op_table() {
  static const std::map<std::string, Op> t = {
      {"I", Op::I}, {"X", Op::X}, {"Y", Op::Y}, {"Z", Op::Z}, {"H", Op::H}, {"H_XZ", Op::H},
      {"S", Op::S}, {"SQRT_Z", Op::S}, {"S_DAG", Op::S_DAG}, {"SQRT_Z_DAG", Op::S_DAG},
      {"SQRT_X", Op::SQRT_X}, {"SQRT_X_DAG", Op::SQRT_X_DAG}, {"T", Op::T}, {"T_DAG", Op::T_DAG},
      {"R_X", Op::R_X}, {"R_Y", Op::R_Y}, {"R_Z", Op::R_Z}, {"U3", Op::U3},
      {"CX", Op::CX}, {"CNOT", Op::CX}, {"ZCX", Op::CX}, {"CY", Op::CY}, {"ZCY", Op::CY},
      {"CZ", Op::CZ}, {"ZCZ", Op::CZ}, {"SWAP", Op::SWAP},
      {"R", Op::R}, {"RZ", Op::R}, {"RX", Op::RX}, {"M", Op::M}, {"MZ", Op::M}, {"MX", Op::MX},
      {"MR", Op::MR}, {"MRZ", Op::MR}, {"MRX", Op::MRX},
      {"X_ERROR", Op::X_ERROR}, {"Y_ERROR", Op::Y_ERROR}, {"Z_ERROR", Op::Z_ERROR},
      {"DEPOLARIZE1", Op::DEPOLARIZE1}, {"PAULI_CHANNEL_1", Op::PAULI_CHANNEL_1},
      {"DEPOLARIZE2", Op::DEPOLARIZE2}, {"PAULI_CHANNEL_2", Op::PAULI_CHANNEL_2},
      {"DETECTOR", Op::DETECTOR}, {"OBSERVABLE_INCLUDE", Op::OBSERVABLE_INCLUDE}};
  return t;
}

std::string upper(std::string s) {
  for (char& c : s) c = (char)std::toupper((unsigned char)c);
  return s;
}

std::string trim(const std::string& s) {
  size_t a = 0, b = s.size();
  while (a < b && std::isspace((unsigned char)s[a])) ++a;
  while (b > a && std::isspace((unsigned char)s[b - 1])) --b;
  return s.substr(a, b - a);
}

struct Line {
  std::string name;
  std::vector<double> args;
  std::vector<Target> t;
  bool has_args = false;
  std::string rest;
};

Line parse_line(const std::string& line, int lineno) {
  Line L;
  size_t i = 0;
  while (i < line.size() && (std::isalnum((unsigned char)line[i]) || line[i] == '_')) ++i;
  L.name = upper(line.substr(0, i));
  if (L.name.empty()) fail(TSIM_ERR_PARSE, "line " + std::to_string(lineno) + ": no instruction name");
  std::string rest = line.substr(i);
  size_t p = rest.find_first_not_of(" \t");
  if (p != std::string::npos && rest[p] == '(') {
    size_t q = rest.find(')', p);
    if (q == std::string::npos) fail(TSIM_ERR_PARSE, "line " + std::to_string(lineno) + ": missing ')'");
    std::string a = rest.substr(p + 1, q - p - 1);
    std::stringstream ss(a);
    std::string tok;
    while (std::getline(ss, tok, ',')) {
      tok = trim(tok);
      if (tok.empty()) continue;
      char* end = nullptr;
      double v = std::strtod(tok.c_str(), &end);
      if (!end || *end) fail(TSIM_ERR_PARSE, "line " + std::to_string(lineno) + ": bad argument '" + tok + "'");
      L.args.push_back(v);
    }
    L.has_args = true;
    rest = rest.substr(q + 1);
  }
  L.rest = trim(rest);
  return L;
}

void parse_targets(const std::string& rest, std::vector<Target>& out, int lineno) {
  std::stringstream ss(rest);
  std::string tok;
  while (ss >> tok) {
    Target t;
    if (tok.rfind("rec[", 0) == 0 && tok.back() == ']') {
      t.rec = true;
      t.v = std::atoi(tok.substr(4, tok.size() - 5).c_str());
      if (t.v >= 0) fail(TSIM_ERR_PARSE, "line " + std::to_string(lineno) + ": rec index must be negative");
    } else {
      char* end = nullptr;
      long v = std::strtol(tok.c_str(), &end, 10);
      if (!end || *end || v < 0 || v > (1 << 20))
        fail(TSIM_ERR_PARSE, "line " + std::to_string(lineno) + ": bad target '" + tok + "'");
      t.v = (int)v;
    }
    out.push_back(t);
  }
}

void parse_block(const std::vector<std::string>& lines, size_t& pos, bool in_repeat,
                 std::vector<Instr>& out) {
  while (pos < lines.size()) {
    const std::string& s = lines[pos];
    int lineno = (int)pos + 1;
    if (s == "}") {
      if (!in_repeat) fail(TSIM_ERR_PARSE, "unbalanced '}'");
      ++pos;
      return;
    }
    Line L = parse_line(s, lineno);
    if (L.name == "REPEAT") {
      std::string r = L.rest;
      if (r.empty() || r.back() != '{') fail(TSIM_ERR_PARSE, "REPEAT needs '{'");
      long n = std::strtol(trim(r.substr(0, r.size() - 1)).c_str(), nullptr, 10);
      if (n < 0) fail(TSIM_ERR_PARSE, "bad REPEAT count");
      ++pos;
      std::vector<Instr> body;
      parse_block(lines, pos, true, body);
      for (long k = 0; k < n; ++k) out.insert(out.end(), body.begin(), body.end());
      continue;
    }
    if (L.name == "TICK" || L.name == "QUBIT_COORDS" || L.name == "SHIFT_COORDS") {
      ++pos;
      continue;
    }
    auto it = op_table().find(L.name);
    if (it == op_table().end()) fail(TSIM_ERR_UNSUPPORTED_GATE, "unsupported instruction " + L.name);
    Instr ins;
    ins.op = it->second;
    ins.args = L.args;
    parse_targets(L.rest, ins.t, lineno);
    out.push_back(ins);
    ++pos;
  }
  if (in_repeat) fail(TSIM_ERR_PARSE, "missing '}'");
}

std::vector<double> pc1(double px, double py, double pz) {
  // outcome index = e_x + 2 e_z
  return {1.0 - px - py - pz, px, pz, py};
}

int pauli_bits(char c) {  // (x, z) -> x | z << 1
  switch (c) {
    case 'I': return 0;
    case 'X': return 1;
    case 'Y': return 3;
    case 'Z': return 2;
  }
  return 0;
}

std::vector<double> pc2(const std::vector<double>& ps) {
  static const char* order[15] = {"IX", "IY", "IZ", "XI", "XX", "XY", "XZ", "YI",
                                  "YX", "YY", "YZ", "ZI", "ZX", "ZY", "ZZ"};
  std::vector<double> p(16, 0.0);
  double tot = 0;
  for (int i = 0; i < 15; ++i) {
    int a = pauli_bits(order[i][0]), b = pauli_bits(order[i][1]);
    p[(size_t)(a | (b << 2))] += ps[(size_t)i];
    tot += ps[(size_t)i];
  }
  p[0] = 1.0 - tot;
  return p;
}

void need_args(const Instr& in, size_t n, const char* name) {
  if (in.args.size() != n) fail(TSIM_ERR_PARSE, std::string(name) + ": wrong number of arguments");
  for (double a : in.args)
    if (!(a >= 0.0 && a <= 1.0)) fail(TSIM_ERR_PARSE, std::string(name) + ": probability out of range");
}

}  // namespace

Circuit parse_circuit(const std::string& text) {
  std::vector<std::string> lines;
  {
    std::stringstream ss(text);
    std::string l;
    while (std::getline(ss, l)) {
      size_t h = l.find('#');
      if (h != std::string::npos) l = l.substr(0, h);
      l = trim(l);
      // a '{' glued to REPEAT stays on its line; a lone '}' is its own line
      if (!l.empty()) lines.push_back(l);
    }
  }
  Circuit c;
  size_t pos = 0;
  std::vector<Instr> flat;
  parse_block(lines, pos, false, flat);
  int nmeas = 0, bit = 0;
  for (size_t idx = 0; idx < flat.size(); ++idx) {
    Instr& in = flat[idx];
    for (const Target& t : in.t)
      if (!t.rec) c.num_qubits = std::max(c.num_qubits, t.v + 1);
    auto add = [&](Op kind, int q0, int q1, int nb, std::vector<double> probs, int tpos) {
      RawChannel ch;
      ch.kind = kind;
      ch.q0 = q0;
      ch.q1 = q1;
      ch.nbits = nb;
      ch.probs = std::move(probs);
      ch.first_bit = bit;
      ch.instr = (int)idx;
      ch.target_pos = tpos;
      c.channels.push_back(ch);
      bit += nb;
    };
    switch (in.op) {
      case Op::M: case Op::MX: case Op::MR: case Op::MRX: {
        if (in.args.size() > 1) fail(TSIM_ERR_PARSE, "measurement takes at most one argument");
        double p = in.args.empty() ? 0.0 : in.args[0];
        if (!(p >= 0 && p <= 1)) fail(TSIM_ERR_PARSE, "measurement flip probability out of range");
        for (size_t k = 0; k < in.t.size(); ++k) {
          if (in.t[k].rec) fail(TSIM_ERR_PARSE, "measurement of a rec target");
          if (p > 0) add(Op::M, in.t[k].v, -1, 1, {1.0 - p, p}, (int)k);
          ++nmeas;
        }
        break;
      }
      case Op::X_ERROR: case Op::Y_ERROR: case Op::Z_ERROR:
        need_args(in, 1, "X/Y/Z_ERROR");
        for (size_t k = 0; k < in.t.size(); ++k) add(in.op, in.t[k].v, -1, 1, {1.0 - in.args[0], in.args[0]}, (int)k);
        break;
      case Op::DEPOLARIZE1:
        need_args(in, 1, "DEPOLARIZE1");
        for (size_t k = 0; k < in.t.size(); ++k) {
          double q = in.args[0] / 3.0;
          add(in.op, in.t[k].v, -1, 2, pc1(q, q, q), (int)k);
        }
        break;
      case Op::PAULI_CHANNEL_1:
        need_args(in, 3, "PAULI_CHANNEL_1");
        for (size_t k = 0; k < in.t.size(); ++k)
          add(in.op, in.t[k].v, -1, 2, pc1(in.args[0], in.args[1], in.args[2]), (int)k);
        break;
      case Op::DEPOLARIZE2:
        need_args(in, 1, "DEPOLARIZE2");
        if (in.t.size() % 2) fail(TSIM_ERR_PARSE, "DEPOLARIZE2 needs target pairs");
        for (size_t k = 0; k + 1 < in.t.size(); k += 2)
          add(in.op, in.t[k].v, in.t[k + 1].v, 4, pc2(std::vector<double>(15, in.args[0] / 15.0)), (int)k);
        break;
      case Op::PAULI_CHANNEL_2:
        need_args(in, 15, "PAULI_CHANNEL_2");
        if (in.t.size() % 2) fail(TSIM_ERR_PARSE, "PAULI_CHANNEL_2 needs target pairs");
        for (size_t k = 0; k + 1 < in.t.size(); k += 2)
          add(in.op, in.t[k].v, in.t[k + 1].v, 4, pc2(in.args), (int)k);
        break;
      case Op::DETECTOR: {
        std::vector<int> d;
        for (const Target& t : in.t) {
          if (!t.rec) fail(TSIM_ERR_PARSE, "DETECTOR takes rec targets");
          int j = nmeas + t.v;
          if (j < 0) fail(TSIM_ERR_PARSE, "DETECTOR refers before the first measurement");
          d.push_back(j);
        }
        c.detectors.push_back(d);
        break;
      }
      case Op::OBSERVABLE_INCLUDE: {
        if (in.args.size() != 1 || in.args[0] < 0) fail(TSIM_ERR_PARSE, "OBSERVABLE_INCLUDE(k) expected");
        size_t k = (size_t)in.args[0];
        if (c.observables.size() <= k) c.observables.resize(k + 1);
        for (const Target& t : in.t) {
          if (!t.rec) fail(TSIM_ERR_PARSE, "OBSERVABLE_INCLUDE takes rec targets");
          int j = nmeas + t.v;
          if (j < 0) fail(TSIM_ERR_PARSE, "OBSERVABLE_INCLUDE refers before the first measurement");
          c.observables[k].push_back(j);
        }
        break;
      }
      case Op::CX: case Op::CY: case Op::CZ: case Op::SWAP:
        if (in.t.size() % 2) fail(TSIM_ERR_PARSE, "two-qubit gate needs target pairs");
        for (size_t k = 0; k + 1 < in.t.size(); k += 2) {
          if (in.t[k + 1].rec) fail(TSIM_ERR_PARSE, "rec target must be the control");
          if (in.t[k].rec) {
            if (in.op == Op::SWAP) fail(TSIM_ERR_PARSE, "SWAP cannot take rec targets");
            if (nmeas + in.t[k].v < 0) fail(TSIM_ERR_PARSE, "rec refers before the first measurement");
          } else if (in.t[k].v == in.t[k + 1].v) {
            fail(TSIM_ERR_PARSE, "two-qubit gate on one qubit");
          }
        }
        break;
      case Op::R_X: case Op::R_Y: case Op::R_Z: case Op::U3: {
        const size_t na = in.op == Op::U3 ? 3 : 1;
        if (in.args.size() != na) fail(TSIM_ERR_PARSE, "rotation: wrong number of angles (units of pi)");
        for (double a : in.args)
          if (!std::isfinite(a)) fail(TSIM_ERR_PARSE, "rotation angle is not finite");
        for (const Target& t : in.t)
          if (t.rec) fail(TSIM_ERR_PARSE, "unexpected rec target");
        break;
      }
      default:
        for (const Target& t : in.t)
          if (t.rec) fail(TSIM_ERR_PARSE, "unexpected rec target");
        break;
    }
  }
  c.ins = std::move(flat);
  c.num_measurements = nmeas;
  c.num_error_bits = bit;
  return c;
}

}  // namespace tsim
