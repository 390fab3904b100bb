// Circuit text -> flat operation list (noisy circuit model of Sec. 2).
//
// Stim-like grammar (see include/symft.h).  REPEAT blocks are unrolled; every
// measurement event (recorded or the hidden one inside a reset) gets an
// ordinal t in circuit order and every noise location a channel ordinal, which
// key the random streams.  Resets are a hidden Pauli measurement followed by
// record-controlled Pauli feedback, both inside the paper's model (Sec. 2).
#include <cctype>
#include <cmath>
#include <cstdlib>
#include <sstream>
#include <unordered_map>

#include "internal.hpp"

namespace symft {
namespace {

struct Line {
  std::string name;
  std::vector<double> args;
  std::vector<std::string> targets;
  bool has_args = false;
  int lineno = 0;
};

[[noreturn]] void fail(int lineno, const std::string& msg) {
  throw Error(SYMFT_E_PARSE, "line " + std::to_string(lineno) + ": " + msg);
}

bool all_digits(const std::string& s) {
  if (s.empty() || s.size() > 9) return false;
  for (char ch : s)
    if (!std::isdigit(static_cast<unsigned char>(ch))) return false;
  return true;
}

class Parser {
 public:
  explicit Parser(Circuit& c) : c_(c) {}

  void run(const std::vector<Line>& lines, size_t lo, size_t hi) {
    size_t i = lo;
    while (i < hi) {
      const Line& L = lines[i];
      if (L.name == "}") fail(L.lineno, "unmatched }");
      if (L.name == "REPEAT") {
        if (L.targets.size() != 2 || L.targets[1] != "{" || !all_digits(L.targets[0]))
          fail(L.lineno, "malformed REPEAT");
        long n = std::strtol(L.targets[0].c_str(), nullptr, 10);
        size_t j = i + 1;
        int depth = 1;
        for (; j < hi; ++j) {
          if (lines[j].name == "REPEAT") ++depth;
          else if (lines[j].name == "}" && --depth == 0) break;
        }
        if (j >= hi) fail(L.lineno, "unterminated REPEAT");
        for (long r = 0; r < n; ++r) run(lines, i + 1, j);
        i = j + 1;
        continue;
      }
      instr(L);
      ++i;
    }
  }

 private:
  Circuit& c_;
  uint32_t max_q_ = 0;
  bool any_q_ = false;

  uint32_t qubit(const Line& L, const std::string& tok) {
    if (!all_digits(tok)) fail(L.lineno, "bad qubit target '" + tok + "'");
    uint32_t q = static_cast<uint32_t>(std::strtoul(tok.c_str(), nullptr, 10));
    if (q > 100000) fail(L.lineno, "qubit index too large");
    note(q);
    return q;
  }
  void note(uint32_t q) {
    if (!any_q_ || q > max_q_) max_q_ = q;
    any_q_ = true;
    c_.n_qubits = max_q_ + 1;
  }
  uint32_t rec_ordinal(const Line& L, const std::string& tok) {
    if (tok.size() < 7 || tok.compare(0, 5, "rec[-") != 0 || tok.back() != ']')
      fail(L.lineno, "bad record target '" + tok + "'");
    std::string num = tok.substr(5, tok.size() - 6);
    if (!all_digits(num)) fail(L.lineno, "bad record target '" + tok + "'");
    long k = std::strtol(num.c_str(), nullptr, 10);
    if (k < 1 || static_cast<uint64_t>(k) > c_.n_records) fail(L.lineno, "record " + tok + " out of range");
    return c_.record_ordinal[c_.n_records - k];
  }
  std::vector<PauliTerm> product(const Line& L, const std::string& tok) {
    std::vector<PauliTerm> out;
    size_t p = 0;
    while (p <= tok.size()) {
      size_t e = tok.find('*', p);
      if (e == std::string::npos) e = tok.size();
      std::string part = tok.substr(p, e - p);
      if (part.size() < 2 || (part[0] != 'X' && part[0] != 'Y' && part[0] != 'Z'))
        fail(L.lineno, "bad Pauli product '" + tok + "'");
      uint32_t q = qubit(L, part.substr(1));
      for (auto& t : out)
        if (t.q == q) fail(L.lineno, "repeated qubit in product '" + tok + "'");
      out.push_back({q, part[0]});
      p = e + 1;
    }
    return out;
  }
  uint32_t meas(std::vector<PauliTerm> p, bool recorded) {
    Op op;
    op.kind = OP_MEAS;
    op.pauli = std::move(p);
    op.t = c_.n_meas++;
    if (recorded) {
      op.rec = static_cast<int32_t>(c_.n_records++);
      c_.record_ordinal.push_back(op.t);
    }
    c_.ops.push_back(std::move(op));
    return c_.n_meas - 1;
  }
  void feedback(uint32_t q, char p, uint32_t t) {
    Op op;
    op.kind = OP_FB;
    op.pauli = {{q, p}};
    op.conds = {t};
    c_.ops.push_back(std::move(op));
  }
  void noise(int chan, double q, std::vector<double> w, uint32_t a, uint32_t b) {
    Op op;
    op.kind = OP_NOISE;
    op.chan = chan;
    op.q = q;
    op.weights = std::move(w);
    op.q0 = a;
    op.q1 = b;
    op.channel = c_.n_channels++;
    c_.ops.push_back(std::move(op));
  }
  void need_args(const Line& L, size_t n) {
    if (L.args.size() != n) fail(L.lineno, L.name + " expects " + std::to_string(n) + " argument(s)");
  }
  void check_prob(const Line& L, double p) {
    if (!(p >= 0.0 && p <= 1.0)) fail(L.lineno, "probability out of range");
  }

  void instr(const Line& L) {
    static const std::unordered_map<std::string, int> one_q = {
        {"I", G_I}, {"H", G_H}, {"S", G_S}, {"S_DAG", G_S_DAG}, {"SQRT_X", G_SQRT_X},
        {"SQRT_X_DAG", G_SQRT_X_DAG}, {"X", G_X}, {"Y", G_Y}, {"Z", G_Z}};
    static const std::unordered_map<std::string, int> two_q = {
        {"CX", G_CX}, {"CNOT", G_CX}, {"CY", G_CY}, {"CZ", G_CZ}, {"SWAP", G_SWAP}};
    const std::string& n = L.name;
    if (n == "TICK" || n == "QUBIT_COORDS" || n == "SHIFT_COORDS") return;
    auto it1 = one_q.find(n);
    if (it1 != one_q.end()) {
      need_args(L, 0);
      for (auto& t : L.targets) {
        Op op;
        op.kind = OP_CLIFF;
        op.gate = it1->second;
        op.q0 = qubit(L, t);
        c_.ops.push_back(op);
      }
      return;
    }
    auto it2 = two_q.find(n);
    if (it2 != two_q.end()) {
      need_args(L, 0);
      if (L.targets.size() % 2) fail(L.lineno, n + " needs target pairs");
      for (size_t i = 0; i < L.targets.size(); i += 2) {
        const std::string &a = L.targets[i], &b = L.targets[i + 1];
        bool ar = a.rfind("rec", 0) == 0, br = b.rfind("rec", 0) == 0;
        if (ar && br) fail(L.lineno, "feedback between two records");
        if (ar || br) {
          int g = it2->second;
          if (g == G_SWAP) fail(L.lineno, "SWAP cannot be record-controlled");
          if (br && g != G_CZ) fail(L.lineno, n + " target cannot be a record");
          uint32_t t = rec_ordinal(L, ar ? a : b);
          uint32_t q = qubit(L, ar ? b : a);
          feedback(q, g == G_CX ? 'X' : (g == G_CY ? 'Y' : 'Z'), t);
          continue;
        }
        Op op;
        op.kind = OP_CLIFF;
        op.gate = it2->second;
        op.q0 = qubit(L, a);
        op.q1 = qubit(L, b);
        if (op.q0 == op.q1) fail(L.lineno, n + " on identical qubits");
        c_.ops.push_back(op);
      }
      return;
    }
    if (n == "R_X" || n == "R_Y" || n == "R_Z" || n == "T" || n == "T_DAG") {
      double theta;
      char axis = 'Z';
      if (n == "T" || n == "T_DAG") {
        need_args(L, 0);
        theta = (n == "T" ? 1.0 : -1.0) * (M_PI / 4.0);
      } else {
        need_args(L, 1);
        theta = L.args[0];
        axis = n[2];
      }
      for (auto& t : L.targets) {
        Op op;
        op.kind = OP_ROT;
        op.pauli = {{qubit(L, t), axis}};
        op.theta = theta;
        c_.ops.push_back(std::move(op));
      }
      return;
    }
    if (n == "R_PAULI") {
      need_args(L, 1);
      for (auto& t : L.targets) {
        Op op;
        op.kind = OP_ROT;
        op.pauli = product(L, t);
        op.theta = L.args[0];
        c_.ops.push_back(std::move(op));
      }
      return;
    }
    if (n == "M" || n == "MX" || n == "MY" || n == "MR" || n == "MRX" || n == "R" || n == "RX") {
      need_args(L, 0);
      char axis = (n == "MX" || n == "MRX" || n == "RX") ? 'X' : (n == "MY" ? 'Y' : 'Z');
      bool recorded = !(n == "R" || n == "RX");
      bool reset = (n == "MR" || n == "MRX" || n == "R" || n == "RX");
      for (auto& t : L.targets) {
        uint32_t q = qubit(L, t);
        uint32_t ord = meas({{q, axis}}, recorded);
        if (reset) feedback(q, axis == 'Z' ? 'X' : 'Z', ord);
      }
      return;
    }
    if (n == "MPP") {
      need_args(L, 0);
      for (auto& t : L.targets) meas(product(L, t), true);
      return;
    }
    if (n == "X_ERROR" || n == "Y_ERROR" || n == "Z_ERROR" || n == "DEPOLARIZE1" ||
        n == "PAULI_CHANNEL_1") {
      double qtot;
      std::vector<double> w;
      int chan;
      if (n == "PAULI_CHANNEL_1") {
        need_args(L, 3);
        for (double v : L.args) check_prob(L, v);
        qtot = (L.args[0] + L.args[1]) + L.args[2];
        w = {L.args[0], L.args[1], L.args[2]};
        chan = CH_XYZ;
      } else {
        need_args(L, 1);
        qtot = L.args[0];
        if (n == "DEPOLARIZE1") {
          w = {1.0, 1.0, 1.0};
          chan = CH_XYZ;
        } else {
          w = {1.0};
          chan = n[0] == 'X' ? CH_X : (n[0] == 'Y' ? CH_Y : CH_Z);
        }
      }
      check_prob(L, qtot);
      for (auto& t : L.targets) {
        uint32_t q = qubit(L, t);
        noise(chan, qtot, w, q, q);
      }
      return;
    }
    if (n == "DEPOLARIZE2") {
      need_args(L, 1);
      check_prob(L, L.args[0]);
      if (L.targets.size() % 2) fail(L.lineno, "DEPOLARIZE2 needs target pairs");
      for (size_t i = 0; i < L.targets.size(); i += 2) {
        uint32_t a = qubit(L, L.targets[i]), b = qubit(L, L.targets[i + 1]);
        if (a == b) fail(L.lineno, "DEPOLARIZE2 on identical qubits");
        noise(CH_D2, L.args[0], std::vector<double>(15, 1.0), a, b);
      }
      return;
    }
    if (n == "DETECTOR" || n == "OBSERVABLE_INCLUDE") {
      Op op;
      op.kind = n == "DETECTOR" ? OP_DET : OP_OBS;
      for (auto& t : L.targets) op.conds.push_back(rec_ordinal(L, t));
      if (op.kind == OP_DET) {
        op.index = c_.n_dets++;
      } else {
        need_args(L, 1);
        double k = L.args[0];
        if (!(k >= 0 && k < 1e6 && k == std::floor(k))) fail(L.lineno, "bad observable index");
        op.index = static_cast<uint32_t>(k);
        if (op.index + 1 > c_.n_obs) c_.n_obs = op.index + 1;
      }
      c_.ops.push_back(std::move(op));
      return;
    }
    throw Error(SYMFT_E_UNSUPPORTED, "line " + std::to_string(L.lineno) + ": unsupported instruction '" + n + "'");
  }
};

std::vector<Line> lex(const std::string& text) {
  std::vector<Line> out;
  std::istringstream in(text);
  std::string raw;
  int lineno = 0;
  while (std::getline(in, raw)) {
    ++lineno;
    size_t hash = raw.find('#');
    if (hash != std::string::npos) raw.resize(hash);
    std::istringstream ls(raw);
    std::string head;
    if (!(ls >> head)) continue;
    Line L;
    L.lineno = lineno;
    size_t par = head.find('(');
    if (par == std::string::npos) {
      L.name = head;
    } else {
      // arguments may contain spaces: gather up to ')'
      std::string rest = head.substr(par + 1);
      while (rest.find(')') == std::string::npos) {
        std::string more;
        if (!(ls >> more)) fail(lineno, "unterminated argument list");
        rest += more;
      }
      size_t close = rest.find(')');
      std::string after = rest.substr(close + 1);
      if (!after.empty()) fail(lineno, "junk after argument list");
      L.name = head.substr(0, par);
      L.has_args = true;
      std::string args = rest.substr(0, close);
      size_t p = 0;
      while (p < args.size()) {
        size_t e = args.find(',', p);
        if (e == std::string::npos) e = args.size();
        std::string a = args.substr(p, e - p);
        char* end = nullptr;
        double v = std::strtod(a.c_str(), &end);
        if (a.empty() || end == a.c_str() || *end != '\0') fail(lineno, "bad argument '" + a + "'");
        L.args.push_back(v);
        p = e + 1;
      }
    }
    for (char ch : L.name)
      if (!(std::isupper(static_cast<unsigned char>(ch)) || std::isdigit(static_cast<unsigned char>(ch)) ||
            ch == '_' || ch == '}'))
        fail(lineno, "bad instruction name '" + L.name + "'");
    std::string tok;
    while (ls >> tok) L.targets.push_back(tok);
    out.push_back(std::move(L));
  }
  return out;
}

}  // namespace

Circuit parse_circuit(const std::string& text) {
  Circuit c;
  std::vector<Line> lines = lex(text);
  Parser p(c);
  p.run(lines, 0, lines.size());
  return c;
}

}  // namespace symft
