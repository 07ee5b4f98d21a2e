// Mechanism parser and validator (host side of libpyro).
#include "pyro_mech.h"

#include <cerrno>
#include <cmath>
#include <cstdlib>
#include <fstream>
#include <sstream>

namespace pyro {

namespace {

// Whitespace tokenizer over one line.
struct Line {
  std::vector<std::string> tok;
  size_t pos = 0;
  bool done() const { return pos >= tok.size(); }
  bool word(std::string& s) { if (done()) return false; s = tok[pos++]; return true; }
  bool integer(int& v) {
    std::string s; if (!word(s)) return false;
    char* e = nullptr; errno = 0; long x = std::strtol(s.c_str(), &e, 10);
    if (*e != '\0' || errno) return false;
    v = (int)x; return true;
  }
  bool real(double& v) {
    std::string s; if (!word(s)) return false;
    char* e = nullptr; errno = 0; v = std::strtod(s.c_str(), &e);
    return *e == '\0' && errno == 0;
  }
  bool is_number_next() const {
    if (done()) return false;
    const std::string& s = tok[pos];
    char* e = nullptr; std::strtod(s.c_str(), &e);
    return *e == '\0' && e != s.c_str();
  }
};

bool read_lines(const std::string& path, std::vector<Line>& out, std::string& err) {
  std::ifstream f(path);
  if (!f) { err = "cannot open mechanism file '" + path + "'"; return false; }
  std::string s;
  while (std::getline(f, s)) {
    if (s.empty() || s[0] == '#') continue;
    std::istringstream is(s);
    Line ln; std::string t;
    while (is >> t) ln.tok.push_back(t);
    if (!ln.tok.empty()) out.push_back(ln);
  }
  return true;
}

}  // namespace

bool parse_mechanism_file(const std::string& path, Mechanism& m, std::string& err) {
  std::vector<Line> L;
  if (!read_lines(path, L, err)) return false;
  size_t li = 0;
  auto fail = [&](const std::string& what) {
    err = "mechanism '" + path + "' line " + std::to_string(li) + ": " + what;
    return false;
  };
  auto expect = [&](const char* key, int& count) -> bool {
    if (li >= L.size()) return false;
    std::string k;
    return L[li].word(k) && k == key && L[li].integer(count) && (li++, true);
  };
  int ver = 0;
  if (!expect("pyro-mech", ver) || ver != 1) return fail("expected header 'pyro-mech 1'");
  if (li >= L.size() || L[li].tok[0] != "name") return fail("expected 'name'");
  for (size_t i = 1; i < L[li].tok.size(); ++i) m.name += (i > 1 ? " " : "") + L[li].tok[i];
  ++li;
  int ne = 0;
  if (!expect("elements", ne) || ne <= 0) return fail("expected 'elements <n>'");
  for (int i = 0; i < ne; ++i, ++li) {
    if (li >= L.size()) return fail("missing element line");
    std::string k, sym; double w;
    if (!L[li].word(k) || k != "element" || !L[li].word(sym) || !L[li].real(w) || !(w > 0))
      return fail("bad element line");
    m.element_names.push_back(sym);
    m.element_weights.push_back(w);
  }
  int ns = 0;
  if (!expect("species", ns) || ns <= 0) return fail("expected 'species <n>'");
  m.species.resize(ns);
  for (int k = 0; k < ns; ++k, ++li) {
    if (li >= L.size()) return fail("missing species line");
    std::string key; int nc;
    Species& s = m.species[k];
    if (!L[li].word(key) || key != "species" || !L[li].word(s.name) || !L[li].integer(nc) || nc <= 0)
      return fail("bad species line");
    for (int c = 0; c < nc; ++c) {
      std::string e; int cnt;
      if (!L[li].word(e) || !L[li].integer(cnt) || cnt <= 0) return fail("bad composition");
      int ei = -1;
      for (int q = 0; q < ne; ++q) if (m.element_names[q] == e) ei = q;
      if (ei < 0) return fail("unknown element '" + e + "'");
      s.composition.push_back({ei, cnt});
      s.W += cnt * m.element_weights[ei];
    }
  }
  std::vector<bool> seen(ns, false);
  for (int k = 0; k < ns; ++k, ++li) {
    if (li >= L.size()) return fail("missing thermo line");
    std::string key; int idx;
    if (!L[li].word(key) || key != "thermo" || !L[li].integer(idx) || idx < 0 || idx >= ns || seen[idx])
      return fail("bad thermo line");
    seen[idx] = true;
    Species& s = m.species[idx];
    bool ok = L[li].real(s.t_low) && L[li].real(s.t_mid) && L[li].real(s.t_high);
    for (int i = 0; i < 7 && ok; ++i) ok = L[li].real(s.low[i]);
    for (int i = 0; i < 7 && ok; ++i) ok = L[li].real(s.high[i]);
    if (!ok || !L[li].done()) return fail("bad thermo coefficients");
  }
  int nr = 0;
  if (!expect("reactions", nr) || nr < 0) return fail("expected 'reactions <n>'");
  m.reactions.resize(nr);
  for (int j = 0; j < nr; ++j, ++li) {
    if (li >= L.size()) return fail("missing reaction line");
    Line& ln = L[li];
    Reaction& r = m.reactions[j];
    std::string key, kind;
    if (!ln.word(key) || key != "reaction" || !ln.word(kind)) return fail("bad reaction line");
    if (kind == "arrhenius") r.kind = RX_ARRHENIUS;
    else if (kind == "threebody") r.kind = RX_THREEBODY;
    else if (kind == "falloff") r.kind = RX_FALLOFF;
    else if (kind == "plog") r.kind = RX_PLOG;
    else return fail("unknown reaction kind '" + kind + "'");
    bool has_arr = false, ended = false;
    std::string tok;
    while (ln.word(tok)) {
      if (tok == "end") { ended = true; break; }
      if (tok == "rev" || tok == "dup") {
        int v; if (!ln.integer(v)) return fail("bad flag");
        (tok == "rev" ? r.reversible : r.duplicate) = v != 0;
      } else if (tok == "reac" || tok == "prod") {
        int n; if (!ln.integer(n) || n <= 0) return fail("bad side count");
        for (int q = 0; q < n; ++q) {
          int k, nu;
          if (!ln.integer(k) || !ln.integer(nu) || k < 0 || k >= ns || nu <= 0)
            return fail("bad stoichiometry");
          (tok == "reac" ? r.reactants : r.products).push_back({k, nu});
        }
      } else if (tok == "arr") {
        if (!ln.real(r.A) || !ln.real(r.b) || !ln.real(r.theta)) return fail("bad Arrhenius data");
        has_arr = true;
      } else if (tok == "eff") {
        int n; if (!ln.integer(n) || n < 0) return fail("bad efficiency count");
        for (int q = 0; q < n; ++q) {
          int k; double e;
          if (!ln.integer(k) || !ln.real(e) || k < 0 || k >= ns || e < 0) return fail("bad efficiency");
          r.efficiencies.push_back({k, e});
        }
      } else if (tok == "low") {
        if (!ln.real(r.A0) || !ln.real(r.b0) || !ln.real(r.theta0)) return fail("bad low-pressure data");
        r.has_low = true;
      } else if (tok == "troe") {
        r.n_troe = 0;
        while (ln.is_number_next() && r.n_troe < 4) ln.real(r.troe[r.n_troe++]);
      } else if (tok == "sri") {
        r.n_sri = 0;
        while (ln.is_number_next() && r.n_sri < 5) ln.real(r.sri[r.n_sri++]);
      } else if (tok == "plog") {
        int n; if (!ln.integer(n) || n < 2) return fail("plog needs at least 2 nodes");
        r.plog.resize(n);
        for (auto& nd : r.plog)
          if (!ln.real(nd.p) || !ln.real(nd.A) || !ln.real(nd.b) || !ln.real(nd.theta)) return fail("bad plog node");
      } else {
        return fail("unknown reaction token '" + tok + "'");
      }
    }
    if (!ended) return fail("reaction line without 'end'");
    if (!has_arr && r.kind != RX_PLOG) return fail("reaction without 'arr'");
    if (r.kind == RX_PLOG && !has_arr) { r.A = r.plog[0].A; r.b = r.plog[0].b; r.theta = r.plog[0].theta; }
    if (r.reactants.empty() || r.products.empty()) return fail("reaction without reactants or products");
  }
  // optional transport section
  if (li < L.size()) {
    int nt = 0;
    if (!expect("transport", nt) || nt != ns) return fail("expected 'transport <n_species>' or end of file");
    TransportFits& tf = m.transport;
    tf.visc.assign((size_t)ns * 5, 0.0);
    tf.cond.assign((size_t)ns * 5, 0.0);
    tf.diff.assign((size_t)ns * ns * 5, 0.0);
    std::vector<bool> sp(ns, false);
    for (int q = 0; q < ns; ++q, ++li) {
      if (li >= L.size()) return fail("missing tspecies line");
      std::string key; int k;
      if (!L[li].word(key) || key != "tspecies" || !L[li].integer(k) || k < 0 || k >= ns || sp[k])
        return fail("bad tspecies line");
      sp[k] = true;
      bool ok = true;
      for (int i = 0; i < 5 && ok; ++i) ok = L[li].real(tf.visc[(size_t)k * 5 + i]);
      for (int i = 0; i < 5 && ok; ++i) ok = L[li].real(tf.cond[(size_t)k * 5 + i]);
      if (!ok || !L[li].done()) return fail("bad tspecies coefficients");
    }
    std::vector<bool> pr((size_t)ns * ns, false);
    const long long npairs = (long long)ns * (ns - 1) / 2;
    for (long long q = 0; q < npairs; ++q, ++li) {
      if (li >= L.size()) return fail("missing tbinary line");
      std::string key; int k, j;
      if (!L[li].word(key) || key != "tbinary" || !L[li].integer(k) || !L[li].integer(j) || k < 0 || j <= k ||
          j >= ns || pr[(size_t)k * ns + j])
        return fail("bad tbinary line");
      pr[(size_t)k * ns + j] = true;
      bool ok = true;
      for (int i = 0; i < 5 && ok; ++i) {
        double a;
        ok = L[li].real(a);
        tf.diff[((size_t)k * ns + j) * 5 + i] = tf.diff[((size_t)j * ns + k) * 5 + i] = a;
      }
      if (!ok || !L[li].done()) return fail("bad tbinary coefficients");
    }
    if (li < L.size()) return fail("unexpected content after the transport section");
    m.has_transport = true;
  }
  return true;
}

bool validate_mechanism(const Mechanism& m, std::string& err) {
  int ns = m.n_species(), ne = (int)m.element_names.size();
  for (int k = 0; k < ns; ++k) {
    const Species& s = m.species[k];
    if (!(s.W > 0)) { err = "species " + s.name + ": non-positive molecular weight"; return false; }
    if (!(s.t_low < s.t_mid && s.t_mid < s.t_high)) { err = "species " + s.name + ": bad NASA ranges"; return false; }
    // cp/R > 1 on the fitted ranges keeps c_v > 0, so e(T) is strictly increasing
    for (int i = 0; i <= 64; ++i) {
      double T = s.t_low + (s.t_high - s.t_low) * i / 64.0;
      const double* a = T < s.t_mid ? s.low : s.high;
      double cp = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
      if (!(cp > 1.0)) {
        err = "species " + s.name + ": cp/R <= 1 at T = " + std::to_string(T) + " K";
        return false;
      }
    }
  }
  for (int j = 0; j < m.n_reactions(); ++j) {
    const Reaction& r = m.reactions[j];
    std::string tag = "reaction " + std::to_string(j) + ": ";
    if (!(r.A > 0) || !std::isfinite(r.b) || !std::isfinite(r.theta)) { err = tag + "bad Arrhenius data"; return false; }
    std::vector<long> bal(ne, 0);
    for (auto& p : r.reactants) for (auto& c : m.species[p.first].composition) bal[c.first] -= (long)p.second * c.second;
    for (auto& p : r.products) for (auto& c : m.species[p.first].composition) bal[c.first] += (long)p.second * c.second;
    for (int e = 0; e < ne; ++e)
      if (bal[e] != 0) { err = tag + "not element-balanced in " + m.element_names[e]; return false; }
    if (r.kind == RX_FALLOFF) {
      if (!r.has_low || !(r.A0 > 0)) { err = tag + "falloff reaction without low-pressure limit"; return false; }
      if (r.n_troe != 0 && r.n_troe != 3 && r.n_troe != 4) { err = tag + "Troe needs 3 or 4 parameters"; return false; }
      if (r.n_troe >= 3 && !(r.troe[1] > 0 && r.troe[2] > 0)) { err = tag + "Troe T3, T1 must be positive"; return false; }
      if (r.n_sri != 0 && r.n_sri != 3 && r.n_sri != 5) { err = tag + "SRI needs 3 or 5 parameters"; return false; }
      if (r.n_sri && r.n_troe) { err = tag + "both Troe and SRI data"; return false; }
      if (r.n_sri && !(r.sri[0] >= 0 && r.sri[1] >= 0 && r.sri[2] > 0 && r.sri[3] > 0 && std::isfinite(r.sri[4]))) {
        err = tag + "SRI needs a >= 0, b >= 0, c > 0, d > 0"; return false;
      }
    } else if (r.has_low || r.n_troe || r.n_sri) {
      err = tag + "low/troe/sri data on a non-falloff reaction"; return false;
    }
    if (r.kind == RX_PLOG) {
      for (size_t q = 0; q < r.plog.size(); ++q) {
        const PlogNode& nd = r.plog[q];
        if (!(nd.p > 0) || !(nd.A > 0) || !std::isfinite(nd.b) || !std::isfinite(nd.theta) ||
            (q > 0 && !(nd.p > r.plog[q - 1].p))) {
          err = tag + "plog nodes need p > 0 increasing and A > 0"; return false;
        }
      }
      if (!r.efficiencies.empty()) { err = tag + "efficiencies on a plog reaction"; return false; }
    } else if (!r.plog.empty()) {
      err = tag + "plog data on a non-plog reaction"; return false;
    }
    if (r.kind == RX_ARRHENIUS && !r.efficiencies.empty()) { err = tag + "efficiencies on a plain reaction"; return false; }
    int order_r = 0;
    for (auto& p : r.reactants) order_r += p.second;
    if (order_r > 6) { err = tag + "reaction order above 6"; return false; }
  }
  return true;
}

}  // namespace pyro
