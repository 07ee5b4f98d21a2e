// CPU oracle for pointwise combustion thermochemistry — TEST INFRASTRUCTURE.
//
// This file is the plain, slow, obviously correct reference for the GPU library.
// Only the test suite, the smoke check and the CPU-baseline leg of the benchmark
// may load it; the library never does, and nothing here is shared with it
// (its own mechanism parser, its own formulas, no common headers).
//
// Every quantity is the direct definition from the paper's formulation
// appendix (Sec. A), evaluated literally: powers by std::pow, exponentials by
// std::exp, products and sums by loops over species and reactions.  The code is
// templated on the scalar type so that the same definitions run in
//   double                -- the oracle proper,
//   long double           -- a rounding-error envelope for the oracle itself,
//   Dual (below)          -- forward-mode derivatives (Jacobian, JVP, VJP, gross
//                            scales): value and first derivative carried together,
//                            exact up to rounding, with no step size -- automatic
//                            differentiation through a scalar type with redefined
//                            operations, as the paper obtains Eq. rate_gradient.  (A complex
//                            step h is exact only to O(h^2 f'''/f'): where a
//                            variable is far below h -- mass fractions of 1e-75 at
//                            equilibrium states -- that term dominates.)
//
// Readings of passages that the paper leaves silent, ambiguous or garbled are
// marked "reading (cN)"; each states the interpretation taken and why.
//
// Units: SI with kmol.  R = 8314.462618 J/(kmol K), p0 = 1 atm = 101325 Pa.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// math functions by unqualified name: the std overloads for double, long double and
// std::complex, and (found by argument-dependent lookup) those of Dual
using std::exp;
using std::log;
using std::log10;
using std::pow;
using std::sqrt;

const double R_GAS = 8314.462618;   // J/(kmol K)
const double P_ATM = 101325.0;      // Pa

// ---------------------------------------------------------------------------
// Mechanism (own parser of the text interchange format)
// ---------------------------------------------------------------------------

struct OSpecies {
  std::string name;
  std::vector<std::pair<int, int>> comp;   // (element index, count)
  double W = 0;                            // kg/kmol
  double t_low = 0, t_mid = 0, t_high = 0;
  double lo[7] = {0}, hi[7] = {0};
};

enum { K_ARRHENIUS = 0, K_THREEBODY = 1, K_FALLOFF = 2, K_PLOG = 3 };

struct OReaction {
  int kind = K_ARRHENIUS;
  bool reversible = true, duplicate = false;
  std::vector<std::pair<int, int>> reac, prod;   // (species, coefficient)
  double A = 0, b = 0, theta = 0;
  std::vector<std::pair<int, double>> eff;       // efficiencies (default 1)
  bool has_low = false;
  double A0 = 0, b0 = 0, theta0 = 0;
  int n_troe = 0;
  double troe[4] = {0, 0, 0, 0};
  int n_sri = 0;                                 // SRI falloff data (a, b, c[, d, e])
  double sri[5] = {0, 0, 0, 1, 0};
  std::vector<std::vector<double>> plog;         // PLOG nodes (p [Pa], A, b, theta), increasing p
};

struct OMech {
  std::vector<std::string> el_name;
  std::vector<double> el_weight;
  std::vector<OSpecies> sp;
  std::vector<OReaction> rx;
  // transport fits (Sec. A.2), coefficients of (log T)^m, m = 0..4; empty if absent
  std::vector<std::vector<double>> visc, cond;              // [N][5]
  std::vector<std::vector<std::vector<double>>> bdiff;      // [N][N][5], symmetric
  int N() const { return (int)sp.size(); }
  int M() const { return (int)rx.size(); }
};

thread_local std::string g_err;

bool parse_mech(const char* path, OMech& m) {
  std::ifstream f(path);
  if (!f) { g_err = std::string("cannot open ") + path; return false; }
  std::string line, key;
  std::vector<std::string> lines;
  while (std::getline(f, line)) {
    if (line.empty() || line[0] == '#') continue;
    lines.push_back(line);
  }
  size_t li = 0;
  auto next = [&](std::istringstream& is) -> bool {
    if (li >= lines.size()) return false;
    is.clear(); is.str(lines[li++]); return true;
  };
  std::istringstream is;
  if (!next(is)) { g_err = "empty file"; return false; }
  int ver = 0; is >> key >> ver;
  if (key != "pyro-mech" || ver != 1) { g_err = "bad header"; return false; }
  next(is);                                        // name
  int ne = 0; next(is); is >> key >> ne;
  for (int i = 0; i < ne; ++i) {
    next(is); std::string s; double w; is >> key >> s >> w;
    m.el_name.push_back(s); m.el_weight.push_back(w);
  }
  int ns = 0; next(is); is >> key >> ns;
  m.sp.resize(ns);
  for (int k = 0; k < ns; ++k) {
    next(is); int nc; is >> key >> m.sp[k].name >> nc;
    for (int c = 0; c < nc; ++c) {
      std::string e; int cnt; is >> e >> cnt;
      int ei = -1;
      for (int q = 0; q < ne; ++q) if (m.el_name[q] == e) ei = q;
      if (ei < 0) { g_err = "unknown element " + e; return false; }
      m.sp[k].comp.push_back({ei, cnt});
    }
  }
  for (int k = 0; k < ns; ++k) {
    next(is); int idx; is >> key >> idx;
    if (key != "thermo" || idx < 0 || idx >= ns) { g_err = "bad thermo line"; return false; }
    OSpecies& s = m.sp[idx];
    is >> s.t_low >> s.t_mid >> s.t_high;
    for (int i = 0; i < 7; ++i) is >> s.lo[i];
    for (int i = 0; i < 7; ++i) is >> s.hi[i];
    if (!is) { g_err = "short thermo line"; return false; }
  }
  // molecular weights from atomic weights (Sec. A.1: W_k of species k)
  for (auto& s : m.sp) {
    double W = 0;
    for (auto& c : s.comp) W += c.second * m.el_weight[c.first];
    s.W = W;
  }
  int nr = 0; next(is); is >> key >> nr;
  m.rx.resize(nr);
  for (int j = 0; j < nr; ++j) {
    next(is); OReaction& r = m.rx[j];
    std::string kind; is >> key >> kind;
    if (kind == "arrhenius") r.kind = K_ARRHENIUS;
    else if (kind == "threebody") r.kind = K_THREEBODY;
    else if (kind == "falloff") r.kind = K_FALLOFF;
    else if (kind == "plog") r.kind = K_PLOG;
    else { g_err = "unknown reaction kind " + kind; return false; }
    std::string tok;
    while (is >> tok && tok != "end") {
      if (tok == "rev") { int v; is >> v; r.reversible = v != 0; }
      else if (tok == "dup") { int v; is >> v; r.duplicate = v != 0; }
      else if (tok == "reac" || tok == "prod") {
        int n; is >> n;
        for (int q = 0; q < n; ++q) {
          int k, nu; is >> k >> nu;
          (tok == "reac" ? r.reac : r.prod).push_back({k, nu});
        }
      } else if (tok == "arr") { is >> r.A >> r.b >> r.theta; }
      else if (tok == "eff") {
        int n; is >> n;
        for (int q = 0; q < n; ++q) { int k; double e; is >> k >> e; r.eff.push_back({k, e}); }
      } else if (tok == "low") { r.has_low = true; is >> r.A0 >> r.b0 >> r.theta0; }
      else if (tok == "troe" || tok == "sri") {
        // 3 to 5 numbers follow; peek until a keyword
        int cnt = 0;
        double vals[5] = {0, 0, 0, 1, 0};
        std::streampos pos;
        while (true) {
          pos = is.tellg();
          std::string t2; if (!(is >> t2)) break;
          char* endp = nullptr;
          double v = std::strtod(t2.c_str(), &endp);
          if (endp == t2.c_str() || *endp != '\0') { is.seekg(pos); break; }
          if (cnt < 5) vals[cnt++] = v;
        }
        if (tok == "troe") { r.n_troe = std::min(cnt, 4); for (int i = 0; i < 4; ++i) r.troe[i] = vals[i]; }
        else { r.n_sri = cnt; for (int i = 0; i < 5; ++i) r.sri[i] = vals[i]; }
      } else if (tok == "plog") {
        int n; is >> n;
        for (int q = 0; q < n; ++q) {
          std::vector<double> node(4);
          for (int i = 0; i < 4; ++i) is >> node[i];
          r.plog.push_back(node);
        }
      } else { g_err = "unknown reaction token " + tok; return false; }
    }
    if (tok != "end") { g_err = "unterminated reaction"; return false; }
  }
  // optional transport section: per-species viscosity and conductivity fits,
  // then the binary diffusivity fit of every pair k < j
  if (next(is)) {
    int nt = 0; is >> key >> nt;
    if (key != "transport" || nt != ns) { g_err = "bad transport header"; return false; }
    m.visc.assign(ns, std::vector<double>(5, 0.0));
    m.cond.assign(ns, std::vector<double>(5, 0.0));
    m.bdiff.assign(ns, std::vector<std::vector<double>>(ns, std::vector<double>(5, 0.0)));
    for (int q = 0; q < ns; ++q) {
      if (!next(is)) { g_err = "short transport section"; return false; }
      int k; is >> key >> k;
      if (key != "tspecies" || k < 0 || k >= ns) { g_err = "bad tspecies line"; return false; }
      for (int i = 0; i < 5; ++i) is >> m.visc[k][i];
      for (int i = 0; i < 5; ++i) is >> m.cond[k][i];
      if (!is) { g_err = "short tspecies line"; return false; }
    }
    for (int q = 0; q < ns * (ns - 1) / 2; ++q) {
      if (!next(is)) { g_err = "short transport section"; return false; }
      int k, j; is >> key >> k >> j;
      if (key != "tbinary" || k < 0 || j < 0 || k >= ns || j >= ns || k == j) { g_err = "bad tbinary line"; return false; }
      for (int i = 0; i < 5; ++i) { is >> m.bdiff[k][j][i]; m.bdiff[j][k][i] = m.bdiff[k][j][i]; }
      if (!is) { g_err = "short tbinary line"; return false; }
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Scalar helpers (real part for comparisons, so derivative carriers pass through)
// ---------------------------------------------------------------------------

inline double re(double x) { return x; }
inline long double re(long double x) { return x; }
inline double re(const std::complex<double>& x) { return x.real(); }

// ---------------------------------------------------------------------------
// Dual numbers v + d eps with eps^2 = 0: every operation carries the value and its
// derivative along one direction (the chain rule of each elementary function), so
// a definition evaluated on Dual inputs with d = 1 in one variable returns that
// partial derivative exactly up to rounding.
// ---------------------------------------------------------------------------
namespace dualnum {
struct Dual {
  double v = 0.0, d = 0.0;
  Dual() {}
  Dual(double x) : v(x) {}
  Dual(double x, double dx) : v(x), d(dx) {}
  Dual& operator+=(const Dual& b) { v += b.v; d += b.d; return *this; }
  Dual& operator-=(const Dual& b) { v -= b.v; d -= b.d; return *this; }
  Dual& operator*=(const Dual& b) { d = d * b.v + v * b.d; v *= b.v; return *this; }
  Dual& operator/=(const Dual& b) { d = (d * b.v - v * b.d) / (b.v * b.v); v /= b.v; return *this; }
};
inline Dual operator+(Dual a, const Dual& b) { return a += b; }
inline Dual operator-(Dual a, const Dual& b) { return a -= b; }
inline Dual operator*(Dual a, const Dual& b) { return a *= b; }
inline Dual operator/(Dual a, const Dual& b) { return a /= b; }
inline Dual operator+(Dual a, double b) { a.v += b; return a; }
inline Dual operator+(double a, Dual b) { b.v += a; return b; }
inline Dual operator-(Dual a, double b) { a.v -= b; return a; }
inline Dual operator-(double a, const Dual& b) { return Dual(a - b.v, -b.d); }
inline Dual operator*(const Dual& a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator*(double a, const Dual& b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(const Dual& a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator/(double a, const Dual& b) { return Dual(a / b.v, -a * b.d / (b.v * b.v)); }
inline Dual operator-(const Dual& a) { return Dual(-a.v, -a.d); }
inline Dual exp(const Dual& a) { const double e = std::exp(a.v); return Dual(e, a.d * e); }
inline Dual log(const Dual& a) { return Dual(std::log(a.v), a.d / a.v); }
inline Dual log10(const Dual& a) { return Dual(std::log10(a.v), a.d / (a.v * std::log(10.0))); }
inline Dual sqrt(const Dual& a) { const double r = std::sqrt(a.v); return Dual(r, a.d / (2.0 * r)); }
// x^p, constant p: d(x^p) = p x^(p-1) dx (x^0 = 1 with derivative 0)
inline Dual pow(const Dual& a, double p) {
  if (p == 0.0) return Dual(1.0, 0.0);
  return Dual(std::pow(a.v, p), p * std::pow(a.v, p - 1.0) * a.d);
}
// x^y for x > 0: exp(y ln x)
inline Dual pow(const Dual& a, const Dual& b) { return exp(b * log(a)); }
}  // namespace dualnum
using dualnum::Dual;
inline double re(const Dual& x) { return x.v; }

// ---------------------------------------------------------------------------
// Thermodynamics: NASA-7 polynomials (Sec. A.1, Eq. nasa_poly, Eq. nasa_poly_c)
// ---------------------------------------------------------------------------

inline const double* nasa_coeffs(const OSpecies& s, double T) {
  // reading (c6): low range if T < T_mid, else high range; no clamping
  return T < s.t_mid ? s.lo : s.hi;
}

// cp/R = sum_{m=1}^{5} a_m T^{m-1}      (Eq. nasa_poly_c, reading (c3))
template <class S> S cp_R(const OSpecies& s, S T) {
  const double* a = nasa_coeffs(s, re(T));
  S v = 0;
  for (int m = 1; m <= 5; ++m) v += a[m - 1] * pow(T, (double)(m - 1));
  return v;
}

// h/(R T) = a6/T + sum_{m=1}^{5} a_m T^{m-1}/m     (Eq. nasa_poly, first line; reading (c4))
template <class S> S h_RT(const OSpecies& s, S T) {
  const double* a = nasa_coeffs(s, re(T));
  S v = a[5] / T;
  for (int m = 1; m <= 5; ++m) v += a[m - 1] * pow(T, (double)(m - 1)) / (double)m;
  return v;
}

// s/R = a1 ln T + sum_{m=2}^{5} a_m T^{m-1}/(m-1) + a7    (Eq. nasa_poly, second line; reading (c2))
template <class S> S s_R(const OSpecies& s, S T) {
  const double* a = nasa_coeffs(s, re(T));
  S v = a[0] * log(T) + a[6];
  for (int m = 2; m <= 5; ++m) v += a[m - 1] * pow(T, (double)(m - 1)) / (double)(m - 1);
  return v;
}

// g/(R T) = h/(R T) - s/R     (Eq. gibbs)
template <class S> S g_RT(const OSpecies& s, S T) { return h_RT(s, T) - s_R(s, T); }

// ---------------------------------------------------------------------------
// Mixture relations (Sec. A.1 Eq. eos; Sec. A.3.1 Eq. int_energy, Eq. cv)
// ---------------------------------------------------------------------------

// W = (sum Y_i/W_i)^{-1};  rho = p W / (R T)      (Eq. eos)
template <class S> S density(const OMech& m, S p, S T, const S* Y) {
  S inv = 0;
  for (int k = 0; k < m.N(); ++k) inv += Y[k] / m.sp[k].W;
  return p / (R_GAS * T * inv);
}

// e = sum_k Y_k (h_k - R T)/W_k          (Eq. int_energy)
template <class S> S internal_energy(const OMech& m, S T, const S* Y) {
  S e = 0;
  for (int k = 0; k < m.N(); ++k) {
    S hk = R_GAS * T * h_RT(m.sp[k], T);
    e += Y[k] * (hk - R_GAS * T) / m.sp[k].W;
  }
  return e;
}

// c_v = sum_k Y_k (cp_k - R)/W_k = de/dT      (Eq. cv, reading (c5): per-mass form)
template <class S> S cv_mass(const OMech& m, S T, const S* Y) {
  S c = 0;
  for (int k = 0; k < m.N(); ++k) c += Y[k] * (R_GAS * cp_R(m.sp[k], T) - R_GAS) / m.sp[k].W;
  return c;
}

// h = sum_k Y_k h_k / W_k: mixture enthalpy per unit mass (Sec. A.3.1, the
// enthalpy variant of the temperature inversion)
template <class S> S enthalpy_mass(const OMech& m, S T, const S* Y) {
  S h = 0;
  for (int k = 0; k < m.N(); ++k) h += Y[k] * (R_GAS * T * h_RT(m.sp[k], T)) / m.sp[k].W;
  return h;
}

// c_p = sum_k Y_k cp_k / W_k = dh/dT
template <class S> S cp_mass(const OMech& m, S T, const S* Y) {
  S c = 0;
  for (int k = 0; k < m.N(); ++k) c += Y[k] * (R_GAS * cp_R(m.sp[k], T)) / m.sp[k].W;
  return c;
}

// the quantity the inversion matches (e or h) and its temperature derivative (c_v or c_p)
double mixture_caloric(const OMech& m, double T, const double* Y, bool enthalpy) {
  return enthalpy ? enthalpy_mass(m, T, Y) : internal_energy(m, T, Y);
}
double mixture_heat_capacity(const OMech& m, double T, const double* Y, bool enthalpy) {
  return enthalpy ? cp_mass(m, T, Y) : cv_mass(m, T, Y);
}

// Newton iteration for T(e, Y)       (Sec. A.3.1, Eq. delta_temp)
//   T_{m+1} = T_m - (Y.e(T_m) - e) / c_v(T_m)
// reading (c7): stop once |dT| <= tol*T_{m+1}, then take one more step;
// reading (c6): iterates clamped to [100, 5000] K.  Returns iterations used,
// or -1 if max_iter was reached without meeting the stop rule.
// The enthalpy variant (enthalpy = true) is the same iteration on h with c_p.
int temperature_newton(const OMech& m, double e, const double* Y, double T0, double tol,
                       int max_iter, double* T_out, bool enthalpy = false) {
  double T = T0;
  for (int it = 1; it <= max_iter; ++it) {
    double dT = -(mixture_caloric(m, T, Y, enthalpy) - e) / mixture_heat_capacity(m, T, Y, enthalpy);
    double Tn = T + dT;
    if (Tn < 100.0) Tn = 100.0;
    if (Tn > 5000.0) Tn = 5000.0;
    bool done = std::fabs(Tn - T) <= tol * Tn;
    T = Tn;
    if (done) {
      double dT2 = -(mixture_caloric(m, T, Y, enthalpy) - e) / mixture_heat_capacity(m, T, Y, enthalpy);
      T = T + dT2;
      *T_out = T;
      return it + 1;
    }
  }
  *T_out = T;
  return -1;
}

// Bisection on [lo, hi] for e(T) = e, or h(T) = h (independent check of the Newton result).
double temperature_bisect(const OMech& m, double e, const double* Y, double lo, double hi,
                          bool enthalpy = false) {
  double flo = mixture_caloric(m, lo, Y, enthalpy) - e;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double fm = mixture_caloric(m, mid, Y, enthalpy) - e;
    if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
  }
  return 0.5 * (lo + hi);
}

// ---------------------------------------------------------------------------
// Kinetics (Sec. A.1 Eqs. reactions, production_rates, reaction_rates,
// concentrations, rate_coeff, equil_constants)
// ---------------------------------------------------------------------------

// k = A T^b exp(-theta/T)      (Eq. rate_coeff)
template <class S> S arrhenius(double A, double b, double theta, S T) {
  return A * pow(T, b) * exp(-theta / T);
}

// [M]_j = sum_k eps_kj C_k, eps default 1      (reading (c9))
template <class S> S third_body(const OReaction& r, const S* C, int N) {
  S M = 0;
  for (int k = 0; k < N; ++k) {
    double e = 1.0;
    for (auto& p : r.eff) if (p.first == k) e = p.second;
    M += e * C[k];
  }
  return M;
}

// Troe falloff blending (cited in Sec. A.1 for concentration-dependent rate
// coefficients; standard form, reading (c8)).  Lindemann when no Troe data.
template <class S> S falloff_factor(const OReaction& r, S T, S Pr) {
  if (r.n_sri >= 3) {
    // SRI form (reading (p1)): F = d [a exp(-b/T) + exp(-T/c)]^X T^e,  X = 1/(1 + (log10 Pr)^2)
    S lPr = log10(Pr);
    S X = 1.0 / (1.0 + lPr * lPr);
    S base = r.sri[0] * exp(-r.sri[1] / T) + exp(-T / r.sri[2]);
    return r.sri[3] * pow(base, X) * pow(T, r.sri[4]);
  }
  if (r.n_troe < 3) return S(1.0);
  double a = r.troe[0], T3 = r.troe[1], T1 = r.troe[2];
  S Fcent = (1.0 - a) * exp(-T / T3) + a * exp(-T / T1);
  if (r.n_troe >= 4) Fcent += exp(-r.troe[3] / T);
  S lFc = log10(Fcent);
  S c = -0.4 - 0.67 * lFc;
  S n = 0.75 - 1.27 * lFc;
  const double d = 0.14;
  S lPr = log10(Pr);
  S f = (lPr + c) / (n - d * (lPr + c));
  S lF = lFc / (1.0 + f * f);
  return pow(S(10.0), lF);
}

// forward rate coefficient k_f,j (includes [M] for third-body reactions, reading (c14))
// PLOG rate coefficient (reading (p2)): with the mixture pressure p = R T sum_k C_k
// (Eq. eos), k = k_1(T) for p <= p_1, k = k_n(T) for p >= p_n, and in between
// ln k interpolated linearly in ln p between the bracketing nodes
// p_i <= p < p_{i+1}: ln k = ln k_i + (ln k_{i+1} - ln k_i)(ln p - ln p_i)/(ln p_{i+1} - ln p_i).
template <class S> S plog_rate(const OReaction& r, S T, const S* C, int N) {
  S ctot = 0;
  for (int k = 0; k < N; ++k) ctot += C[k];
  S p = R_GAS * T * ctot;
  const auto& nd = r.plog;
  const int n = (int)nd.size();
  if (re(p) <= nd[0][0]) return arrhenius(nd[0][1], nd[0][2], nd[0][3], T);
  if (re(p) >= nd[n - 1][0]) return arrhenius(nd[n - 1][1], nd[n - 1][2], nd[n - 1][3], T);
  int i = 0;
  while (!(re(p) < nd[i + 1][0])) ++i;
  S lk0 = log(arrhenius(nd[i][1], nd[i][2], nd[i][3], T));
  S lk1 = log(arrhenius(nd[i + 1][1], nd[i + 1][2], nd[i + 1][3], T));
  S w = (log(p) - log(nd[i][0])) / (log(nd[i + 1][0]) - log(nd[i][0]));
  return exp(lk0 + (lk1 - lk0) * w);
}

template <class S> S forward_rate_coefficient(const OMech& m, const OReaction& r, S T, const S* C) {
  int N = m.N();
  if (r.kind == K_ARRHENIUS) return arrhenius(r.A, r.b, r.theta, T);
  if (r.kind == K_PLOG) return plog_rate(r, T, C, N);
  if (r.kind == K_THREEBODY) return arrhenius(r.A, r.b, r.theta, T) * third_body(r, C, N);
  // falloff: k = k_inf * Pr/(1+Pr) * F,  Pr = k0 [M] / k_inf
  S kinf = arrhenius(r.A, r.b, r.theta, T);
  S k0 = arrhenius(r.A0, r.b0, r.theta0, T);
  S Pr = k0 * third_body(r, C, N) / kinf;
  if (re(Pr) < 1e-300) Pr = Pr - re(Pr) + 1e-300;   // guard log10(0) (reading (c8))
  // Pr/(1+Pr) written as 1/(1 + 1/Pr): the same value, but its derivative does
  // not subtract two nearly equal numbers when Pr >> 1
  return kinf / (1.0 + 1.0 / Pr) * falloff_factor(r, T, Pr);
}

// K_j = (p0/(R T))^{sum_i nu_ij} exp(-sum_i nu_ij g_i/(R T))      (Eq. equil_constants, reading (c1))
template <class S> S equilibrium_constant(const OMech& m, const OReaction& r, S T) {
  double dnu = 0;
  S dg = 0;
  for (auto& p : r.prod) { dnu += p.second; dg += (double)p.second * g_RT(m.sp[p.first], T); }
  for (auto& p : r.reac) { dnu -= p.second; dg -= (double)p.second * g_RT(m.sp[p.first], T); }
  return pow(P_ATM / (R_GAS * T), dnu) * exp(-dg);
}

template <class S> S conc_product(const std::vector<std::pair<int, int>>& side, const S* C) {
  S p = 1.0;
  for (auto& q : side)
    for (int i = 0; i < q.second; ++i) p *= C[q.first];
  return p;
}

// C_k = rho Y_k / W_k      (Eq. concentrations)
template <class S> void concentrations(const OMech& m, S rho, const S* Y, S* C) {
  for (int k = 0; k < m.N(); ++k) C[k] = rho * Y[k] / m.sp[k].W;
}

// Rates of progress, law of mass action (Eq. reaction_rates):
//   R_j = k_j [prod C^nu' - (1/K_j) prod C^nu'']  = Rf_j - Rr_j
template <class S> void rates_of_progress(const OMech& m, S rho, S T, const S* Y, S* Rf, S* Rr,
                                          S* kf_out = nullptr, S* Kc_out = nullptr) {
  int N = m.N();
  std::vector<S> C(N);
  concentrations(m, rho, Y, C.data());
  for (int j = 0; j < m.M(); ++j) {
    const OReaction& r = m.rx[j];
    S kf = forward_rate_coefficient(m, r, T, C.data());
    S Kc = equilibrium_constant(m, r, T);
    Rf[j] = kf * conc_product(r.reac, C.data());
    Rr[j] = r.reversible ? kf / Kc * conc_product(r.prod, C.data()) : S(0.0);
    if (kf_out) kf_out[j] = kf;
    if (Kc_out) Kc_out[j] = Kc;
  }
}

// Net production rates (Eq. production_rates): omega_i = sum_j nu_ij R_j,
// nu = nu'' - nu' (Eq. reactions).  Optionally the gross scale
// G_i = sum_j |nu_ij| (|Rf_j| + |Rr_j|) used for the parity tolerance (reading (c15)).
template <class S> void net_production_rates(const OMech& m, S rho, S T, const S* Y, S* omega,
                                             double* gross = nullptr) {
  int N = m.N(), M = m.M();
  std::vector<S> Rf(M), Rr(M);
  rates_of_progress(m, rho, T, Y, Rf.data(), Rr.data());
  for (int k = 0; k < N; ++k) omega[k] = 0.0;
  if (gross) for (int k = 0; k < N; ++k) gross[k] = 0.0;
  for (int j = 0; j < M; ++j) {
    const OReaction& r = m.rx[j];
    S Rj = Rf[j] - Rr[j];
    // nu_ij for every species of the reaction (a species may appear on both sides)
    std::map<int, int> nu;
    for (auto& p : r.prod) nu[p.first] += p.second;
    for (auto& p : r.reac) nu[p.first] -= p.second;
    for (auto& q : nu) {
      omega[q.first] += (double)q.second * Rj;
      if (gross) gross[q.first] += std::abs(q.second) * (std::fabs((double)re(Rf[j])) + std::fabs((double)re(Rr[j])));
    }
  }
}

// Temperature rate of the adiabatic isochoric reactor (Sec. A.1 Eq. massfrac_ode with
// e fixed, reading (c13)):  dT/dt = -sum_k (h_k - R T) omega_k / (rho c_v)
template <class S> S temperature_rate(const OMech& m, S rho, S T, const S* Y, const S* omega) {
  S num = 0;
  for (int k = 0; k < m.N(); ++k) num += (R_GAS * T * h_RT(m.sp[k], T) - R_GAS * T) * omega[k];
  return -num / (rho * cv_mass(m, T, Y));
}

typedef std::complex<double> cplx;
const double CS_H = 1e-30;   // complex-step size (the learned guess's loss derivative only)

// Chemical Jacobian J_jk = dS_j/dY_k of the source S_j = W_j omega_j (Eq. massfrac_ode,
// Eq. chem_jacobian) at fixed rho and e: T follows Y through the inversion of
// Eq. int_energy, and differentiating e = sum_i Y_i e_i(T) at fixed e gives
// dT/dY_k = -e_k(T)/c_v (Eq. cv).  One dual evaluation per column moves Y_k with
// derivative 1 and T with derivative dT/dY_k together, so the derivative part of
// omega carries d omega/dY_k + d omega/dT dT/dY_k.  J is row-major [j][k], N x N.
void source_jacobian_adiabatic(const OMech& m, double rho, double T, const double* Y, double* J) {
  const int N = m.N();
  const double cv = cv_mass(m, T, Y);
  std::vector<Dual> y(N), w(N);
  for (int c = 0; c < N; ++c) {
    for (int k = 0; k < N; ++k) y[k] = Dual(Y[k], k == c ? 1.0 : 0.0);
    const double ec = (R_GAS * T * h_RT(m.sp[c], T) - R_GAS * T) / m.sp[c].W;   // e_c per unit mass
    Dual Tc(T, -ec / cv);
    net_production_rates<Dual>(m, Dual(rho), Tc, y.data(), w.data());
    for (int j = 0; j < N; ++j) J[j * N + c] = m.sp[j].W * w[j].d;
  }
}

// Solve A x = b (A n x n row-major, overwritten; b overwritten by x) by Gaussian
// elimination with partial pivoting.  Returns false for a zero pivot.
bool solve_dense(int n, double* A, double* b) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i) if (std::fabs(A[i * n + k]) > std::fabs(A[p * n + k])) p = i;
    if (A[p * n + k] == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      double l = A[i * n + k] / A[k * n + k];
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
      b[i] -= l * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * b[j];
    b[i] = s / A[i * n + i];
  }
  return true;
}

// One Crank-Nicolson step of Eq. massfrac_ode for the adiabatic isochoric reactor
// (Eqs. crank_nicol_rhs, crank_nicol_newton_system, crank_nicol_newton_update,
// crank_nicol_jac).  Reading: Eq. massfrac_ode gives dY/dt = S/rho, so the
// residual is F = Y - Y^m - dt/(2 rho) (S(Y) + S(Y^m)) and the Newton matrix is
// I - dt/(2 rho) J with J = dS/dY at fixed (rho, e).  Newton starts from Y^m;
// T follows each iterate through T(e, Y).  Stop rule as for the temperature
// solve: once max_k |dY_k| <= tol, one more step.  Returns the Newton steps
// taken, or -1 (no convergence within max_newton, or a singular matrix).
int cn_step(const OMech& m, double rho, double dt, const double* Ym, double Tm, double tol, int max_newton,
            double* Y_out, double* T_out) {
  const int N = m.N();
  const double e = internal_energy(m, Tm, Ym);
  const double h = dt / (2.0 * rho);
  std::vector<double> Sm(N), w(N), Y(Ym, Ym + N), A((size_t)N * N), b(N);
  net_production_rates(m, rho, Tm, Ym, w.data());
  for (int k = 0; k < N; ++k) Sm[k] = m.sp[k].W * w[k];
  double T = Tm;
  bool flag = false;
  int it = 0;
  for (; it < max_newton + 1; ) {
    ++it;
    double Tn;
    if (temperature_newton(m, e, Y.data(), T, 1e-14, 100, &Tn) < 0) return -1;
    T = Tn;
    net_production_rates(m, rho, T, Y.data(), w.data());
    source_jacobian_adiabatic(m, rho, T, Y.data(), A.data());
    for (int j = 0; j < N; ++j) {
      b[j] = -(Y[j] - Ym[j] - h * (m.sp[j].W * w[j] + Sm[j]));
      for (int k = 0; k < N; ++k) A[j * N + k] = (j == k ? 1.0 : 0.0) - h * A[j * N + k];
    }
    if (!solve_dense(N, A.data(), b.data())) return -1;
    double dmax = 0;
    for (int k = 0; k < N; ++k) { Y[k] += b[k]; dmax = std::max(dmax, std::fabs(b[k])); }
    if (flag) break;
    if (dmax <= tol) flag = true;
    else if (it >= max_newton) { it = -1; break; }
  }
  if (it > 0) {
    double Tn;
    if (temperature_newton(m, e, Y.data(), T, 1e-14, 100, &Tn) < 0) return -1;
    T = Tn;
  }
  for (int k = 0; k < N; ++k) Y_out[k] = Y[k];
  *T_out = T;
  return it;
}

// ---------------------------------------------------------------------------
// Mixture-averaged transport (Sec. A.2: Eq. mixavg_flux, Eq. diff_mix_rule,
// Eq. mixavg_viscosity, Eq. mixavg_conductivity, Eq. species_cond).
// Reading (t1): "log" in the fits is the natural logarithm.  Reading (t2): the
// binary diffusivity fits carry no pressure factor, as printed.
// ---------------------------------------------------------------------------

template <class S> S poly_logT(const std::vector<double>& c, S T) {
  S lt = log(T), v = 0;
  for (int m = 0; m <= 4; ++m) v += c[m] * pow(lt, (double)m);
  return v;
}

// mu_i = sqrt(T) [sum_m b_im (log T)^m]^2
template <class S> S species_viscosity(const OMech& m, int k, S T) {
  S b = poly_logT(m.visc[k], T);
  return sqrt(T) * b * b;
}
// kappa_i = sqrt(T) sum_m c_im (log T)^m      (Eq. species_cond)
template <class S> S species_conductivity(const OMech& m, int k, S T) {
  return sqrt(T) * poly_logT(m.cond[k], T);
}
// D_ij = sqrt(T) sum_m a_ijm (log T)^m
template <class S> S binary_diffusivity(const OMech& m, int k, int j, S T) {
  return sqrt(T) * poly_logT(m.bdiff[k][j], T);
}

// mole fractions X_k = W Y_k / W_k with W = (sum_k Y_k/W_k)^-1 (Eq. eos)
template <class S> S mole_fractions(const OMech& m, const S* Y, S* X) {
  S inv = 0;
  for (int k = 0; k < m.N(); ++k) inv += Y[k] / m.sp[k].W;
  S W = 1.0 / inv;
  for (int k = 0; k < m.N(); ++k) X[k] = W * Y[k] / m.sp[k].W;
  return W;
}

// Wilke's Phi_kj = [1 + sqrt((mu_k/mu_j) sqrt(W_j/W_k))]^2 / sqrt(8 (1 + W_k/W_j))
template <class S> S wilke_phi(const OMech& m, int k, int j, S mu_k, S mu_j) {
  double Wk = m.sp[k].W, Wj = m.sp[j].W;
  S t = 1.0 + sqrt((mu_k / mu_j) * sqrt(Wj / Wk));
  return t * t / sqrt(8.0 * (1.0 + Wk / Wj));
}

// mu = sum_k X_k mu_k / sum_j Phi_kj X_j      (Eq. mixavg_viscosity)
template <class S> S mixture_viscosity(const OMech& m, S T, const S* Y) {
  int N = m.N();
  std::vector<S> X(N), mu(N);
  mole_fractions(m, Y, X.data());
  for (int k = 0; k < N; ++k) mu[k] = species_viscosity(m, k, T);
  S out = 0;
  for (int k = 0; k < N; ++k) {
    S den = 0;
    for (int j = 0; j < N; ++j) den += wilke_phi(m, k, j, mu[k], mu[j]) * X[j];
    out += X[k] * mu[k] / den;
  }
  return out;
}

// kappa = (1/2) [sum_k X_k kappa_k + (sum_k X_k/kappa_k)^-1]      (Eq. mixavg_conductivity)
template <class S> S mixture_conductivity(const OMech& m, S T, const S* Y) {
  int N = m.N();
  std::vector<S> X(N);
  mole_fractions(m, Y, X.data());
  S a = 0, h = 0;
  for (int k = 0; k < N; ++k) {
    S kk = species_conductivity(m, k, T);
    a += X[k] * kk;
    h += X[k] / kk;
  }
  return 0.5 * (a + 1.0 / h);
}

// D_km = (W - X_k W_k)/W (sum_{j != k} X_j/D_kj)^-1      (Eq. diff_mix_rule)
template <class S> void mixture_diffusivities(const OMech& m, S T, const S* Y, S* Dm) {
  int N = m.N();
  std::vector<S> X(N);
  S W = mole_fractions(m, Y, X.data());
  for (int k = 0; k < N; ++k) {
    S sum = 0;
    for (int j = 0; j < N; ++j)
      if (j != k) sum += X[j] / binary_diffusivity(m, k, j, T);
    Dm[k] = (W - X[k] * m.sp[k].W) / W / sum;
  }
}

// ---------------------------------------------------------------------------
// BF16 MLP for the Newton initial guess (model definition; FP64 arithmetic
// with bf16 rounding at the same points as the GPU network).
// ---------------------------------------------------------------------------

double round_bf16(double x) {
  // round-to-nearest-even to 8 significant bits (bf16), via float
  float f = (float)x;
  uint32_t u; std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return f;
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  u &= 0xffff0000u;
  std::memcpy(&f, &u, 4);
  return f;
}

template <class S> S silu(S x) { return x / (1.0 + exp(-x)); }
template <class S> S rbf(S x) { return x - re(x) + round_bf16(re(x)); }   // straight-through rounding


template <class S>
S mlp_forward_one(int D, int H, const double* P, const S* x, std::vector<S>& a1, std::vector<S>& a2,
                  std::vector<S>& z1, std::vector<S>& z2) {
  const double* W1 = P; const double* b1 = W1 + H * D;
  const double* W2 = b1 + H; const double* b2 = W2 + H * H;
  const double* w3 = b2 + H; const double* b3 = w3 + H;
  for (int o = 0; o < H; ++o) {
    S z = b1[o];
    for (int i = 0; i < D; ++i) z += W1[o * D + i] * rbf(x[i]);
    z1[o] = z; a1[o] = rbf(silu(z));
  }
  for (int o = 0; o < H; ++o) {
    S z = b2[o];
    for (int i = 0; i < H; ++i) z += W2[o * H + i] * a1[i];
    z2[o] = z; a2[o] = rbf(silu(z));
  }
  S y = b3[0];
  for (int i = 0; i < H; ++i) y += w3[i] * a2[i];
  return y;
}

}  // namespace

// ===========================================================================
// C interface (ctypes).  All arrays SoA: X[k*n + p].
// ===========================================================================

extern "C" {

const char* orc_last_error() { return g_err.c_str(); }

void* orc_load(const char* path) {
  OMech* m = new OMech();
  if (!parse_mech(path, *m)) { delete m; return nullptr; }
  return m;
}

void orc_free(void* h) { delete (OMech*)h; }

int orc_info(void* h, int* N, int* M) {
  OMech* m = (OMech*)h; *N = m->N(); *M = m->M(); return 0;
}

int orc_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

void orc_mol_weights(void* h, double* W) {
  OMech* m = (OMech*)h;
  for (int k = 0; k < m->N(); ++k) W[k] = m->sp[k].W;
}

// out[4] = cp/R, h/RT, s/R, g/RT of species k at T
void orc_species_thermo(void* h, int k, double T, double* out) {
  OMech* m = (OMech*)h;
  out[0] = cp_R(m->sp[k], T); out[1] = h_RT(m->sp[k], T);
  out[2] = s_R(m->sp[k], T);  out[3] = g_RT(m->sp[k], T);
}

// temperature derivatives (dual numbers): out[0] = d(h/R)/dT, out[1] = d(s/R)/dT, out[2] = d(cp/R)/dT
void orc_species_thermo_dT(void* h, int k, double T, double* out) {
  OMech* m = (OMech*)h;
  Dual Tc(T, 1.0);
  out[0] = (Tc * h_RT(m->sp[k], Tc)).d;
  out[1] = s_R(m->sp[k], Tc).d;
  out[2] = cp_R(m->sp[k], Tc).d;
}

void orc_density(void* h, int64_t n, const double* p, const double* T, const double* Y, double* rho) {
  OMech* m = (OMech*)h; int N = m->N();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    rho[i] = density(*m, p[i], T[i], y.data());
  }
}

void orc_internal_energy(void* h, int64_t n, const double* T, const double* Y, double* e, double* cv) {
  OMech* m = (OMech*)h; int N = m->N();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    e[i] = internal_energy(*m, T[i], y.data());
    if (cv) cv[i] = cv_mass(*m, T[i], y.data());
  }
}

// Returns the number of points that did not converge.
int64_t orc_temperature(void* h, int64_t n, const double* e, const double* Y, const double* guess,
                        double T_guess, double tol, int max_iter, double* T, int32_t* iters) {
  OMech* m = (OMech*)h; int N = m->N();
  int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+:bad)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    double T0 = guess ? guess[i] : T_guess;
    int it = temperature_newton(*m, e[i], y.data(), T0, tol, max_iter, &T[i]);
    if (iters) iters[i] = it;
    if (it < 0) ++bad;
  }
  return bad;
}

void orc_temperature_bisect(void* h, int64_t n, const double* e, const double* Y, double lo, double hi,
                            double* T) {
  OMech* m = (OMech*)h; int N = m->N();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    T[i] = temperature_bisect(*m, e[i], y.data(), lo, hi);
  }
}

void orc_enthalpy(void* h, int64_t n, const double* T, const double* Y, double* hm, double* cp) {
  OMech* m = (OMech*)h; int N = m->N();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    hm[i] = enthalpy_mass(*m, T[i], y.data());
    if (cp) cp[i] = cp_mass(*m, T[i], y.data());
  }
}

// T(h, Y) by the enthalpy variant of the Newton inversion; returns the number of
// points that did not converge.
int64_t orc_temperature_enthalpy(void* h, int64_t n, const double* hm, const double* Y, const double* guess,
                                 double T_guess, double tol, int max_iter, double* T, int32_t* iters) {
  OMech* m = (OMech*)h; int N = m->N();
  int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+:bad)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    double T0 = guess ? guess[i] : T_guess;
    int it = temperature_newton(*m, hm[i], y.data(), T0, tol, max_iter, &T[i], true);
    if (iters) iters[i] = it;
    if (it < 0) ++bad;
  }
  return bad;
}

void orc_temperature_bisect_enthalpy(void* h, int64_t n, const double* hm, const double* Y, double lo,
                                     double hi, double* T) {
  OMech* m = (OMech*)h; int N = m->N();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    T[i] = temperature_bisect(*m, hm[i], y.data(), lo, hi, true);
  }
}

// Per-reaction quantities at each point: kf, Kc, Rf, Rr (each [M][n]); any may be null.
void orc_reaction_data(void* h, int64_t n, const double* rho, const double* T, const double* Y,
                       double* kf, double* Kc, double* Rf, double* Rr) {
  OMech* m = (OMech*)h; int N = m->N(), M = m->M();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N), a(M), b(M), c(M), d(M);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    rates_of_progress(*m, rho[i], T[i], y.data(), a.data(), b.data(), c.data(), d.data());
    for (int j = 0; j < M; ++j) {
      if (Rf) Rf[j * n + i] = a[j];
      if (Rr) Rr[j * n + i] = b[j];
      if (kf) kf[j * n + i] = c[j];
      if (Kc) Kc[j * n + i] = d[j];
    }
  }
}

// omega [N][n] and (optional) gross scale [N][n]; if T_in is null, T is solved
// from e (Newton from T_guess) and written to T_out.
void orc_net_production_rates(void* h, int64_t n, const double* rho, const double* T_in, const double* Y,
                              double* omega, double* gross) {
  OMech* m = (OMech*)h; int N = m->N();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N), w(N), g(N);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    net_production_rates(*m, rho[i], T_in[i], y.data(), w.data(), gross ? g.data() : nullptr);
    for (int k = 0; k < N; ++k) {
      omega[k * n + i] = w[k];
      if (gross) gross[k * n + i] = g[k];
    }
  }
}

// the same in long double (rounding envelope of the double oracle)
void orc_net_production_rates_ld(void* h, int64_t n, const double* rho, const double* T_in,
                                 const double* Y, double* omega) {
  OMech* m = (OMech*)h; int N = m->N();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<long double> y(N), w(N);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    net_production_rates<long double>(*m, rho[i], T_in[i], y.data(), w.data(), nullptr);
    for (int k = 0; k < N; ++k) omega[k * n + i] = (double)w[k];
  }
}

// dT/dt of the adiabatic isochoric reactor, [n]
void orc_temperature_rate(void* h, int64_t n, const double* rho, const double* T, const double* Y,
                          double* Tdot) {
  OMech* m = (OMech*)h; int N = m->N();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N), w(N);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    net_production_rates(*m, rho[i], T[i], y.data(), w.data());
    Tdot[i] = temperature_rate(*m, rho[i], T[i], y.data(), w.data());
  }
}

// Dense Jacobian d(Tdot, omega)/d(T, Y) at fixed rho, one dual evaluation per column,
// reading (c13).
// J[(r*(N+1) + c)*n + p]; row 0 = Tdot, rows 1..N = omega; column 0 = T, columns 1..N = Y.
void orc_jacobian(void* h, int64_t n, const double* rho, const double* T, const double* Y, double* J) {
  OMech* m = (OMech*)h; int N = m->N(); int NP = N + 1;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<Dual> y(N), w(N);
    for (int c = 0; c < NP; ++c) {
      Dual Tc(T[i], c == 0 ? 1.0 : 0.0);
      for (int k = 0; k < N; ++k) y[k] = Dual(Y[k * n + i], (c == k + 1) ? 1.0 : 0.0);
      Dual rc(rho[i]);
      net_production_rates<Dual>(*m, rc, Tc, y.data(), w.data());
      Dual td = temperature_rate<Dual>(*m, rc, Tc, y.data(), w.data());
      J[(0 * NP + c) * n + i] = td.d;
      for (int k = 0; k < N; ++k) J[((k + 1) * NP + c) * n + i] = w[k].d;
    }
  }
}

// JVP of omega(rho, T, Y) along v = (drho, dT, dY): domega = sum_c (d omega/d x_c) v_c, [N][n],
// the columns by dual evaluations one variable at a time.
void orc_jvp(void* h, int64_t n, const double* rho, const double* T, const double* Y,
             const double* drho, const double* dT, const double* dY, double* domega) {
  OMech* m = (OMech*)h; int N = m->N();
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<Dual> y(N), w(N);
    std::vector<double> acc(N, 0.0);
    for (int c = 0; c < N + 2; ++c) {
      const double vc = c == 0 ? drho[i] : c == 1 ? dT[i] : dY[(c - 2) * n + i];
      if (vc == 0.0) continue;
      Dual rc(rho[i], c == 0 ? 1.0 : 0.0), Tc(T[i], c == 1 ? 1.0 : 0.0);
      for (int k = 0; k < N; ++k) y[k] = Dual(Y[k * n + i], (c == k + 2) ? 1.0 : 0.0);
      net_production_rates<Dual>(*m, rc, Tc, y.data(), w.data());
      for (int k = 0; k < N; ++k) acc[k] += w[k].d * vc;
    }
    for (int k = 0; k < N; ++k) domega[k * n + i] = acc[k];
  }
}

// VJP of omega(rho, T, Y): (rho_bar, T_bar, Y_bar) = J^T omega_bar with J = d omega/d(rho, T, Y)
// formed column by column (dual numbers).
void orc_vjp(void* h, int64_t n, const double* rho, const double* T, const double* Y,
             const double* wbar, double* rho_bar, double* T_bar, double* Y_bar) {
  OMech* m = (OMech*)h; int N = m->N();
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<Dual> y(N), w(N);
    for (int c = 0; c < N + 2; ++c) {
      Dual rc(rho[i], c == 0 ? 1.0 : 0.0), Tc(T[i], c == 1 ? 1.0 : 0.0);
      for (int k = 0; k < N; ++k) y[k] = Dual(Y[k * n + i], (c == k + 2) ? 1.0 : 0.0);
      net_production_rates<Dual>(*m, rc, Tc, y.data(), w.data());
      double acc = 0;
      for (int k = 0; k < N; ++k) acc += wbar[k * n + i] * w[k].d;
      if (c == 0) rho_bar[i] = acc;
      else if (c == 1) T_bar[i] = acc;
      else Y_bar[(c - 2) * n + i] = acc;
    }
  }
}

// Gross scale of every derivative entry: reading (c15) carried over to the
// derivatives.  The tolerance of a production-rate entry is set by the sizes of
// the terms that cancel in it, so for omega_k and a variable x_c
//   GJ_kc = sum_j |nu_kj| (|d Rf_j/d x_c| + |d Rr_j/d x_c|),
// the forward and reverse rates of progress (Eq. reaction_rates) differentiated
// separately (dual numbers).  For the temperature rate of the adiabatic
// isochoric reactor, Tdot = -sum_k ehat_k omega_k / (rho c_v) with
// ehat_k = h_k - R T (reading (c13)), the same magnitudes are carried through
// its product and quotient rules:
//   GJ_0c = [sum_k (|d ehat_k/d x_c| G_k + |ehat_k| GJ_kc)] / (rho c_v)
//           + Tg |d(rho c_v)/d x_c| / (rho c_v),   Tg = sum_k |ehat_k| G_k / (rho c_v),
// G_k = sum_j |nu_kj| (|Rf_j| + |Rr_j|) the gross scale of omega_k.
// GJ[(r*(N+2) + c)*n + p]: rows r = 0 (Tdot), 1..N (omega_1..N); columns c = 0 (rho),
// 1 (T), 2..N+1 (Y_1..Y_N).
void orc_jacobian_gross(void* h, int64_t n, const double* rho, const double* T, const double* Y, double* GJ) {
  OMech* m = (OMech*)h; const int N = m->N(), M = m->M(), NC = N + 2;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N), Rf(M), Rr(M), G(N, 0.0), eh(N), deh(N);
    std::vector<Dual> yc(N), Rfc(M), Rrc(M);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    rates_of_progress(*m, rho[i], T[i], y.data(), Rf.data(), Rr.data());
    std::vector<std::map<int, int>> nu(M);
    for (int j = 0; j < M; ++j) {
      for (auto& p : m->rx[j].prod) nu[j][p.first] += p.second;
      for (auto& p : m->rx[j].reac) nu[j][p.first] -= p.second;
      for (auto& q : nu[j]) G[q.first] += std::abs(q.second) * (std::fabs(Rf[j]) + std::fabs(Rr[j]));
    }
    const double cv = cv_mass(*m, T[i], y.data()), rcv = rho[i] * cv;
    double Tg = 0.0;
    for (int k = 0; k < N; ++k) {
      eh[k] = R_GAS * T[i] * h_RT(m->sp[k], T[i]) - R_GAS * T[i];
      Dual Tc(T[i], 1.0);
      deh[k] = (R_GAS * Tc * h_RT(m->sp[k], Tc) - R_GAS * Tc).d;   // cp_k - R
      Tg += std::fabs(eh[k]) * G[k] / rcv;
    }
    for (int c = 0; c < NC; ++c) {
      Dual rc(rho[i], c == 0 ? 1.0 : 0.0), Tc(T[i], c == 1 ? 1.0 : 0.0);
      for (int k = 0; k < N; ++k) yc[k] = Dual(y[k], (c == k + 2) ? 1.0 : 0.0);
      rates_of_progress<Dual>(*m, rc, Tc, yc.data(), Rfc.data(), Rrc.data());
      std::vector<double> col(N, 0.0);
      for (int j = 0; j < M; ++j) {
        const double df = std::fabs(Rfc[j].d), dr = std::fabs(Rrc[j].d);
        for (auto& q : nu[j]) col[q.first] += std::abs(q.second) * (df + dr);
      }
      const double drcv = std::fabs((rc * cv_mass<Dual>(*m, Tc, yc.data())).d);
      double g0 = Tg * drcv / rcv;
      for (int k = 0; k < N; ++k) {
        g0 += ((c == 1 ? std::fabs(deh[k]) * G[k] : 0.0) + std::fabs(eh[k]) * col[k]) / rcv;
        GJ[((int64_t)(k + 1) * NC + c) * n + i] = col[k];
      }
      GJ[(int64_t)c * n + i] = g0;
    }
  }
}

// Chemical Jacobian dS/dY at fixed (rho, e), [N*N][n]: J[(j*N + k)*n + p] = dS_j/dY_k.
void orc_jacobian_adiabatic(void* h, int64_t n, const double* rho, const double* T, const double* Y,
                            double* J) {
  OMech* m = (OMech*)h; int N = m->N();
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N), A((size_t)N * N);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    source_jacobian_adiabatic(*m, rho[i], T[i], y.data(), A.data());
    for (int q = 0; q < N * N; ++q) J[(int64_t)q * n + i] = A[q];
  }
}

// Source terms S = W omega at fixed (rho, e) as a function of Y alone (for finite
// differences of the adiabatic Jacobian): T solved from e each call.  [N][n]
void orc_source_at_energy(void* h, int64_t n, const double* rho, const double* e, const double* Y,
                          double* S) {
  OMech* m = (OMech*)h; int N = m->N();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N), w(N);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    double T;
    temperature_newton(*m, e[i], y.data(), 1200.0, 1e-14, 100, &T);
    net_production_rates(*m, rho[i], T, y.data(), w.data());
    for (int k = 0; k < N; ++k) S[k * n + i] = m->sp[k].W * w[k];
  }
}

// Dense solve (Gaussian elimination with partial pivoting), one system: A [n*n]
// row-major, b [n]; x returned in b.  Returns 0, or -1 for a singular matrix.
int orc_solve_dense(int n, double* A, double* b) { return solve_dense(n, A, b) ? 0 : -1; }

int orc_has_transport(void* h) { return ((OMech*)h)->visc.empty() ? 0 : 1; }

// species fits at T: out = (mu_k, kappa_k)
void orc_species_transport(void* h, int k, double T, double* out) {
  const OMech& m = *(OMech*)h;
  out[0] = species_viscosity(m, k, T);
  out[1] = species_conductivity(m, k, T);
}

double orc_binary_diffusivity(void* h, int k, int j, double T) {
  return binary_diffusivity(*(OMech*)h, k, j, T);
}

// Phi [N*N] (row k, column j) at T
void orc_wilke_phi(void* h, double T, double* Phi) {
  const OMech& m = *(OMech*)h;
  int N = m.N();
  for (int k = 0; k < N; ++k)
    for (int j = 0; j < N; ++j)
      Phi[k * N + j] = wilke_phi(m, k, j, species_viscosity(m, k, T), species_viscosity(m, j, T));
}

// mu [n], kappa [n], Dm [N][n] (each nullable)
void orc_transport(void* h, int64_t n, const double* T, const double* Y, double* mu, double* kappa, double* Dm) {
  const OMech& m = *(OMech*)h;
  const int N = m.N();
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N), d(N);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    if (mu) mu[i] = mixture_viscosity(m, T[i], y.data());
    if (kappa) kappa[i] = mixture_conductivity(m, T[i], y.data());
    if (Dm) {
      mixture_diffusivities(m, T[i], y.data(), d.data());
      for (int k = 0; k < N; ++k) Dm[k * n + i] = d[k];
    }
  }
}

// the same in long double (rounding envelope of the double oracle)
void orc_transport_ld(void* h, int64_t n, const double* T, const double* Y, double* mu, double* kappa, double* Dm) {
  const OMech& m = *(OMech*)h;
  const int N = m.N();
  for (int64_t i = 0; i < n; ++i) {
    std::vector<long double> y(N), d(N);
    for (int k = 0; k < N; ++k) y[k] = Y[k * n + i];
    long double t = T[i];
    mu[i] = (double)mixture_viscosity<long double>(m, t, y.data());
    kappa[i] = (double)mixture_conductivity<long double>(m, t, y.data());
    mixture_diffusivities<long double>(m, t, y.data(), d.data());
    for (int k = 0; k < N; ++k) Dm[k * n + i] = (double)d[k];
  }
}

// One Crank-Nicolson step per point; returns the number of points that failed.
int64_t orc_cn_step(void* h, int64_t n, double dt, const double* rho, const double* Tm, const double* Ym,
                    double tol, int max_newton, double* Y_out, double* T_out, int32_t* iters) {
  OMech* m = (OMech*)h; int N = m->N();
  int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+:bad)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<double> y(N), yo(N);
    for (int k = 0; k < N; ++k) y[k] = Ym[k * n + i];
    double T;
    int it = cn_step(*m, rho[i], dt, y.data(), Tm[i], tol, max_newton, yo.data(), &T);
    for (int k = 0; k < N; ++k) Y_out[k * n + i] = yo[k];
    T_out[i] = T;
    if (iters) iters[i] = it;
    if (it < 0) ++bad;
  }
  return bad;
}

// ---------------------------------------------------------------------------
// MLP (D_in -> H -> H -> 1, SiLU).  Parameters packed as
//   W1[H][D], b1[H], W2[H][H], b2[H], w3[H], b3[1]     (row-major, doubles)
// Input features x[n][D] (already normalised; rounded to bf16 here), output
// y[n] = network output in normalised units.  Weights are used as given
// (the caller passes bf16-exact values); hidden activations are rounded to
// bf16 after SiLU, the output is not.
// ---------------------------------------------------------------------------

void orc_mlp_forward(int D, int H, const double* P, int64_t n, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p) {
    std::vector<double> a1(H), a2(H), z1(H), z2(H);
    y[p] = mlp_forward_one<double>(D, H, P, x + p * D, a1, a2, z1, z2);
  }
}

// Gradient of L = (1/n) sum_p (y_p - t_p)^2 w.r.t. all parameters (same packing),
// by the chain rule (backpropagation), rounding treated as identity.
double orc_mlp_loss_grad(int D, int H, const double* P, int64_t n, const double* x, const double* t,
                         double* grad) {
  int NPAR = H * D + H + H * H + H + H + 1;
  for (int q = 0; q < NPAR; ++q) grad[q] = 0;
  const double* W2 = P + H * D + H;
  const double* w3 = W2 + H * H + H;
  double loss = 0;
  for (int64_t p = 0; p < n; ++p) {
    std::vector<double> a1(H), a2(H), z1(H), z2(H), d2(H), d1(H);
    const double* xp = x + p * D;
    double y = mlp_forward_one<double>(D, H, P, xp, a1, a2, z1, z2);
    double r = y - t[p];
    loss += r * r;
    double dy = 2.0 * r / (double)n;
    double* gW1 = grad; double* gb1 = gW1 + H * D; double* gW2 = gb1 + H;
    double* gb2 = gW2 + H * H; double* gw3 = gb2 + H; double* gb3 = gw3 + H;
    gb3[0] += dy;
    for (int i = 0; i < H; ++i) {
      gw3[i] += dy * a2[i];
      double s = 1.0 / (1.0 + exp(-z2[i]));
      d2[i] = dy * w3[i] * (s * (1.0 + z2[i] * (1.0 - s)));   // d silu/dz
    }
    for (int o = 0; o < H; ++o) {
      gb2[o] += d2[o];
      for (int i = 0; i < H; ++i) gW2[o * H + i] += d2[o] * a1[i];
    }
    for (int i = 0; i < H; ++i) {
      double acc = 0;
      for (int o = 0; o < H; ++o) acc += d2[o] * W2[o * H + i];
      double s = 1.0 / (1.0 + exp(-z1[i]));
      d1[i] = acc * (s * (1.0 + z1[i] * (1.0 - s)));
    }
    for (int o = 0; o < H; ++o) {
      gb1[o] += d1[o];
      for (int i = 0; i < D; ++i) gW1[o * D + i] += d1[o] * round_bf16(xp[i]);
    }
  }
  return loss / (double)n;
}

// complex-step derivative of the same loss along a parameter direction v (pin for the backprop)
double orc_mlp_loss_dir(int D, int H, const double* P, const double* v, int64_t n, const double* x,
                        const double* t) {
  int NPAR = H * D + H + H * H + H + H + 1;
  std::vector<double> Pr(NPAR);
  // complex parameters: evaluate with a complex copy
  std::vector<cplx> Pc(NPAR);
  for (int q = 0; q < NPAR; ++q) Pc[q] = cplx(P[q], CS_H * v[q]);
  cplx L = 0;
  for (int64_t p = 0; p < n; ++p) {
    const cplx* W1 = Pc.data(); const cplx* b1 = W1 + H * D;
    const cplx* W2 = b1 + H; const cplx* b2 = W2 + H * H;
    const cplx* w3 = b2 + H; const cplx* b3 = w3 + H;
    std::vector<cplx> a1(H), a2(H);
    for (int o = 0; o < H; ++o) {
      cplx z = b1[o];
      for (int i = 0; i < D; ++i) z += W1[o * D + i] * round_bf16(x[p * D + i]);
      a1[o] = rbf(silu(z));
    }
    for (int o = 0; o < H; ++o) {
      cplx z = b2[o];
      for (int i = 0; i < H; ++i) z += W2[o * H + i] * a1[i];
      a2[o] = rbf(silu(z));
    }
    cplx y = b3[0];
    for (int i = 0; i < H; ++i) y += w3[i] * a2[i];
    cplx r = y - t[p];
    L += r * r;
  }
  (void)Pr;
  return (L / (double)n).imag() / CS_H;
}

}  // extern "C"
