// Helpers shared by the emitters (pyro_emit.cpp: thread-per-state kernels;
// pyro_emit_warp.cpp: warp-per-state kernels): literals, the FP64-pipe operation
// tally, per-species NASA-7 coefficient sets and stoichiometry helpers.
#pragma once

#include <cmath>
#include <cstdio>
#include <map>
#include <sstream>
#include <string>
#include <utility>
#include <vector>

#include "pyro_mech.h"

namespace pyro {
namespace emitc {

const long double R_GAS = 8314.462618L;   // J/(kmol K)
const long double P_ATM = 101325.0L;      // Pa

inline std::string lit(double x) {
  char b[64];
  std::snprintf(b, sizeof b, "%.17e", x);
  return b;
}
inline std::string litf(double x) {
  char b[64];
  std::snprintf(b, sizeof b, "%.9ef", x);
  return b;
}

struct Src {
  std::ostringstream o;
  // FP64 pipe ops emitted in the straight-line per-point path
  double dfma = 0, dadd = 0, dmul = 0;
  void fma(int n = 1) { dfma += n; }
  void add(int n = 1) { dadd += n; }
  void mul(int n = 1) { dmul += n; }
  void exp_();                                     // device exponential (see g_exp_ops)
  void log_() { dfma += 5; dadd += 1; dmul += 1; }  // pdm::log
  void rcp_() { dfma += 4; }                       // pdm::rcp
  double ops() const { return dfma + dadd + dmul; }
  double flops() const { return 2 * dfma + dadd + dmul; }
  template <class T> Src& operator<<(const T& v) { o << v; return *this; }
};

inline int g_exp_ops = 4;   // FP64-pipe operations of the device exponential in use
inline void Src::exp_() {
  if (g_exp_ops == 4) { dfma += 3; dmul += 1; } else { dfma += 2; }
}

// Per-species, per-range coefficient sets.
struct SpeciesCoef {
  // L_k = ln(phi_k/W_k) = cl*lnT + ci/T + c0 + T*(c1 + T*(c2 + T*(c3 + T*c4)))
  double cl[2], ci[2], c0[2], c1[2], c2[2], c3[2], c4[2];
  // e_k/R per unit mass fraction: d0 + d1 T + ... + d5 T^5  (= (h_k/R - T)/W_k)
  double d[2][6];
  // h_k/(R T) = h0 + T*(h1 + T*(h2 + T*(h3 + T*h4))) + h5/T
  double h[2][6];
  // cp_k/R = p0 + T*(p1 + T*(p2 + T*(p3 + T*p4))),  d(cp_k/R)/dT = q0 + T*(q1 + T*(q2 + T*q3))
  double cp[2][5], cpd[2][4];
};

inline SpeciesCoef species_coef(const Species& s) {
  SpeciesCoef c;
  long double lnRp0 = logl(R_GAS / P_ATM);
  long double lnW = logl((long double)s.W);
  for (int r = 0; r < 2; ++r) {
    const double* a = r == 0 ? s.low : s.high;
    c.cl[r] = (double)(1.0L - a[0]);
    c.ci[r] = a[5];
    c.c0[r] = (double)((long double)a[0] - a[6] + lnRp0 - lnW);
    c.c1[r] = (double)(-(long double)a[1] / 2);
    c.c2[r] = (double)(-(long double)a[2] / 6);
    c.c3[r] = (double)(-(long double)a[3] / 12);
    c.c4[r] = (double)(-(long double)a[4] / 20);
    long double W = s.W;
    c.d[r][0] = (double)(a[5] / W);
    c.d[r][1] = (double)((a[0] - 1.0L) / W);
    c.d[r][2] = (double)(a[1] / (2 * W));
    c.d[r][3] = (double)(a[2] / (3 * W));
    c.d[r][4] = (double)(a[3] / (4 * W));
    c.d[r][5] = (double)(a[4] / (5 * W));
    c.h[r][0] = a[0];
    c.h[r][1] = (double)((long double)a[1] / 2);
    c.h[r][2] = (double)((long double)a[2] / 3);
    c.h[r][3] = (double)((long double)a[3] / 4);
    c.h[r][4] = (double)((long double)a[4] / 5);
    c.h[r][5] = a[5];
    for (int q = 0; q < 5; ++q) c.cp[r][q] = a[q];
    for (int q = 0; q < 4; ++q) c.cpd[r][q] = (q + 1) * a[q + 1];
  }
  return c;
}

// select between the two ranges (hi: bool variable in scope)
inline std::string sel(const double v[2]) {
  if (v[0] == v[1]) return lit(v[0]);
  return "(hi ? " + lit(v[1]) + " : " + lit(v[0]) + ")";
}


// net stoichiometric coefficients of a reaction
inline std::map<int, int> net_nu(const Reaction& r) {
  std::map<int, int> nu;
  for (auto& p : r.products) nu[p.first] += p.second;
  for (auto& p : r.reactants) nu[p.first] -= p.second;
  return nu;
}

// factors of a side with multiplicity
inline std::vector<int> side_factors(const std::vector<std::pair<int, int>>& side) {
  std::vector<int> f;
  for (auto& p : side) for (int i = 0; i < p.second; ++i) f.push_back(p.first);
  return f;
}

inline bool has_plog(const Mechanism& m) {
  for (auto& r : m.reactions) if (r.kind == RX_PLOG) return true;
  return false;
}

inline bool common_tmid(const Mechanism& m) {
  for (auto& sp : m.species) if (sp.t_mid != m.species[0].t_mid) return false;
  return true;
}

}  // namespace emitc
}  // namespace pyro
