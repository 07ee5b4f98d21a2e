// Emitter: mechanism -> CUDA C specialised to that mechanism (sm_103a).
//
// Work split: one thread per state point, straight-line code per species and per
// reaction with every mechanism constant folded into immediates.  Per-point
// species quantities are staged in shared memory in [species][thread] layout
// (conflict-free), net production rates accumulate in registers.
//
// Arithmetic (the FP64 pipe is the bound; counts are tallied in EmitResult.stats):
//
//  * Species (Sec. A.1 Eq. gibbs, Eq. nasa_poly): with
//      phi_k = (R T / p0) exp(g_k / (R T)),
//    Eq. equil_constants gives 1/K_j = prod_k phi_k^{nu_kj} exactly, so with
//    activities a_k = phi_k C_k the law of mass action (Eq. reaction_rates) is
//      R_j = k_j / prod_k phi_k^{nu'_kj} * (prod a^{nu'} - prod a^{nu''}).
//    Per species the kernel forms L_k = ln(phi_k / W_k) (one 6-FMA polynomial in
//    T, ln T, 1/T) and a_k = exp(L_k) * rho Y_k (Eq. concentrations folded).
//  * Per reaction one exponential of
//      ln A_j - sum nu'_ij ln W_i + b_j ln T - theta_j / T - sum nu'_ij L_i,
//    products of activities, one difference, one multiply, and +-nu R_j into the
//    production rates (Eq. production_rates).  Duplicate reactions share the
//    activity products.
//  * Third-body concentration [M]_j = rho (sum_k Y_k/W_k + sum_eff (eps-1) Y_k/W_k);
//    Troe falloff (k = k_inf Pr/(1+Pr) F) with log F = log Fcent den^2/(den^2+x^2),
//    x = log10 Pr + c, den = n - 0.14 x, which equals the usual
//    log Fcent / (1 + (x/den)^2) without the division by den.
//  * Temperature from internal energy (Sec. A.3.1 Eq. int_energy, Eq. delta_temp):
//    the species polynomials are collapsed into one mixture polynomial per NASA
//    range, e(T)/R = sum_m B_m T^m with B_m = sum_k Y_k d_km; Newton iterations
//    first in FP32 (until |dT| <= 1e-5 T), then in FP64 with the FP32 c_v as the
//    Newton slope until |dT| <= tol T, plus one further step.
#include "pyro_emit.h"

#include <cmath>
#include <cstdio>
#include <set>
#include <sstream>

namespace pyro {

namespace {

const long double R_GAS = 8314.462618L;   // J/(kmol K)
const long double P_ATM = 101325.0L;      // Pa

std::string lit(double x) {
  char b[64];
  std::snprintf(b, sizeof b, "%.17e", x);
  return b;
}
std::string litf(double x) {
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
  void exp_() { dfma += 3; dmul += 1; }           // pdm::exp: 3 DFMA + 1 DMUL
  void log_() { dfma += 5; dadd += 1; dmul += 1; }  // pdm::log
  void rcp_() { dfma += 4; }                       // pdm::rcp
  double ops() const { return dfma + dadd + dmul; }
  double flops() const { return 2 * dfma + dadd + dmul; }
  template <class T> Src& operator<<(const T& v) { o << v; return *this; }
};

// Per-species, per-range coefficient sets.
struct SpeciesCoef {
  // L_k = ln(phi_k/W_k) = cl*lnT + ci/T + c0 + T*(c1 + T*(c2 + T*(c3 + T*c4)))
  double cl[2], ci[2], c0[2], c1[2], c2[2], c3[2], c4[2];
  // e_k/R per unit mass fraction: d0 + d1 T + ... + d5 T^5  (= (h_k/R - T)/W_k)
  double d[2][6];
};

SpeciesCoef species_coef(const Species& s) {
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
  }
  return c;
}

// select between the two ranges (hi: bool variable in scope)
std::string sel(const double v[2]) {
  if (v[0] == v[1]) return lit(v[0]);
  return "(hi ? " + lit(v[1]) + " : " + lit(v[0]) + ")";
}

void emit_prelude(Src& s, const Mechanism& m, const EmitOptions& opt) {
  int N = m.n_species();
  s << "// Generated for mechanism '" << m.name << "': " << N << " species, "
    << m.n_reactions() << " reactions.\n";
  s << "#include \"pyro_device_math.cuh\"\n";
  s << "typedef long long i64;\n";
  s << "#define BLK " << opt.block << "\n#define NSP " << N << "\n";
  s << "#define MINB " << opt.min_blocks << "\n";
  s << "#define TMID " << lit(m.species.empty() ? 1000.0 : m.species[0].t_mid) << "\n";
  s << "__constant__ double pyro_tab_exp[512] = {";
  for (int j = 0; j < 512; ++j) s << (j ? "," : "") << lit((double)exp2l((j + 0.5L) / 512.0L));
  s << "};\n__constant__ double pyro_tab_log[256] = {";
  for (int j = 0; j < 128; ++j) {
    long double c = 1.0L + (j + 0.5L) / 128.0L;
    s << (j ? "," : "") << lit((double)(1.0L / c)) << "," << lit((double)logl(c));
  }
  s << "};\n";
  s << R"(
__device__ __forceinline__ void pyro_load_tables(double* se, double* sl) {
  for (int i = threadIdx.x; i < 512; i += blockDim.x) se[i] = pyro_tab_exp[i];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) sl[i] = pyro_tab_log[i];
}
)";
}

// ---------------------------------------------------------------------------
// temperature solve
// ---------------------------------------------------------------------------

bool common_tmid(const Mechanism& m) {
  for (auto& sp : m.species) if (sp.t_mid != m.species[0].t_mid) return false;
  return true;
}

void emit_tsolve(Src& s, const Mechanism& m, const std::vector<SpeciesCoef>& C, const EmitOptions& opt,
                 std::map<std::string, double>& st) {
  int N = m.n_species();
  // FP32 collapse (both ranges) and FP64 collapse (one range)
  s << "// Newton inversion of e = sum_k Y_k e_k(T) (Sec. A.3.1, Eq. delta_temp); returns T,\n"
       "// writes the iteration count (FP32 + FP64 steps) or -1 if max_iter FP64 steps\n"
       "// did not meet |dT| <= tol T.\n";
  s << "__device__ __forceinline__ double pyro_tsolve(const double* __restrict__ Yp, i64 n, double e,\n"
       "    double T0, int max_iter, float tolf, int* iters) {\n";
  s << "  const double eR = e * " << lit((double)(1.0L / R_GAS)) << ";\n";
  Src dummy;
  s << "  float bl0=0.f,bl1=0.f,bl2=0.f,bl3=0.f,bl4=0.f,bl5=0.f,bh0=0.f,bh1=0.f,bh2=0.f,bh3=0.f,bh4=0.f,bh5=0.f;\n";
  for (int k = 0; k < N; ++k) {
    s << "  { float y = pdm::to_float_trunc(__ldg(Yp + (i64)" << k << " * n));";
    for (int q = 0; q < 6; ++q) s << " bl" << q << " = fmaf(y, " << litf(C[k].d[0][q]) << ", bl" << q << ");";
    for (int q = 0; q < 6; ++q) s << " bh" << q << " = fmaf(y, " << litf(C[k].d[1][q]) << ", bh" << q << ");";
    s << " }\n";
  }
  s << R"(  float Tf = pdm::to_float_trunc(T0);
  const float eRf = pdm::to_float_trunc(eR);
  int it32 = 0;
  if (opt_mixed) {
    for (; it32 < 40; ) {
      ++it32;
      bool hf = Tf >= (float)TMID;
      float c0 = hf ? bh0 : bl0, c1 = hf ? bh1 : bl1, c2 = hf ? bh2 : bl2;
      float c3 = hf ? bh3 : bl3, c4 = hf ? bh4 : bl4, c5 = hf ? bh5 : bl5;
      float ef = fmaf(Tf, fmaf(Tf, fmaf(Tf, fmaf(Tf, fmaf(Tf, c5, c4), c3), c2), c1), c0);
      float cvf = fmaf(Tf, fmaf(Tf, fmaf(Tf, fmaf(Tf, 5.f * c5, 4.f * c4), 3.f * c3), 2.f * c2), c1);
      float dT = (eRf - ef) * __frcp_rn(cvf);
      float Tn = fminf(fmaxf(Tf + dT, 100.f), 5000.f);
      bool conv = fabsf(Tn - Tf) <= 1e-5f * Tn;
      Tf = Tn;
      if (conv) break;
    }
  }
  double T = opt_mixed ? pdm::to_double(Tf) : T0;
  bool hi = pdm::to_float_trunc(T) >= (float)TMID;
  double B0, B1, B2, B3, B4, B5;
)";
  // collapse macro for a given range flag 'hi'
  s << "  auto collapse = [&](bool hi) {\n    B0 = 0.0; B1 = 0.0; B2 = 0.0; B3 = 0.0; B4 = 0.0; B5 = 0.0;\n";
  for (int k = 0; k < N; ++k) {
    s << "    { double y = __ldg(Yp + (i64)" << k << " * n);";
    for (int q = 0; q < 6; ++q) {
      double v[2] = {C[k].d[0][q], C[k].d[1][q]};
      s << " B" << q << " = fma(y, " << sel(v) << ", B" << q << ");";
    }
    s << " }\n";
  }
  s << "  };\n";
  st["tsolve_collapse_fp64_ops"] = 6.0 * N;
  s << R"(  collapse(hi);
  int it64 = 0;
  bool flag = false, ok = false;
  for (int it = 0; it < max_iter + 1; ++it) {
    ++it64;
    float Tcur = pdm::to_float_trunc(T);
    bool h2 = Tcur >= (float)TMID;
    if (h2 != hi) { hi = h2; collapse(hi); }
    double e64 = fma(T, fma(T, fma(T, fma(T, fma(T, B5, B4), B3), B2), B1), B0);
    double res = e64 - eR;
    double dT;
    if (opt_mixed) {
      float c0 = hi ? bh1 : bl1, c1 = hi ? bh2 : bl2, c2 = hi ? bh3 : bl3, c3 = hi ? bh4 : bl4, c4 = hi ? bh5 : bl5;
      float cvf = fmaf(Tcur, fmaf(Tcur, fmaf(Tcur, fmaf(Tcur, 5.f * c4, 4.f * c3), 3.f * c2), 2.f * c1), c0);
      dT = res * pdm::to_double(-__frcp_rn(cvf));
    } else {
      double cv = fma(T, fma(T, fma(T, 5.0 * B5 * T + 4.0 * B4, 3.0 * B3), 2.0 * B2), B1);
      dT = -res * pdm::rcp(cv);
    }
    double Tn = T + dT;
    float Tnf = pdm::to_float_trunc(Tn);
    bool clamped = !(Tnf >= 100.f && Tnf <= 5000.f);
    Tn = clamped ? (Tnf < 100.f ? 100.0 : 5000.0) : Tn;
    bool conv = !clamped && fabsf(pdm::to_float_trunc(dT)) <= tolf * pdm::to_float_trunc(Tn);
    T = Tn;
    if (flag) { ok = true; break; }
    if (conv) flag = true;
    else if (it >= max_iter - 1) break;
  }
  *iters = ok ? it32 + it64 : -1;
  return T;
}
)";
  // per-iteration FP64 costs
  st["tsolve_iter_fp64_ops_mixed"] = 5 + 1 + 1 + 1;            // Horner, res, dT, T+dT
  st["tsolve_iter_fp64_ops_fp64"] = 5 + 1 + 4 + 4 + 4 + 1 + 1;  // + cv Horner (4) + multiples (4) + rcp (4)
}

// ---------------------------------------------------------------------------
// species and reactions of the forward path
// ---------------------------------------------------------------------------

std::string sidx(int k) { return "[" + std::to_string(k) + " * BLK + t]"; }

void emit_species_forward(Src& s, const Mechanism& m, const std::vector<SpeciesCoef>& C) {
  int N = m.n_species();
  s << "    double ysum = 0.0;   // sum_k Y_k / W_k\n";
  for (int k = 0; k < N; ++k) {
    const SpeciesCoef& c = C[k];
    s << "    { const double y = __ldg(Yp + (i64)" << k << " * n);\n";
    s << "      double q = fma(T, " << sel(c.c4) << ", " << sel(c.c3) << ");\n";
    s << "      q = fma(T, q, " << sel(c.c2) << "); q = fma(T, q, " << sel(c.c1) << "); q = fma(T, q, " << sel(c.c0) << ");\n";
    s << "      q = fma(" << sel(c.cl) << ", lnT, q); q = fma(" << sel(c.ci) << ", invT, q);\n";
    s.fma(6);
    s << "      sL" << sidx(k) << " = q;\n";
    s << "      sA" << sidx(k) << " = pdm::exp(q, s_exp) * (rho * y);\n";
    s.exp_(); s.mul(2);
    s << "      ysum = fma(y, " << lit(1.0 / m.species[k].W) << ", ysum); }\n";
    s.fma(1);
  }
}

// net stoichiometric coefficients of a reaction
std::map<int, int> net_nu(const Reaction& r) {
  std::map<int, int> nu;
  for (auto& p : r.products) nu[p.first] += p.second;
  for (auto& p : r.reactants) nu[p.first] -= p.second;
  return nu;
}

std::string product_expr(Src& s, const std::vector<std::pair<int, int>>& side) {
  std::string e;
  int nf = 0;
  for (auto& p : side)
    for (int i = 0; i < p.second; ++i) {
      e += (nf ? " * " : "") + std::string("sA") + sidx(p.first);
      ++nf;
    }
  s.mul(nf - 1);
  return e;
}

// ln of the Arrhenius part of k~ minus species terms: emits "double x = ..."
void emit_arg(Src& s, const Mechanism& m, const Reaction& r, double A, double b, double theta,
              const std::string& var) {
  long double lnA = logl((long double)A);
  for (auto& p : r.reactants) lnA -= p.second * logl((long double)m.species[p.first].W);
  s << "      double " << var << " = fma(" << lit(b) << ", lnT, " << lit((double)lnA) << ");";
  s << " " << var << " = fma(" << lit(-theta) << ", invT, " << var << ");";
  s.fma(2);
  for (auto& p : r.reactants) {
    if (p.second == 1) { s << " " << var << " -= sL" << sidx(p.first) << ";"; s.add(); }
    else { s << " " << var << " = fma(" << lit(-(double)p.second) << ", sL" << sidx(p.first) << ", " << var << ");"; s.fma(); }
  }
  s << "\n";
}

void emit_omega_update(Src& s, const Reaction& r, const std::string& R) {
  for (auto& q : net_nu(r)) {
    if (q.second == 0) continue;
    if (q.second == 1) { s << " w" << q.first << " += " << R << ";"; s.add(); }
    else if (q.second == -1) { s << " w" << q.first << " -= " << R << ";"; s.add(); }
    else { s << " w" << q.first << " = fma(" << lit((double)q.second) << ", " << R << ", w" << q.first << ");"; s.fma(); }
  }
  s << "\n";
}

void emit_third_body(Src& s, const Mechanism& m, const Reaction& r) {
  // [M] = rho * (ysum + sum_eff (eps - 1) Y_k / W_k)
  s << "      double mtb = ysum;";
  for (auto& e : r.efficiencies) {
    double c = (e.second - 1.0) / m.species[e.first].W;
    if (c == 0.0) continue;
    s << " mtb = fma(__ldg(Yp + (i64)" << e.first << " * n), " << lit(c) << ", mtb);";
    s.fma();
  }
  s << " mtb *= rho;\n";
  s.mul();
}

void emit_reaction_group(Src& s, const Mechanism& m, const std::vector<int>& grp) {
  const Reaction& r = m.reactions[grp[0]];
  s << "    { // reaction";
  for (int j : grp) s << " " << j;
  s << (r.kind == RX_THREEBODY ? " (three-body)" : r.kind == RX_FALLOFF ? " (falloff)" : "") << "\n";
  // k~ (sum over duplicates)
  for (size_t q = 0; q < grp.size(); ++q) {
    const Reaction& rq = m.reactions[grp[q]];
    emit_arg(s, m, rq, rq.A, rq.b, rq.theta, "x" + std::to_string(q));
  }
  s << "      double kt = pdm::exp(x0, s_exp);";
  s.exp_();
  for (size_t q = 1; q < grp.size(); ++q) { s << " kt += pdm::exp(x" << q << ", s_exp);"; s.exp_(); s.add(); }
  s << "\n";
  if (r.kind == RX_THREEBODY) {
    emit_third_body(s, m, r);
    s << "      kt *= mtb;\n";
    s.mul();
  } else if (r.kind == RX_FALLOFF) {
    emit_third_body(s, m, r);
    // ln Pr = ln k0 - ln kinf + ln [M]
    s << "      double lnPr = fma(" << lit(r.b0 - r.b) << ", lnT, " << lit((double)(logl(r.A0) - logl(r.A))) << ");";
    s << " lnPr = fma(" << lit(-(r.theta0 - r.theta)) << ", invT, lnPr); lnPr += pdm::log(mtb, s_log);\n";
    s.fma(2); s.log_(); s.add();
    // Pr/(1+Pr) = 1/(1 + exp(-ln Pr))
    s << "      double fpr = pdm::rcp(1.0 + pdm::exp(-lnPr, s_exp));\n";
    s.exp_(); s.add(); s.rcp_();
    if (r.n_troe >= 3) {
      double a = r.troe[0], T3 = r.troe[1], T1 = r.troe[2];
      s << "      double fc = ";
      if (a < 1.0) {
        s << "pdm::exp(fma(T, " << lit(-1.0 / T3) << ", " << lit((double)logl(1.0L - a)) << "), s_exp)";
        s.fma(); s.exp_();
      } else {
        s << lit(1.0 - a) << " * pdm::exp(T * " << lit(-1.0 / T3) << ", s_exp)";
        s.mul(2); s.exp_();
      }
      if (a > 0.0) {
        s << " + pdm::exp(fma(T, " << lit(-1.0 / T1) << ", " << lit((double)logl((long double)a)) << "), s_exp)";
        s.fma(); s.exp_(); s.add();
      }
      if (r.n_troe == 4) {
        s << " + pdm::exp(" << lit(-r.troe[3]) << " * invT, s_exp)";
        s.mul(); s.exp_(); s.add();
      }
      s << ";\n";
      const double inv_ln10 = (double)(1.0L / logl(10.0L));
      s << "      double lfc = pdm::log(fc, s_log) * " << lit(inv_ln10) << ";\n";
      s.log_(); s.mul();
      s << "      double cc = fma(-0.67, lfc, -0.4); double nn = fma(-1.27, lfc, 0.75);\n";
      s.fma(2);
      s << "      double xx = fma(lnPr, " << lit(inv_ln10) << ", cc); double den = fma(-0.14, xx, nn);\n";
      s.fma(2);
      s << "      double den2 = den * den; double lf = lfc * den2 * pdm::rcp(fma(xx, xx, den2));\n";
      s.mul(3); s.fma(); s.rcp_();
      s << "      double F = pdm::exp(lf * " << lit((double)logl(10.0L)) << ", s_exp);\n";
      s.mul(); s.exp_();
      s << "      kt *= fpr * F;\n";
      s.mul(2);
    } else {
      s << "      kt *= fpr;\n";
      s.mul();
    }
  }
  std::string pf = product_expr(s, r.reactants);
  if (r.reversible) {
    std::string pr = product_expr(s, r.products);
    s << "      const double R = kt * (" << pf << " - " << pr << ");\n";
    s.add(); s.mul();
  } else {
    s << "      const double R = kt * (" << pf << ");\n";
    s.mul();
  }
  s << "     ";
  emit_omega_update(s, r, "R");
  s << "    }\n";
}

// group plain reversible duplicates with identical stoichiometry
std::vector<std::vector<int>> reaction_groups(const Mechanism& m) {
  std::vector<std::vector<int>> g;
  std::vector<bool> used(m.n_reactions(), false);
  for (int j = 0; j < m.n_reactions(); ++j) {
    if (used[j]) continue;
    std::vector<int> grp{j};
    used[j] = true;
    const Reaction& r = m.reactions[j];
    if (r.duplicate && r.kind == RX_ARRHENIUS) {
      for (int q = j + 1; q < m.n_reactions(); ++q) {
        const Reaction& o = m.reactions[q];
        if (!used[q] && o.duplicate && o.kind == RX_ARRHENIUS && o.reversible == r.reversible &&
            o.reactants == r.reactants && o.products == r.products) {
          grp.push_back(q);
          used[q] = true;
        }
      }
    }
    g.push_back(grp);
  }
  return g;
}

}  // namespace

EmitResult emit_module(const Mechanism& m, const EmitOptions& opt) {
  EmitResult out;
  Src s;
  int N = m.n_species();
  std::vector<SpeciesCoef> C;
  for (auto& sp : m.species) C.push_back(species_coef(sp));
  emit_prelude(s, m, opt);
  s << "#define opt_mixed " << (opt.mixed_newton ? 1 : 0) << "\n";
  emit_tsolve(s, m, C, opt, out.stats);

  // ---- diagnostic math kernel -------------------------------------------------
  s << R"(
extern "C" __global__ void __launch_bounds__(BLK) pyro_math(int fn, i64 n, const double* __restrict__ x,
    double* __restrict__ y) {
  __shared__ double s_exp[512];
  __shared__ double s_log[256];
  pyro_load_tables(s_exp, s_log);
  __syncthreads();
  for (i64 p = (i64)blockIdx.x * BLK + threadIdx.x; p < n; p += (i64)gridDim.x * BLK) {
    double v = x[p];
    y[p] = fn == 0 ? pdm::exp(v, s_exp) : fn == 1 ? pdm::log(v, s_log) : pdm::rcp(v);
  }
}
)";

  // ---- density (Eq. eos) -------------------------------------------------------
  s << "\nextern \"C\" __global__ void __launch_bounds__(BLK) pyro_density(i64 n, const double* __restrict__ g_p,\n"
       "    const double* __restrict__ g_T, const double* __restrict__ g_Y, double* __restrict__ g_rho) {\n"
       "  for (i64 p = (i64)blockIdx.x * BLK + threadIdx.x; p < n; p += (i64)gridDim.x * BLK) {\n"
       "    const double* Yp = g_Y + p;\n    double ys = 0.0;\n";
  for (int k = 0; k < N; ++k)
    s << "    ys = fma(__ldg(Yp + (i64)" << k << " * n), " << lit(1.0 / m.species[k].W) << ", ys);\n";
  s << "    g_rho[p] = g_p[p] * pdm::rcp(" << lit((double)R_GAS) << " * g_T[p] * ys);\n  }\n}\n";

  // ---- internal energy and c_v (Eq. int_energy, Eq. cv) -------------------------
  s << "\nextern \"C\" __global__ void __launch_bounds__(BLK) pyro_energy(i64 n, const double* __restrict__ g_T,\n"
       "    const double* __restrict__ g_Y, double* __restrict__ g_e, double* __restrict__ g_cv) {\n"
       "  for (i64 p = (i64)blockIdx.x * BLK + threadIdx.x; p < n; p += (i64)gridDim.x * BLK) {\n"
       "    const double* Yp = g_Y + p;\n    const double T = g_T[p];\n"
       "    const bool hi = pdm::to_float_trunc(T) >= (float)TMID;\n"
       "    double B0 = 0.0, B1 = 0.0, B2 = 0.0, B3 = 0.0, B4 = 0.0, B5 = 0.0;\n";
  for (int k = 0; k < N; ++k) {
    s << "    { double y = __ldg(Yp + (i64)" << k << " * n);";
    for (int q = 0; q < 6; ++q) {
      double v[2] = {C[k].d[0][q], C[k].d[1][q]};
      s << " B" << q << " = fma(y, " << sel(v) << ", B" << q << ");";
    }
    s << " }\n";
  }
  s << "    g_e[p] = " << lit((double)R_GAS) << " * fma(T, fma(T, fma(T, fma(T, fma(T, B5, B4), B3), B2), B1), B0);\n"
       "    if (g_cv) g_cv[p] = " << lit((double)R_GAS)
    << " * fma(T, fma(T, fma(T, fma(T, 5.0 * B5, 4.0 * B4), 3.0 * B3), 2.0 * B2), B1);\n  }\n}\n";

  // ---- temperature --------------------------------------------------------------
  s << R"(
extern "C" __global__ void __launch_bounds__(BLK) pyro_temperature(i64 n, const double* __restrict__ g_e,
    const double* __restrict__ g_Y, const double* __restrict__ g_guess, double T_guess, int max_iter, double tol,
    double* __restrict__ g_T, int* __restrict__ g_iters, unsigned long long* __restrict__ g_fail) {
  const float tolf = (float)tol;
  for (i64 p = (i64)blockIdx.x * BLK + threadIdx.x; p < n; p += (i64)gridDim.x * BLK) {
    int it;
    double T = pyro_tsolve(g_Y + p, n, g_e[p], g_guess ? g_guess[p] : T_guess, max_iter, tolf, &it);
    g_T[p] = T;
    if (g_iters) g_iters[p] = it;
    if (it < 0) atomicAdd(g_fail, 1ull);
  }
}
)";

  // ---- net production rates (Eq. production_rates) ------------------------------
  Src r;   // count the forward per-point path separately
  r << "\nextern \"C\" __global__ void __launch_bounds__(BLK, MINB) pyro_omega(i64 n, const double* __restrict__ g_rho,\n"
       "    const double* __restrict__ g_Tin, int energy_mode, const double* __restrict__ g_Y,\n"
       "    double* __restrict__ g_Tout, double* __restrict__ g_omega, double T_guess, int max_iter, double tol,\n"
       "    unsigned long long* __restrict__ g_fail) {\n"
       "  __shared__ double s_exp[512];\n  __shared__ double s_log[256];\n"
       "  extern __shared__ double s_dyn[];\n"
       "  double* sL = s_dyn;\n  double* sA = s_dyn + NSP * BLK;\n"
       "  pyro_load_tables(s_exp, s_log);\n  __syncthreads();\n"
       "  const int t = threadIdx.x;\n  const float tolf = (float)tol;\n"
       "  for (i64 p = (i64)blockIdx.x * BLK + t; p < n; p += (i64)gridDim.x * BLK) {\n"
       "    const double* Yp = g_Y + p;\n    const double rho = g_rho[p];\n"
       "    double T;\n"
       "    if (energy_mode) {\n      int it;\n"
       "      T = pyro_tsolve(Yp, n, g_Tin[p], T_guess, max_iter, tolf, &it);\n"
       "      if (it < 0) atomicAdd(g_fail, 1ull);\n      if (g_Tout) g_Tout[p] = T;\n"
       "    } else {\n      T = g_Tin[p];\n    }\n"
       "    const double lnT = pdm::log(T, s_log);\n    const double invT = pdm::rcp(T);\n"
       "    const bool hi = pdm::to_float_trunc(T) >= (float)TMID;\n";
  r.log_(); r.rcp_();
  emit_species_forward(r, m, C);
  r << "    double ";
  for (int k = 0; k < N; ++k) r << (k ? ", " : "") << "w" << k << " = 0.0";
  r << ";\n";
  for (auto& grp : reaction_groups(m)) emit_reaction_group(r, m, grp);
  for (int k = 0; k < N; ++k) r << "    g_omega[(i64)" << k << " * n + p] = w" << k << ";\n";
  r << "  }\n}\n";
  s << r.o.str();

  out.stats["omega_fp64_ops_per_point"] = r.ops();
  out.stats["omega_fp64_flops_per_point"] = r.flops();
  out.stats["omega_dfma_per_point"] = r.dfma;
  out.stats["omega_dadd_per_point"] = r.dadd;
  out.stats["omega_dmul_per_point"] = r.dmul;
  out.stats["n_species"] = N;
  out.stats["n_reactions"] = m.n_reactions();
  out.stats["block"] = opt.block;
  out.smem_dyn_bytes_omega = 2 * N * opt.block * (int)sizeof(double);
  out.source = s.o.str();
  return out;
}

}  // namespace pyro
