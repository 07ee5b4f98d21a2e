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
#include "pyro_emit_common.h"
#include "pyro_emit_warp.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <set>
#include <sstream>

namespace pyro {

namespace {
using namespace emitc;

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
// An opaque copy of a value: keeps the compiler from hoisting and keeping alive
// hundreds of address computations across the straight-line code.
__device__ __forceinline__ i64 opq(i64 v) { asm volatile("" : "+l"(v)); return v; }
)";
  // exponential flavour: 2 or 4 FP64 operations, inlined or one shared (called) body
  if (opt.exp_call)
    s << "__device__ __noinline__ double pyro_exp_call(double x, const double* __restrict__ t) { return pdm::"
      << (opt.exp_ops == 4 ? "exp4" : "exp") << "(x, t); }\n#define PEXP(x, t) pyro_exp_call((x), (t))\n";
  else
    s << "#define PEXP(x, t) pdm::" << (opt.exp_ops == 4 ? "exp4" : "exp") << "((x), (t))\n";
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


void emit_tsolve(Src& s, const Mechanism& m, const std::vector<SpeciesCoef>& C, const EmitOptions& opt,
                 std::map<std::string, double>& st) {
  int N = m.n_species();
  // FP32 collapse (both ranges) and FP64 collapse (one range)
  s << "// Newton inversion of e = sum_k Y_k e_k(T) (Sec. A.3.1, Eq. delta_temp), or with\n"
       "// ENTH of h = sum_k Y_k h_k(T) (the enthalpy variant: the linear coefficient of each\n"
       "// species polynomial gains 1/W_k, c_v becomes c_p); returns T, writes the iteration\n"
       "// count (FP32 + FP64 steps) or -1 if max_iter FP64 steps did not meet |dT| <= tol T.\n";
  s << "template <bool ENTH>\n__device__ __forceinline__ double pyro_tsolve(const double* __restrict__ Yp, i64 n, double e,\n"
       "    double T0, int max_iter, float tolf, int* iters) {\n";
  s << "  const double eR = e * " << lit((double)(1.0L / R_GAS)) << ";\n";
  Src dummy;
  s << "  float bl0=0.f,bl1=0.f,bl2=0.f,bl3=0.f,bl4=0.f,bl5=0.f,bh0=0.f,bh1=0.f,bh2=0.f,bh3=0.f,bh4=0.f,bh5=0.f;\n";
  for (int k = 0; k < N; ++k) {
    const double invW = 1.0 / m.species[k].W;
    auto cf = [&](int r, int q) {
      if (q != 1) return litf(C[k].d[r][q]);
      return "(ENTH ? " + litf(C[k].d[r][1] + invW) + " : " + litf(C[k].d[r][1]) + ")";
    };
    s << "  { float y = pdm::to_float_trunc(__ldg(Yp + (i64)" << k << " * n));";
    for (int q = 0; q < 6; ++q) s << " bl" << q << " = fmaf(y, " << cf(0, q) << ", bl" << q << ");";
    for (int q = 0; q < 6; ++q) s << " bh" << q << " = fmaf(y, " << cf(1, q) << ", bh" << q << ");";
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
    const double invW = 1.0 / m.species[k].W;
    s << "    { double y = __ldg(Yp + (i64)" << k << " * n);";
    for (int q = 0; q < 6; ++q) {
      double v[2] = {C[k].d[0][q], C[k].d[1][q]};
      if (q == 1) {
        double vh[2] = {C[k].d[0][1] + invW, C[k].d[1][1] + invW};
        s << " B1 = fma(y, (ENTH ? " << sel(vh) << " : " << sel(v) << "), B1);";
      } else {
        s << " B" << q << " = fma(y, " << sel(v) << ", B" << q << ");";
      }
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
    s << "      sA" << sidx(k) << " = PEXP(q, s_exp) * (rho * y);\n";
    s.exp_(); s.mul(2);
    s << "      ysum = fma(y, " << lit(1.0 / m.species[k].W) << ", ysum); }\n";
    s.fma(1);
  }
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
// With folded: the reactant sum sum nu'_i L_i is the variable nuL in scope (formed
// from per-reaction folded coefficients) instead of per-species shared entries.
bool g_fold = false;

void emit_arg(Src& s, const Mechanism& m, const Reaction& r, double A, double b, double theta,
              const std::string& var) {
  long double lnA = logl((long double)A);
  for (auto& p : r.reactants) lnA -= p.second * logl((long double)m.species[p.first].W);
  s << "      double " << var << " = fma(" << lit(b) << ", lnT, " << lit((double)lnA) << ");";
  s << " " << var << " = fma(" << lit(-theta) << ", invT, " << var << ");";
  s.fma(2);
  if (g_fold) { s << " " << var << " -= nuL;\n"; s.add(); return; }
  for (auto& p : r.reactants) {
    if (p.second == 1) { s << " " << var << " -= sL" << sidx(p.first) << ";"; s.add(); }
    else { s << " " << var << " = fma(" << lit(-(double)p.second) << ", sL" << sidx(p.first) << ", " << var << ");"; s.fma(); }
  }
  s << "\n";
}


// PLOG exponent (standard form: ln k linear in ln p between the bracketing nodes,
// end nodes outside the node range) minus sum nu' L_i, into `var`.  Needs lnp =
// ln(R T rho sum_k Y_k/W_k) (Eq. eos) in scope.  The bracketing segment is chosen
// by FP64 comparisons, so both sides of a node pick values that agree to rounding.
// With deriv: also <var>_tau = d var/dT at fixed p-argument terms plus the
// pressure path d ln p/dT = 1/T, and <var>_pm = d var/d ln p (0 outside the range).
void emit_plog_arg(Src& s, const Mechanism& m, const Reaction& r, const std::string& var, bool deriv) {
  long double lnWs = 0;
  for (auto& p : r.reactants) lnWs += p.second * logl((long double)m.species[p.first].W);
  const int n = (int)r.plog.size();
  std::vector<double> la(n), lp(n), inv(n > 1 ? n - 1 : 1);
  for (int q = 0; q < n; ++q) {
    la[q] = (double)(logl((long double)r.plog[q].A) - lnWs);
    lp[q] = (double)logl((long double)r.plog[q].p);
  }
  for (int q = 0; q + 1 < n; ++q) inv[q] = (double)(1.0L / (logl((long double)r.plog[q + 1].p) - logl((long double)r.plog[q].p)));
  auto node = [&](int q, const char* sfx) {
    return "pla" + std::string(sfx) + " = " + lit(la[q]) + "; pb" + sfx + " = " + lit(r.plog[q].b) + "; pt" + sfx +
           " = " + lit(r.plog[q].theta) + ";";
  };
  s << "      double plaa, pba, pta, plab, pbb, ptb; " << node(0, "a") << " " << node(1, "b") << "\n";
  s << "      double plp = " << lit(lp[0]) << ", pinv = " << lit(inv[0]) << ";\n";
  for (int q = 1; q + 1 < n; ++q)
    s << "      if (lnp >= " << lit(lp[q]) << ") { " << node(q, "a") << " " << node(q + 1, "b") << " plp = "
      << lit(lp[q]) << "; pinv = " << lit(inv[q]) << "; }\n";
  s << "      double pxa = fma(pba, lnT, plaa); pxa = fma(-pta, invT, pxa);\n"
       "      double pxb = fma(pbb, lnT, plab); pxb = fma(-ptb, invT, pxb);\n"
       "      const double pfu = (lnp - plp) * pinv;\n"
       "      const double pf = fmin(fmax(pfu, 0.0), 1.0);\n"
       "      double " << var << " = fma(pf, pxb - pxa, pxa);";
  s.fma(5); s.add(3); s.mul(1); s.add(2 + (n > 2 ? n - 2 : 0));
  if (g_fold) { s << " " << var << " -= nuL;"; s.add(); }
  else for (auto& p : r.reactants) {
    if (p.second == 1) { s << " " << var << " -= sL" << sidx(p.first) << ";"; s.add(); }
    else { s << " " << var << " = fma(" << lit(-(double)p.second) << ", sL" << sidx(p.first) << ", " << var << ");"; s.fma(); }
  }
  s << "\n";
  if (deriv) {
    s.add(2); s.mul(3); s.fma(4);
    s << "      const double pdx = (pfu > 0.0 && pfu < 1.0) ? (pxb - pxa) * pinv : 0.0;\n"
         "      const double pta_ = fma(pba, invT, pta * invT2), ptb_ = fma(pbb, invT, ptb * invT2);\n"
         "      const double " << var << "_tau = fma(pdx, invT, fma(pf, ptb_ - pta_, pta_));\n"
         "      const double " << var << "_pm = pdx;\n";
  }
}

// SRI falloff factor (standard form): F = d [a exp(-b/T) + exp(-T/c)]^X T^e,
// X = 1/(1 + (log10 Pr)^2).  Needs lnPr, T, invT, lnT in scope; defines F and,
// with deriv, dlnF_dlnPr and dlnF_dT (at fixed Pr).
void emit_sri(Src& s, const Reaction& r, bool deriv) {
  const double inv_ln10 = (double)(1.0L / logl(10.0L));
  const double a = r.sri[0], b = r.sri[1], c = r.sri[2];
  const double d = r.n_sri >= 5 ? r.sri[3] : 1.0, e = r.n_sri >= 5 ? r.sri[4] : 0.0;
  s << "      const double su = lnPr * " << lit(inv_ln10) << ";\n"
       "      const double sX = pdm::rcp(fma(su, su, 1.0));\n";
  s.mul(); s.fma(); s.rcp_();
  if (a > 0.0) {
    s << "      const double sea = " << lit(a) << " * PEXP(" << lit(-b) << " * invT, s_exp);\n";
    s.mul(2); s.exp_();
  } else {
    s << "      const double sea = 0.0;\n";
  }
  s << "      const double seb = PEXP(T * " << lit(-1.0 / c) << ", s_exp);\n"
       "      const double sS = sea + seb;\n"
       "      const double slS = pdm::log(sS, s_log);\n"
       "      const double F = PEXP(fma(sX, slS, fma(" << lit(e) << ", lnT, " << lit((double)logl((long double)d))
    << ")), s_exp);\n";
  s.mul(); s.exp_(); s.add(); s.log_(); s.fma(2); s.exp_();
  if (deriv) {
    s.mul(9); s.fma(2); s.rcp_();
    s << "      const double dlnF_dlnPr = slS * (-2.0 * su * sX * sX * " << lit(inv_ln10) << ");\n"
         "      const double dlnF_dT = fma(sX * fma(sea, " << lit(b) << " * invT2, seb * " << lit(-1.0 / c)
      << "), pdm::rcp(sS), " << lit(e) << " * invT);\n";
  }
}

// Accumulators of the per-species sums (production rates, tangents, adjoints):
// named registers, or -- for large mechanisms -- the kernel's output array
// itself (read-modify-write through an opaque stride, L2-resident per block).
struct AccCfg {
  bool mem = false;
  std::string base;   // pointer to the point's entry of the output array
  std::string stride = "n";   // row stride of that array
};
AccCfg g_acc;

std::string acc(const std::string& name, int k) {
  if (!g_acc.mem) return name + std::to_string(k);
  return g_acc.base + "[(i64)" + std::to_string(k) + " * opq(" + g_acc.stride + ")]";
}

void emit_acc_init(Src& s, const std::string& name, int N) {
  if (!g_acc.mem) {
    s << "    double ";
    for (int k = 0; k < N; ++k) s << (k ? ", " : "") << name << k << " = 0.0";
    s << ";\n";
  } else {
    s << "    #pragma unroll 1\n    for (int k = 0; k < NSP; ++k) " << g_acc.base << "[(i64)k * " << g_acc.stride << "] = 0.0;\n";
  }
}

void emit_omega_update(Src& s, const Reaction& r, const std::string& R) {
  for (auto& q : net_nu(r)) {
    if (q.second == 0) continue;
    std::string a = acc("w", q.first);
    if (q.second == 1) { s << " " << a << " += " << R << ";"; s.add(); }
    else if (q.second == -1) { s << " " << a << " -= " << R << ";"; s.add(); }
    else { s << " " << a << " = fma(" << lit((double)q.second) << ", " << R << ", " << a << ");"; s.fma(); }
  }
  s << "\n";
}

void emit_third_body(Src& s, const Mechanism& m, const Reaction& r) {
  // [M] = rho * (ysum + sum_eff (eps - 1) Y_k / W_k)
  s << "      double mtb = ysum;";
  for (auto& e : r.efficiencies) {
    double c = (e.second - 1.0) / m.species[e.first].W;
    if (c == 0.0) continue;
    s << " mtb = fma(__ldg(Yp + (i64)" << e.first << " * opq(n)), " << lit(c) << ", mtb);";
    s.fma();
  }
  s << " mtb *= rho;\n";
  s.mul();
}

void emit_reaction_group(Src& s, const Mechanism& m, const std::vector<int>& grp) {
  const Reaction& r = m.reactions[grp[0]];
  s << "    { // reaction";
  for (int j : grp) s << " " << j;
  s << (r.kind == RX_THREEBODY ? " (three-body)" : r.kind == RX_FALLOFF ? " (falloff)"
        : r.kind == RX_PLOG ? " (plog)" : "") << "\n";
  // k~ (sum over duplicates)
  for (size_t q = 0; q < grp.size(); ++q) {
    const Reaction& rq = m.reactions[grp[q]];
    if (rq.kind == RX_PLOG) emit_plog_arg(s, m, rq, "x" + std::to_string(q), false);
    else emit_arg(s, m, rq, rq.A, rq.b, rq.theta, "x" + std::to_string(q));
  }
  s << "      double kt = PEXP(x0, s_exp);";
  s.exp_();
  for (size_t q = 1; q < grp.size(); ++q) { s << " kt += PEXP(x" << q << ", s_exp);"; s.exp_(); s.add(); }
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
    s << "      double fpr = pdm::rcp(1.0 + PEXP(-lnPr, s_exp));\n";
    s.exp_(); s.add(); s.rcp_();
    if (r.n_sri >= 3) {
      emit_sri(s, r, false);
      s << "      kt *= fpr * F;\n";
      s.mul(2);
    } else if (r.n_troe >= 3) {
      double a = r.troe[0], T3 = r.troe[1], T1 = r.troe[2];
      s << "      double fc = ";
      if (a < 1.0) {
        s << "PEXP(fma(T, " << lit(-1.0 / T3) << ", " << lit((double)logl(1.0L - a)) << "), s_exp)";
        s.fma(); s.exp_();
      } else {
        s << lit(1.0 - a) << " * PEXP(T * " << lit(-1.0 / T3) << ", s_exp)";
        s.mul(2); s.exp_();
      }
      if (a > 0.0) {
        s << " + PEXP(fma(T, " << lit(-1.0 / T1) << ", " << lit((double)logl((long double)a)) << "), s_exp)";
        s.fma(); s.exp_(); s.add();
      }
      if (r.n_troe == 4) {
        s << " + PEXP(" << lit(-r.troe[3]) << " * invT, s_exp)";
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
      s << "      double F = PEXP(lf * " << lit((double)logl(10.0L)) << ", s_exp);\n";
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

// ---------------------------------------------------------------------------
// derivative kernels (JVP, VJP, dense Jacobian)
// ---------------------------------------------------------------------------
//
// All three differentiate the same expression as the forward kernel:
//   R_j = kk_j (P'_j - P''_j),  kk_j = exp(x_j) g_j(T, M_j),  P' = prod a^{nu'},
//   a_i = exp(L_i(T)) rho Y_i,  x_j = lnA'_j + b_j ln T - theta_j / T - sum nu'_ij L_i,
// with g = 1 (plain), M (third body), Pr/(1+Pr) F (falloff), M_j = rho (sum_i eps_ij Y_i/W_i).
// Per reaction:  dR/dT = kk [D tau + P'' (S' - S'')],  tau = b/T + theta/T^2 + d ln g/dT,
// S = sum nu L'_i, L'_i = dL_i/dT = (1 - h_i/RT)/T;  dR/dM = D dkk/dM;  dR/dY_i through a_i
// (da_i/dY_i = exp(L_i) rho) and through M_j (dM_j/dY_i = rho eps_ij / W_i).

enum class DMode { JVP, VJP, JAC };

// per-species setup of the derivative kernels
void emit_species_deriv(Src& s, const Mechanism& m, const std::vector<SpeciesCoef>& C, DMode mode) {
  int N = m.n_species();
  s << "    double ysum = 0.0;\n";
  if (mode == DMode::JVP) s << "    double dysum = 0.0;\n";
  for (int k = 0; k < N; ++k) {
    const SpeciesCoef& c = C[k];
    s << "    { const double y = __ldg(Yp + (i64)" << k << " * n);\n";
    s << "      double q = fma(T, " << sel(c.c4) << ", " << sel(c.c3) << ");\n";
    s << "      q = fma(T, q, " << sel(c.c2) << "); q = fma(T, q, " << sel(c.c1) << "); q = fma(T, q, " << sel(c.c0) << ");\n";
    s << "      q = fma(" << sel(c.cl) << ", lnT, q); q = fma(" << sel(c.ci) << ", invT, q);\n";
    double h4[2] = {c.h[0][4], c.h[1][4]}, h3[2] = {c.h[0][3], c.h[1][3]}, h2[2] = {c.h[0][2], c.h[1][2]};
    double h1[2] = {c.h[0][1], c.h[1][1]}, h0[2] = {c.h[0][0], c.h[1][0]}, h5[2] = {c.h[0][5], c.h[1][5]};
    s << "      double hr = fma(T, " << sel(h4) << ", " << sel(h3) << "); hr = fma(T, hr, " << sel(h2)
      << "); hr = fma(T, hr, " << sel(h1) << "); hr = fma(T, hr, " << sel(h0) << "); hr = fma(" << sel(h5)
      << ", invT, hr);\n";
    s << "      const double Lp = fma(-hr, invT, invT);\n";
    s << "      const double E = PEXP(q, s_exp);\n";
    s << "      const double a = E * (rho * y);\n";
    s.fma(6); s.exp_(); s.mul(2);                      // L_k polynomial, exp, a_k
    if (mode != DMode::JAC) s.fma(6);                   // h_k/RT and L'_k (dead code in JAC mode)
    if (mode == DMode::JAC) { s << "      (void)Lp; sA" << sidx(k) << " = a; sE" << sidx(k) << " = E * rho;"; s.mul(); }
    else s << "      sL" << sidx(k) << " = q; sA" << sidx(k) << " = a;";
    if (mode == DMode::VJP) s << " sLp" << sidx(k) << " = Lp; sC" << sidx(k) << " = 0.0;";
    if (mode == DMode::JVP) {
      s << "\n      const double dy = __ldg(dYp + (i64)" << k << " * n);\n";
      s << "      sdA" << sidx(k) << " = fma(a, fma(Lp, dT, drr), E * (rho * dy)); sdL" << sidx(k) << " = Lp * dT;";
      s << " dysum = fma(dy, " << lit(1.0 / m.species[k].W) << ", dysum);";
      s.fma(3); s.mul(3);
    }
    s << "\n      ysum = fma(y, " << lit(1.0 / m.species[k].W) << ", ysum); }\n";
    s.fma();
  }
}


std::string prod_of(const std::vector<int>& f, const char* arr, int skip = -1) {
  std::string e;
  int nf = 0;
  for (int q = 0; q < (int)f.size(); ++q) {
    if (q == skip) continue;
    e += (nf ? " * " : "") + std::string(arr) + sidx(f[q]);
    ++nf;
  }
  return nf ? e : "1.0";
}

// d(prod a^{nu})/d(something) = sum over factor occurrences of (tangent of that factor) * others
std::string dprod(const std::vector<int>& f, const char* arr, const char* darr) {
  std::string e;
  for (int q = 0; q < (int)f.size(); ++q) {
    std::string o = prod_of(f, arr, q);
    e += (q ? " + " : "") + std::string(darr) + sidx(f[q]) + (o == "1.0" ? "" : " * " + o);
  }
  return "(" + e + ")";
}

// FP64 operations of dprod over nf factors: nf terms of (nf - 1) products, nf - 1 sums
void count_dprod(Src& s, int nf) {
  if (nf <= 1) return;
  s.mul(nf * (nf - 1));
  s.add(nf - 1);
}

// emits, inside a reaction block: x, kt, tau, [mS, M, kM], kk, Pf, Pr, D, R
void emit_reaction_core(Src& s, const Mechanism& m, const Reaction& r) {
  if (r.kind == RX_PLOG) {
    emit_plog_arg(s, m, r, "x", true);
    s << "      const double kt = PEXP(x, s_exp);\n";
    s << "      double tau = x_tau;\n";
    s.exp_();
  } else {
    emit_arg(s, m, r, r.A, r.b, r.theta, "x");
    s << "      const double kt = PEXP(x, s_exp);\n";
    s << "      double tau = fma(" << lit(r.b) << ", invT, " << lit(r.theta) << " * invT2);\n";
    s.exp_(); s.fma(); s.mul();
  }
  if (r.kind == RX_ARRHENIUS) {
    s << "      const double kk = kt;\n";
  } else if (r.kind == RX_PLOG) {
    // k depends on the total concentration M = rho sum Y/W through ln p = ln(R T M)
    s << "      const double mS = ysum;\n      const double M = rho * mS;\n"
         "      const double kk = kt; const double kM = kt * x_pm * pdm::rcp(M);\n";
    s.mul(3); s.rcp_();
  } else {
    s << "      double mS = ysum;";
    for (auto& e : r.efficiencies) {
      double c = (e.second - 1.0) / m.species[e.first].W;
      if (c != 0.0) { s << " mS = fma(__ldg(Yp + (i64)" << e.first << " * opq(n)), " << lit(c) << ", mS);"; s.fma(); }
    }
    s << "\n      const double M = rho * mS;\n";
    s.mul();
    if (r.kind == RX_THREEBODY) {
      s << "      const double kk = kt * M; const double kM = kt;\n";
      s.mul();
    } else {
      const double inv_ln10 = (double)(1.0L / logl(10.0L));
      s << "      const double lnPr = fma(" << lit(r.b0 - r.b) << ", lnT, " << lit((double)(logl(r.A0) - logl(r.A)))
        << ") + fma(" << lit(-(r.theta0 - r.theta)) << ", invT, pdm::log(M, s_log));\n";
      s << "      const double pT = fma(" << lit(r.b0 - r.b) << ", invT, " << lit(r.theta0 - r.theta) << " * invT2);\n";
      // 1 - Pr/(1+Pr) = q Pr/(1+Pr) with q = 1/Pr: formed as a product (the difference
      // cancels to nothing for Pr >> 1)
      s << "      const double qpr = PEXP(-lnPr, s_exp);\n      const double fpr = pdm::rcp(1.0 + qpr);\n"
           "      const double cpr = qpr * fpr;\n";
      s.fma(3); s.add(2); s.mul(2); s.log_(); s.exp_(); s.rcp_();   // lnPr, pT, fpr, 1 - fpr
      if (r.n_sri >= 3) {
        emit_sri(s, r, true);
        s << "      const double sPr = cpr + dlnF_dlnPr;\n";
        s << "      tau += fma(sPr, pT, dlnF_dT);\n";
        s << "      const double kk = kt * fpr * F;\n";
        s.add(3); s.fma(); s.mul(2);
      } else if (r.n_troe >= 3) {
        double a = r.troe[0], T3 = r.troe[1], T1 = r.troe[2];
        if (a < 1.0) {
          s << "      const double t1 = PEXP(fma(T, " << lit(-1.0 / T3) << ", " << lit((double)logl(1.0L - a)) << "), s_exp);\n";
          s.fma(); s.exp_();
        } else {
          s << "      const double t1 = " << lit(1.0 - a) << " * PEXP(T * " << lit(-1.0 / T3) << ", s_exp);\n";
          s.mul(2); s.exp_();
        }
        if (a > 0.0) {
          s << "      const double t2 = PEXP(fma(T, " << lit(-1.0 / T1) << ", " << lit((double)logl((long double)a)) << "), s_exp);\n";
          s.fma(); s.exp_();
        } else {
          s << "      const double t2 = 0.0;\n";
        }
        if (r.n_troe == 4) {
          s << "      const double t3 = PEXP(" << lit(-r.troe[3]) << " * invT, s_exp);\n";
          s.mul(); s.exp_();
        } else {
          s << "      const double t3 = 0.0;\n";
        }
        // fc, dfc, lfc, cc, nn, xx, den, den2, rD, f, F, rD2, Axx, Aden, sPr, sfc, tau, kk
        s.add(2); s.fma(2); s.mul(2); s.log_(); s.mul(); s.fma(4); s.mul(); s.fma(); s.rcp_(); s.mul(3); s.exp_();
        s.mul(1 + 4 + 5); s.fma(1); s.add(2); s.fma(2); s.fma(); s.mul(2); s.rcp_(); s.add(); s.mul(2);
        s << "      const double fc = t1 + t2 + t3;\n";
        s << "      const double dfc = fma(t1, " << lit(-1.0 / T3) << ", fma(t2, " << lit(-1.0 / T1) << ", t3 * "
          << lit(r.n_troe == 4 ? r.troe[3] : 0.0) << " * invT2));\n";
        s << "      const double lfc = pdm::log(fc, s_log) * " << lit(inv_ln10) << ";\n";
        s << "      const double cc = fma(-0.67, lfc, -0.4); const double nn = fma(-1.27, lfc, 0.75);\n";
        s << "      const double xx = fma(lnPr, " << lit(inv_ln10) << ", cc); const double den = fma(-0.14, xx, nn);\n";
        s << "      const double den2 = den * den; const double rD = pdm::rcp(fma(xx, xx, den2));\n";
        s << "      const double f = den2 * rD; const double F = PEXP(lfc * f * " << lit((double)logl(10.0L)) << ", s_exp);\n";
        s << "      const double rD2 = rD * rD;\n";
        s << "      const double Axx = lfc * (-2.0 * den2 * xx * rD2); const double Aden = lfc * (2.0 * den * xx * xx * rD2);\n";
        s << "      const double sPr = cpr + fma(-0.14, Aden, Axx);\n";
        s << "      const double sfc = fma(-0.67, Axx, fma(-1.1762, Aden, f));\n";
        s << "      tau += fma(sPr, pT, sfc * dfc * pdm::rcp(fc));\n";
        s << "      const double kk = kt * fpr * F;\n";
      } else {
        s << "      const double sPr = cpr;\n      tau += sPr * pT;\n      const double kk = kt * fpr;\n";
        s.add(2); s.mul(2);
      }
      s << "      const double kM = kk * sPr * pdm::rcp(M);\n";
      s.mul(2); s.rcp_();
    }
  }
  s << "      const double Pf = " << prod_of(side_factors(r.reactants), "sA") << ";\n";
  s.mul((int)side_factors(r.reactants).size() - 1);
  if (r.reversible) {
    s << "      const double Pr = " << prod_of(side_factors(r.products), "sA") << ";\n";
    s.mul((int)side_factors(r.products).size() - 1); s.add();
  } else {
    s << "      const double Pr = 0.0;\n";
  }
  s << "      const double D = Pf - Pr;\n      const double R = kk * D;\n";
  s.mul();
}

// net (nu'' - nu') over species of a reaction, and the set of species
std::vector<std::pair<int, int>> reaction_species(const Reaction& r) {
  std::vector<std::pair<int, int>> v;
  for (auto& q : net_nu(r)) v.push_back(q);
  return v;
}

int nu_of(const std::vector<std::pair<int, int>>& side, int k) {
  for (auto& p : side) if (p.first == k) return p.second;
  return 0;
}

void emit_jvp_kernel(Src& s, const Mechanism& m, const std::vector<SpeciesCoef>& C, int blk, const EmitOptions& opt) {
  int N = m.n_species();
  s << "\n// JVP: d omega = (d omega/d rho) d rho + (d omega/dT) dT + sum_i (d omega/dY_i) dY_i\n";
  s << "extern \"C\" __global__ void __launch_bounds__(" << blk << ") pyro_jvp(i64 n, const double* __restrict__ g_rho,\n"
       "    const double* __restrict__ g_T, const double* __restrict__ g_Y, const double* __restrict__ g_drho,\n"
       "    const double* __restrict__ g_dT, const double* __restrict__ g_dY, double* __restrict__ g_dw,\n"
       "    double* __restrict__ g_store) {\n"
       "  __shared__ double s_exp[512];\n  __shared__ double s_log[256];\n  extern __shared__ double s_dyn[];\n"
       "  double* sL = " << (opt.dgstore ? "g_store + (i64)blockIdx.x * 4 * NSP * BLKD" : "s_dyn") << ";\n"
       "  double* sA = sL + NSP * BLKD; double* sdA = sA + NSP * BLKD; double* sdL = sdA + NSP * BLKD;\n"
       "  pyro_load_tables(s_exp, s_log);\n  __syncthreads();\n  const int t = threadIdx.x;\n"
       "  for (i64 p = (i64)blockIdx.x * BLKD + t; p < n; p += (i64)gridDim.x * BLKD) {\n"
       "    const double* Yp = g_Y + p; const double* dYp = g_dY + p;\n"
       "    const double rho = g_rho[p], T = g_T[p], drho = g_drho[p], dT = g_dT[p];\n"
       "    const double lnT = pdm::log(T, s_log), invT = pdm::rcp(T), invT2 = invT * invT;\n"
       "    const double drr = drho * pdm::rcp(rho);\n"
       "    const bool hi = pdm::to_float_trunc(T) >= (float)TMID;\n";
  s.log_(); s.rcp_(); s.mul(); s.rcp_(); s.mul();
  emit_species_deriv(s, m, C, DMode::JVP);
  if (has_plog(m)) {
    s << "    const double lnp = lnT + pdm::log(rho * ysum, s_log) + " << lit((double)logl(R_GAS)) << ";\n";
    s.log_(); s.mul(); s.add(2);
  }
  g_acc.mem = opt.acc_mem;
  g_acc.base = "Wp";
  if (opt.acc_mem) s << "    double* Wp = g_dw + p;\n";
  emit_acc_init(s, "w", N);
  for (int j = 0; j < m.n_reactions(); ++j) {
    const Reaction& r = m.reactions[j];
    s << "    { // reaction " << j << "\n";
    emit_reaction_core(s, m, r);
    s << "      double dx = tau * dT;";
    s.mul();
    for (auto& p : r.reactants) { s << " dx = fma(" << lit(-(double)p.second) << ", sdL" << sidx(p.first) << ", dx);"; s.fma(); }
    s << "\n";
    if (r.kind == RX_ARRHENIUS) {
      s << "      const double dkk = kk * dx;\n";
      s.mul();
    } else {
      s << "      double dmS = dysum;";
      for (auto& e : r.efficiencies) {
        double c = (e.second - 1.0) / m.species[e.first].W;
        if (c != 0.0) { s << " dmS = fma(__ldg(dYp + (i64)" << e.first << " * opq(n)), " << lit(c) << ", dmS);"; s.fma(); }
      }
      s << "\n      const double dM = fma(drho, mS, rho * dmS);\n";
      s << "      const double dkk = fma(kk, dx, kM * dM);\n";
      s.fma(2); s.mul(2);
    }
    s << "      const double dPf = " << dprod(side_factors(r.reactants), "sA", "sdA") << ";\n";
    count_dprod(s, (int)side_factors(r.reactants).size());
    if (r.reversible) {
      s << "      const double dPr = " << dprod(side_factors(r.products), "sA", "sdA") << ";\n";
      count_dprod(s, (int)side_factors(r.products).size());
      s.add();
    } else {
      s << "      const double dPr = 0.0;\n";
    }
    s << "      const double dR = fma(dkk, D, kk * (dPf - dPr));\n     ";
    s.fma(); s.mul();
    emit_omega_update(s, r, "dR");
    s << "    }\n";
  }
  if (!opt.acc_mem)
    for (int k = 0; k < N; ++k) s << "    g_dw[(i64)" << k << " * n + p] = w" << k << ";\n";
  g_acc.mem = false;
  s << "  }\n}\n";
}

void emit_vjp_kernel(Src& s, const Mechanism& m, const std::vector<SpeciesCoef>& C, int blk, const EmitOptions& opt) {
  int N = m.n_species();
  s << "\n// VJP: (rho_bar, T_bar, Y_bar) = (d omega/d(rho, T, Y))^T omega_bar\n";
  s << "extern \"C\" __global__ void __launch_bounds__(" << blk << ") pyro_vjp(i64 n, const double* __restrict__ g_rho,\n"
       "    const double* __restrict__ g_T, const double* __restrict__ g_Y, const double* __restrict__ g_wb,\n"
       "    double* __restrict__ g_rhob, double* __restrict__ g_Tb, double* __restrict__ g_Yb,\n"
       "    double* __restrict__ g_store) {\n"
       "  __shared__ double s_exp[512];\n  __shared__ double s_log[256];\n  extern __shared__ double s_dyn[];\n"
       "  double* sL = " << (opt.dgstore ? "g_store + (i64)blockIdx.x * 4 * NSP * BLKD" : "s_dyn") << ";\n"
       "  double* sA = sL + NSP * BLKD; double* sLp = sA + NSP * BLKD; double* sC = sLp + NSP * BLKD;\n"
       "  pyro_load_tables(s_exp, s_log);\n  __syncthreads();\n  const int t = threadIdx.x;\n"
       "  for (i64 p = (i64)blockIdx.x * BLKD + t; p < n; p += (i64)gridDim.x * BLKD) {\n"
       "    const double* Yp = g_Y + p; const double* Wb = g_wb + p;\n"
       "    const double rho = g_rho[p], T = g_T[p];\n"
       "    const double lnT = pdm::log(T, s_log), invT = pdm::rcp(T), invT2 = invT * invT;\n"
       "    const bool hi = pdm::to_float_trunc(T) >= (float)TMID;\n";
  s.log_(); s.rcp_(); s.mul();
  emit_species_deriv(s, m, C, DMode::VJP);
  if (has_plog(m)) {
    s << "    const double lnp = lnT + pdm::log(rho * ysum, s_log) + " << lit((double)logl(R_GAS)) << ";\n";
    s.log_(); s.mul(); s.add(2);
  }
  s << "    double Tb = 0.0, Mtot = 0.0, rhobM = 0.0;\n";
  g_acc.mem = opt.acc_mem;
  g_acc.base = "Ab";
  if (opt.acc_mem) s << "    double* Ab = g_Yb + p;\n";
  emit_acc_init(s, "ab", N);
  for (int j = 0; j < m.n_reactions(); ++j) {
    const Reaction& r = m.reactions[j];
    s << "    { // reaction " << j << "\n";
    // R_bar = sum_k nu_kj omega_bar_k
    s << "      double Rb = 0.0;";
    for (auto& q : net_nu(r)) {
      if (q.second == 0) continue;
      s << " Rb = fma(" << lit((double)q.second) << ", __ldg(Wb + (i64)" << q.first << " * opq(n)), Rb);";
      s.fma();
    }
    s << "\n";
    emit_reaction_core(s, m, r);
    s << "      const double xb = Rb * R;\n      Tb = fma(xb, tau, Tb);";
    s.mul(); s.fma();
    for (auto& p : r.reactants) {
      s << " Tb = fma(" << lit(-(double)p.second) << " * xb, sLp" << sidx(p.first) << ", Tb);";
      s.fma(); if (p.second != 1) s.mul();
    }
    s << "\n      const double Db = Rb * kk;\n";
    s.mul();
    auto fr = side_factors(r.reactants);
    for (int q = 0; q < (int)fr.size(); ++q) {
      s << "      " << acc("ab", fr[q]) << " = fma(Db, " << prod_of(fr, "sA", q) << ", " << acc("ab", fr[q]) << ");\n";
      s.fma(); s.mul(std::max(0, (int)fr.size() - 2));
    }
    if (r.reversible) {
      auto fp = side_factors(r.products);
      for (int q = 0; q < (int)fp.size(); ++q) {
        s << "      " << acc("ab", fp[q]) << " = fma(-Db, " << prod_of(fp, "sA", q) << ", " << acc("ab", fp[q]) << ");\n";
        s.fma(); s.mul(std::max(0, (int)fp.size() - 2));
      }
    }
    if (r.kind != RX_ARRHENIUS) {
      s << "      const double Mb = Rb * kM * D; Mtot += Mb; rhobM = fma(Mb, mS, rhobM);\n";
      s.mul(2); s.add(); s.fma();
      for (auto& e : r.efficiencies) {
        double c = (e.second - 1.0) / m.species[e.first].W;
        if (c != 0.0) { s << "      sC" << sidx(e.first) << " = fma(Mb, " << lit(c) << ", sC" << sidx(e.first) << ");\n"; s.fma(); }
      }
    }
    s << "    }\n";
  }
  s << "    double rhob = 0.0;\n";
  for (int k = 0; k < N; ++k) {
    s << "    { const double abk = " << acc("ab", k) << "; const double ta = abk * sA" << sidx(k)
      << "; Tb = fma(ta, sLp" << sidx(k) << ", Tb); rhob += ta;\n";
    s << "      g_Yb[(i64)" << k << " * n + p] = fma(abk, PEXP(sL" << sidx(k) << ", s_exp) * rho, rho * fma(Mtot, "
      << lit(1.0 / m.species[k].W) << ", sC" << sidx(k) << ")); }\n";
    s.mul(3); s.fma(3); s.add(); s.exp_();
  }
  g_acc.mem = false;
  s << "    g_Tb[p] = Tb;\n    g_rhob[p] = fma(rhob, pdm::rcp(rho), rhobM);\n  }\n}\n";
  s.rcp_(); s.fma();
}

struct JacSlots {
  int n = 0;
  std::vector<int> R, Rt, RM;                 // per reaction
  std::vector<std::map<int, int>> Q;          // per reaction: species -> slot
};

// Which outputs the Jacobian kernel assembles from the per-reaction partials:
//  TY    d(Tdot, omega)/d(T, Y) at fixed rho, [(N+1)^2][n]
//  ADIA  dS_j/dY_k at fixed (rho, e), S = W omega (Eq. chem_jacobian), [N^2][n]
//  CN    the Crank-Nicolson Newton system (Eqs. crank_nicol_newton_update,
//        crank_nicol_jac) at the current iterate: matrix I - (dt/2rho) dS/dY|_(rho,e)
//        in groups of CN_G states ([n/CN_G][N^2][CN_G], the layout the batched solve
//        reads) and right-hand side -F = c + (dt/2rho) S - Y, c = Y^m + (dt/2rho) S^m.
enum class JacMode { TY, ADIA, CN };

// Tables of the row assembly of the Jacobian-type kernels (table mode): per row k
// the reactions with nu_kj != 0 (slots of R_j, Rt_j, RM_j, index j; nu_kj), per
// reaction the species partial slots (i, slot) and the third-body efficiency
// terms (i, eps_i - 1), per species W, 1/W and the NASA h/RT and cp/R
// coefficients of both ranges.
void emit_jac_tables(Src& s, const Mechanism& m, const std::vector<SpeciesCoef>& C, const JacSlots& sl,
                     const std::string& sfx) {
  const int N = m.n_species(), M = m.n_reactions();
  std::vector<std::vector<std::pair<int, int>>> rows(N);
  for (int j = 0; j < M; ++j)
    for (auto& q : net_nu(m.reactions[j])) if (q.second) rows[q.first].push_back({j, q.second});
  std::vector<int> rptr{0}, rent, qptr{0}, qent, eptr{0}, ei;
  std::vector<double> rnu, ec, sp;
  for (int k = 0; k < N; ++k) {
    for (auto& jn : rows[k]) {
      const int j = jn.first;
      rent.insert(rent.end(), {sl.R[j], sl.Rt[j], sl.RM[j], j});
      rnu.push_back((double)jn.second);
    }
    rptr.push_back((int)rnu.size());
  }
  for (int j = 0; j < M; ++j) {
    for (auto& qi : sl.Q[j]) qent.insert(qent.end(), {qi.first, qi.second});
    qptr.push_back((int)qent.size() / 2);
    if (sl.RM[j] >= 0)
      for (auto& e : m.reactions[j].efficiencies) {
        if (e.second == 1.0) continue;
        ei.push_back(e.first);
        ec.push_back(e.second - 1.0);
      }
    eptr.push_back((int)ei.size());
  }
  for (int k = 0; k < N; ++k) {
    sp.push_back(m.species[k].W);
    sp.push_back(1.0 / m.species[k].W);
    for (int rg = 0; rg < 2; ++rg) {
      for (int q = 0; q < 6; ++q) sp.push_back(C[k].h[rg][q]);
      for (int q = 0; q < 5; ++q) sp.push_back(C[k].cp[rg][q]);
    }
  }
  auto ints = [&](const char* nm, const std::vector<int>& v) {
    s << "__device__ const int " << nm << sfx << "[" << std::max<size_t>(v.size(), 1) << "] = {";
    for (size_t i = 0; i < v.size(); ++i) s << (i ? "," : "") << v[i];
    if (v.empty()) s << "0";
    s << "};\n";
  };
  auto dbls = [&](const char* nm, const std::vector<double>& v) {
    s << "__device__ const double " << nm << sfx << "[" << std::max<size_t>(v.size(), 1) << "] = {";
    for (size_t i = 0; i < v.size(); ++i) s << (i ? "," : "") << lit(v[i]);
    if (v.empty()) s << "0.0";
    s << "};\n";
  };
  s << "\n";
  ints("pyro_jr_ptr", rptr); ints("pyro_jr_ent", rent); dbls("pyro_jr_nu", rnu);
  ints("pyro_jq_ptr", qptr); ints("pyro_jq_ent", qent);
  ints("pyro_je_ptr", eptr); ints("pyro_je_i", ei); dbls("pyro_je_c", ec);
  dbls("pyro_jsp", sp);
}

// Row k's sums over its reactions: w = sum nu R, jt = sum nu Rt, u = sum nu RM
// (table mode).  Needs the tables with suffix sfx, W, and the row bounds re0, re1.
std::string jac_table_row_sums(const std::string& sfx) {
  return "      double w = 0.0, jt = 0.0, u = 0.0;\n"
         "      for (int ie = re0; ie < re1; ++ie) {\n"
         "        const double nu = __ldg(pyro_jr_nu" + sfx + " + ie);\n"
         "        const int* en = pyro_jr_ent" + sfx + " + 4 * ie;\n"
         "        w = fma(nu, W[(i64)__ldg(en) * BLKD], w); jt = fma(nu, W[(i64)__ldg(en + 1) * BLKD], jt);\n"
         "        const int rm = __ldg(en + 2);\n"
         "        if (rm >= 0) u = fma(nu, W[(i64)rm * BLKD], u);\n"
         "      }\n";
}

// Row k's species terms (table mode): for every reaction j of the row and every
// species i with a partial of R_j, ADD(i, v) with v = nu_kj dR_j/dY_i at fixed T
// (the activity partial, and the third-body term (eps_i - 1) RM_j rho/W_i).
std::string jac_table_row_terms(const std::string& sfx, const std::string& add) {
  return "      for (int ie = re0; ie < re1; ++ie) {\n"
         "        const double nu = __ldg(pyro_jr_nu" + sfx + " + ie);\n"
         "        const int* en = pyro_jr_ent" + sfx + " + 4 * ie;\n"
         "        const int jr = __ldg(en + 3), rm = __ldg(en + 2);\n"
         "        const int iq1 = __ldg(pyro_jq_ptr" + sfx + " + jr + 1);\n"
         "        for (int iq = __ldg(pyro_jq_ptr" + sfx + " + jr); iq < iq1; ++iq) {\n"
         "          const int i = __ldg(pyro_jq_ent" + sfx + " + 2 * iq);\n"
         "          const double v = nu * W[(i64)__ldg(pyro_jq_ent" + sfx + " + 2 * iq + 1) * BLKD];\n"
         "          " + add + "\n"
         "        }\n"
         "        if (rm >= 0) {\n"
         "          const double ru = nu * W[(i64)rm * BLKD];\n"
         "          const int if1 = __ldg(pyro_je_ptr" + sfx + " + jr + 1);\n"
         "          for (int ifc = __ldg(pyro_je_ptr" + sfx + " + jr); ifc < if1; ++ifc) {\n"
         "            const int i = __ldg(pyro_je_i" + sfx + " + ifc);\n"
         "            const double v = (__ldg(pyro_je_c" + sfx + " + ifc) * ru) * sE[i * BLKD + t];\n"
         "            " + add + "\n"
         "          }\n"
         "        }\n"
         "      }\n";
}

// FP64 operations of the table-driven row assembly (per state): per row the sums
// over its reactions, the species energy (ty: (T, Y) Jacobian with the Tdot
// column accumulators) or the row factor, the dense rank-1 fill and the species
// terms of every reaction of the row.
void count_table_rows(Src& s, const Mechanism& m, const JacSlots& sl, bool ty) {
  const int N = m.n_species();
  for (int k = 0; k < N; ++k) {
    for (int j = 0; j < m.n_reactions(); ++j) {
      int nu = 0;
      for (auto& q : net_nu(m.reactions[j])) if (q.first == k) nu = q.second;
      if (!nu) continue;
      s.fma(2 + (sl.RM[j] >= 0 ? 1 : 0));                          // w, jt, u sums
      const int nq = (int)sl.Q[j].size();
      if (ty) { s.mul(nq); s.add(nq); s.fma(nq); } else { s.mul(nq); s.fma(nq); }
      if (sl.RM[j] >= 0) {
        s.mul();                                                     // ru
        for (auto& e : m.reactions[j].efficiencies)
          if (e.second != 1.0) { s.mul(2); if (ty) { s.add(); s.fma(); } else s.fma(); }
      }
    }
    if (ty) { s.fma(5 + 4 + 1 + 4); s.add(); s.mul(1 + N); }          // h/RT, cp/R, e_k, 4 sums, cpm, dense fill
    else { s.mul(2); s.fma(N); s.mul(N); }                           // fu, fj, dense fill
  }
}

void emit_jacobian_kernel(Src& s, const Mechanism& m, const std::vector<SpeciesCoef>& C, int blk, int* nslots,
                          JacMode mode = JacMode::TY, bool gstore = false, bool table = false) {
  int N = m.n_species(), M = m.n_reactions(), NP = N + 1;
  JacSlots sl;
  sl.R.resize(M); sl.Rt.resize(M); sl.RM.assign(M, -1); sl.Q.resize(M);
  for (int j = 0; j < M; ++j) {
    const Reaction& r = m.reactions[j];
    sl.R[j] = sl.n++;
    sl.Rt[j] = sl.n++;
    if (r.kind != RX_ARRHENIUS) sl.RM[j] = sl.n++;
    std::set<int> sp;
    for (auto& p : r.reactants) sp.insert(p.first);
    if (r.reversible) for (auto& p : r.products) sp.insert(p.first);
    for (int i : sp) sl.Q[j][i] = sl.n++;
  }
  // per-block scratch: the slots, then (gstore) the two per-state species arrays
  const int stride = sl.n + (gstore ? 2 * N : 0);
  *nslots = stride;
  auto slot = [&](int q) { return "W[" + std::to_string(q) + " * BLKD]"; };
  // Per reaction, folded at emit time (species share T_mid): the reactant sum
  // sum_i nu'_i L_i (coefficients of lnT, 1/T, 1, T, .., T^4) and, for
  // dS = sum_i c_i L'_i = (sum_i c_i - sum_i c_i h_i/RT)/T with c_i = nu'_i - nu''_i,
  // the polynomial sum_i c_i h_i/RT (1, T, .., T^4, 1/T) -- per NASA range.  Only
  // two per-state arrays (activities a_i and E_i rho) stay in shared memory.
  s << "\n__device__ const double pyro_jfold_" << (int)mode << "[" << 26 * std::max(M, 1) << "] = {";
  int qf = 0;
  std::vector<long double> fold_c(M);
  for (int j = 0; j < M; ++j) {
    const Reaction& r = m.reactions[j];
    std::set<int> sp;
    for (auto& p : r.reactants) sp.insert(p.first);
    if (r.reversible) for (auto& p : r.products) sp.insert(p.first);
    long double csum = 0;
    for (int rg = 0; rg < 2; ++rg) {
      long double nl[7] = {0, 0, 0, 0, 0, 0, 0}, hh[6] = {0, 0, 0, 0, 0, 0};
      for (auto& p : r.reactants) {
        const SpeciesCoef& c = C[p.first];
        long double v = p.second;
        nl[0] += v * c.cl[rg]; nl[1] += v * c.ci[rg]; nl[2] += v * c.c0[rg]; nl[3] += v * c.c1[rg];
        nl[4] += v * c.c2[rg]; nl[5] += v * c.c3[rg]; nl[6] += v * c.c4[rg];
      }
      for (int i : sp) {
        long double ci = nu_of(r.reactants, i) - (r.reversible ? nu_of(r.products, i) : 0);
        if (rg == 0) csum += ci;
        for (int q = 0; q < 6; ++q) hh[q] += ci * C[i].h[rg][q];
      }
      for (int q = 0; q < 7; ++q) s << (qf++ ? "," : "") << lit((double)nl[q]);
      for (int q = 0; q < 6; ++q) s << "," << lit((double)hh[q]), ++qf;
    }
    fold_c[j] = csum;
  }
  if (qf == 0) s << "0.0";
  s << "};\n";
  const std::string ftab = "pyro_jfold_" + std::to_string((int)mode);
  // the exp/log tables in global memory (read through L1 instead of staged in shared memory)
  s << "__device__ const double pyro_tab_exp_g[512] = {";
  for (int j = 0; j < 512; ++j) s << (j ? "," : "") << lit((double)exp2l((j + 0.5L) / 512.0L));
  s << "};\n__device__ const double pyro_tab_log_g[256] = {";
  for (int j = 0; j < 128; ++j) {
    long double c = 1.0L + (j + 0.5L) / 128.0L;
    s << (j ? "," : "") << lit((double)(1.0L / c)) << "," << lit((double)logl(c));
  }
  s << "};\n";
  // exp/log tables read through L1: the 6 KB they would take in shared memory is
  // what lets a fourth 64-thread block fit on an SM
  const std::string sfx = "_" + std::to_string((int)mode);
  if (table) emit_jac_tables(s, m, C, sl, sfx);
  const std::string prologue =
      "  const double* __restrict__ s_exp = pyro_tab_exp_g;\n  const double* __restrict__ s_log = pyro_tab_log_g;\n" +
      (gstore ? "  double* sA = g_scratch + (i64)blockIdx.x * " + std::to_string(stride) + " * BLKD + " +
                    std::to_string(sl.n) + " * BLKD;\n  double* sE = sA + NSP * BLKD;\n"
              : std::string("  extern __shared__ double s_dyn[];\n  double* sA = s_dyn; double* sE = sA + NSP * BLKD;\n")) +
      "  const int t = threadIdx.x;\n";
  if (mode == JacMode::TY) {
    s << "\n// Dense Jacobian d(Tdot, omega)/d(T, Y) at fixed rho, [(N+1)^2][n]; row 0 = Tdot of the adiabatic\n"
         "// isochoric reactor, rows 1..N = omega; column 0 = T, columns 1..N = Y.  Phase 1 writes the\n"
         "// per-reaction partials to the block's scratch, phase 2 assembles the rows.\n";
    s << "extern \"C\" __global__ void __launch_bounds__(" << blk << ") pyro_jacobian(i64 n, const double* __restrict__ g_rho,\n"
         "    const double* __restrict__ g_T, const double* __restrict__ g_Y, double* __restrict__ g_J,\n"
         "    double* __restrict__ g_scratch) {\n" << prologue <<
         "  double* W = g_scratch + (i64)blockIdx.x * " << stride << " * BLKD + t;\n"
         "  for (i64 p = (i64)blockIdx.x * BLKD + t; p < n; p += (i64)gridDim.x * BLKD) {\n"
         "    const double* Yp = g_Y + p;\n    double* Jp = g_J + p;\n"
         "    const double rho = g_rho[p], T = g_T[p];\n";
  } else if (mode == JacMode::ADIA) {
    s << "\n// Chemical Jacobian dS_j/dY_k of S = W omega at fixed (rho, e) (Eq. chem_jacobian), [N^2][n],\n"
         "// row j, column k: W_j (d omega_j/dY_k + d omega_j/dT dT/dY_k), dT/dY_k = -e_k/c_v.\n";
    s << "extern \"C\" __global__ void __launch_bounds__(" << blk << ") pyro_jacobian_adiabatic(i64 n,\n"
         "    const double* __restrict__ g_rho, const double* __restrict__ g_T, const double* __restrict__ g_Y,\n"
         "    double* __restrict__ g_J, double* __restrict__ g_scratch) {\n" << prologue <<
         "  double* W = g_scratch + (i64)blockIdx.x * " << stride << " * BLKD + t;\n"
         "  for (i64 p = (i64)blockIdx.x * BLKD + t; p < n; p += (i64)gridDim.x * BLKD) {\n"
         "    const double* Yp = g_Y + p;\n    double* Jp = g_J + p;\n"
         "    const double rho = g_rho[p], T = g_T[p];\n";
  } else {
    s << "\n// Crank-Nicolson Newton system at the current iterate Y (state arrays [N][n], n = stride;\n"
         "// cnt states) for the *g_count active states listed in g_list; the system of the i-th\n"
         "// listed state goes to slot i.  state: 0 first iteration (forms c from S^m = S(Y^m)),\n"
         "// 1 iterating, 2 converged (one more step pending), 3 done, 4 failed.  Clears the\n"
         "// counter of the list the following solve builds.\n";
    s << "extern \"C\" __global__ void __launch_bounds__(" << blk << ") pyro_cn_assemble(i64 cnt, i64 n,\n"
         "    const double* __restrict__ g_rho, const double* __restrict__ g_e, const double* __restrict__ g_Y,\n"
         "    double* __restrict__ g_c, double* __restrict__ g_T, int* __restrict__ g_state, double dt,\n"
         "    int max_iter, double tol, double* __restrict__ g_A, double* __restrict__ g_b,\n"
         "    double* __restrict__ g_scratch, unsigned long long* __restrict__ g_fail,\n"
         "    const int* __restrict__ g_list, const int* __restrict__ g_count, int* __restrict__ g_count_next,\n"
         "    int a_at_state) {\n" << prologue <<
         "  double* W = g_scratch + (i64)blockIdx.x * " << stride << " * BLKD + t;\n"
         "  const float tolf = (float)tol;\n"
         "  const i64 na = *g_count;\n"
         "  if (blockIdx.x == 0 && t == 0) *g_count_next = 0;\n"
         "  for (i64 q = (i64)blockIdx.x * BLKD + t; q < na; q += (i64)gridDim.x * BLKD) {\n"
         "    const i64 p = g_list[q];\n"
         "    const int stp = g_state[p];\n"
         "    const double* Yp = g_Y + p;\n"
         "    const i64 qa = a_at_state ? p : q;   // matrix at the state's own index (chord) or its slot\n"
         "    double* Jp = g_A + (qa / CN_G) * (i64)(NSP * NSP * CN_G) + (qa % CN_G);\n"
         "    const double rho = g_rho[p];\n"
         "    int tit;\n"
         "    const double T = pyro_tsolve<false>(Yp, n, g_e[p], g_T[p], max_iter, tolf, &tit);\n"
         "    if (tit < 0) { g_state[p] = 4; atomicAdd(g_fail, 1ull); continue; }\n"
         "    g_T[p] = T;\n";
  }
  s << "    const double lnT = pdm::log(T, s_log), invT = pdm::rcp(T), invT2 = invT * invT;\n"
       "    const bool hi = pdm::to_float_trunc(T) >= (float)TMID;\n";
  s.log_(); s.rcp_(); s.mul();
  emit_species_deriv(s, m, C, DMode::JAC);
  if (has_plog(m)) {
    s << "    const double lnp = lnT + pdm::log(rho * ysum, s_log) + " << lit((double)logl(R_GAS)) << ";\n";
    s.log_(); s.mul(); s.add(2);
  }
  // ---- phase 1
  s << "    const int fr = hi ? 13 : 0;\n";
  for (int j = 0; j < M; ++j) {
    const Reaction& r = m.reactions[j];
    s << "    { // reaction " << j << "\n";
    s << "      const double* fj = " << ftab << " + " << 26 * j << " + fr;\n"
         "      const double nuL = fma(__ldg(fj), lnT, fma(__ldg(fj + 1), invT, fma(T, fma(T, fma(T, fma(T, __ldg(fj + 6), "
         "__ldg(fj + 5)), __ldg(fj + 4)), __ldg(fj + 3)), __ldg(fj + 2))));\n";
    s.fma(6);
    g_fold = true;
    emit_reaction_core(s, m, r);
    g_fold = false;
    std::set<int> sp;
    for (auto& p : r.reactants) sp.insert(p.first);
    if (r.reversible) for (auto& p : r.products) sp.insert(p.first);
    // S' - S'' = sum_i (nu'_i - nu''_i) L'_i, L'_i = (1 - h_i/RT)/T, from the folded polynomial
    s << "      const double Hj = fma(__ldg(fj + 12), invT, fma(T, fma(T, fma(T, fma(T, __ldg(fj + 11), __ldg(fj + 10)), "
         "__ldg(fj + 9)), __ldg(fj + 8)), __ldg(fj + 7)));\n"
         "      const double dS = (" << lit((double)fold_c[j]) << " - Hj) * invT;\n";
    s << "      " << slot(sl.R[j]) << " = R; " << slot(sl.Rt[j]) << " = kk * fma(D, tau, Pr * dS);\n";
    s.fma(5); s.add(); s.mul(); s.mul(2); s.fma();
    if (sl.RM[j] >= 0) { s << "      " << slot(sl.RM[j]) << " = kM * D;\n"; s.mul(); }
    auto fr = side_factors(r.reactants);
    auto fp = side_factors(r.products);
    for (int i : sp) {
      std::string e;
      for (int q = 0; q < (int)fr.size(); ++q)
        if (fr[q] == i) { e = " + " + prod_of(fr, "sA", q); break; }
      int nr_ = nu_of(r.reactants, i);
      std::string termf = e.empty() ? "" : "(" + lit((double)nr_) + " * " + e.substr(3) + ")";
      std::string termr;
      if (r.reversible)
        for (int q = 0; q < (int)fp.size(); ++q)
          if (fp[q] == i) { termr = "(" + lit((double)nu_of(r.products, i)) + " * " + prod_of(fp, "sA", q) + ")"; break; }
      std::string diff = termf.empty() ? "-" + termr : termr.empty() ? termf : termf + " - " + termr;
      s << "      " << slot(sl.Q[j][i]) << " = kk * sE" << sidx(i) << " * (" << diff << ");\n";
      // kk * sE * (.), the products of the other factors, nu * product (nu != 1), the difference
      s.mul(2);
      if (!termf.empty()) { s.mul(std::max(0, (int)fr.size() - 2)); if (nr_ != 1) s.mul(); }
      if (!termr.empty()) { s.mul(std::max(0, (int)fp.size() - 2)); if (nu_of(r.products, i) != 1) s.mul(); }
      if (!termf.empty() && !termr.empty()) s.add();
    }
    s << "    }\n";
  }
  if (mode != JacMode::TY) {
    // ---- phase 2 at fixed (rho, e): sL becomes s_i = rho/W_i, sA becomes
    // dT/dY_i|_e = -e_i/c_v (Eq. int_energy: e = sum_i Y_i e_i(T), c_v = de/dT).
    s << "    asm volatile(\"\" ::: \"memory\");\n";
    s << "    const double RT = " << lit((double)R_GAS) << " * T;\n    double cv = 0.0;\n";
    for (int i = 0; i < N; ++i) {
      const SpeciesCoef& c = C[i];
      double h4[2] = {c.h[0][4], c.h[1][4]}, h3[2] = {c.h[0][3], c.h[1][3]}, h2[2] = {c.h[0][2], c.h[1][2]};
      double h1[2] = {c.h[0][1], c.h[1][1]}, h0[2] = {c.h[0][0], c.h[1][0]}, h5[2] = {c.h[0][5], c.h[1][5]};
      double p4[2] = {c.cp[0][4], c.cp[1][4]}, p3[2] = {c.cp[0][3], c.cp[1][3]}, p2[2] = {c.cp[0][2], c.cp[1][2]};
      double p1[2] = {c.cp[0][1], c.cp[1][1]}, p0[2] = {c.cp[0][0], c.cp[1][0]};
      s << "    { const double y = __ldg(Yp + (i64)" << i << " * n);\n";
      s << "      double hr = fma(T, " << sel(h4) << ", " << sel(h3) << "); hr = fma(T, hr, " << sel(h2)
        << "); hr = fma(T, hr, " << sel(h1) << "); hr = fma(T, hr, " << sel(h0) << "); hr = fma(" << sel(h5)
        << ", invT, hr);\n";
      s << "      double cp = fma(T, " << sel(p4) << ", " << sel(p3) << "); cp = fma(T, cp, " << sel(p2)
        << "); cp = fma(T, cp, " << sel(p1) << "); cp = fma(T, cp, " << sel(p0) << ");\n";
      s << "      sA" << sidx(i) << " = fma(RT, hr, -RT) * " << lit(1.0 / m.species[i].W) << ";\n";
      s << "      cv = fma(y * " << lit((double)R_GAS / m.species[i].W) << ", cp - 1.0, cv);\n";
      s << "      sE" << sidx(i) << " = rho * " << lit(1.0 / m.species[i].W) << "; }\n";
      s.fma(5 + 4 + 1 + 1); s.mul(3); s.add();   // h/RT, cp/R, e_i, c_v term, rho/W_i
    }
    s << "    const double mrcv = -pdm::rcp(cv);\n";
    s << "    #pragma unroll 1\n    for (int i = 0; i < NSP; ++i) sA[i * BLKD + t] *= mrcv;\n";
    s.mul(1 + N); s.rcp_();
    if (mode == JacMode::CN) {
      s << "    const double hh = 0.5 * dt * pdm::rcp(rho);\n";
      s << "    const i64 nr = CN_G;\n";
    }
    if (table) {
      count_table_rows(s, m, sl, false);
      // rows by loops over the tables; the entries of row k accumulate in place
      s << "    #pragma unroll 1\n    for (int k = 0; k < NSP; ++k) {\n"
           "      const int re0 = __ldg(pyro_jr_ptr" << sfx << " + k), re1 = __ldg(pyro_jr_ptr" << sfx << " + k + 1);\n"
        << jac_table_row_sums(sfx) <<
           "      const double Wk = __ldg(pyro_jsp" << sfx << " + 24 * k);\n";
      if (mode == JacMode::CN) s << "      const double F = -hh * Wk;\n";
      else s << "      const double F = Wk;\n      const i64 nr = n;\n";
      s << "      const double fu = F * u, fj = F * jt;\n"
           "      double* Jr = Jp + (i64)k * NSP * nr;\n"
           "      #pragma unroll 1\n"
           "      for (int i = 0; i < NSP; ++i) Jr[(i64)i * nr] = fma(sE[i * BLKD + t], fu, fj * sA[i * BLKD + t]);\n";
      if (mode == JacMode::CN) s << "      Jr[(i64)k * nr] += 1.0;\n";
      s << jac_table_row_terms(sfx, "Jr[(i64)i * nr] = fma(F, v, Jr[(i64)i * nr]);");
      if (mode == JacMode::CN)
        s << "      { const double y = __ldg(Yp + (i64)k * n);\n"
             "        const double sk = (hh * Wk) * w;\n"
             "        double ck;\n"
             "        if (stp == 0) { ck = y + sk; g_c[(i64)k * cnt + p] = ck; } else { ck = g_c[(i64)k * cnt + p]; }\n"
             "        g_b[(i64)k * cnt + q] = (ck + sk) - y; }\n";
      else
        s << "      (void)w;\n";
      s << "    }\n  }\n}\n";
      return;
    }
    std::vector<std::vector<std::pair<int, int>>> rows(N);
    for (int j = 0; j < M; ++j)
      for (auto& q : net_nu(m.reactions[j])) if (q.second) rows[q.first].push_back({j, q.second});
    for (int k = 0; k < N; ++k) {
      s << "    { // row of species " << k << "\n      double w = 0.0, jt = 0.0, u = 0.0;\n";
      std::map<int, std::string> acc, cr;
      for (auto& jn : rows[k]) {
        int j = jn.first;
        std::string nu = lit((double)jn.second);
        s << "      w = fma(" << nu << ", " << slot(sl.R[j]) << ", w); jt = fma(" << nu << ", " << slot(sl.Rt[j]) << ", jt);";
        if (sl.RM[j] >= 0) s << " u = fma(" << nu << ", " << slot(sl.RM[j]) << ", u);";
        s << "\n";
        for (auto& qi : sl.Q[j]) {
          std::string name = "q" + std::to_string(qi.first);
          if (!acc.count(qi.first)) { acc[qi.first] = name; s << "      double " << name << " = 0.0;\n"; }
          s << "      " << name << " = fma(" << nu << ", " << slot(qi.second) << ", " << name << ");\n";
        }
        if (sl.RM[j] >= 0) {
          for (auto& e : m.reactions[j].efficiencies) {
            if (e.second == 1.0) continue;
            std::string name = "c" + std::to_string(e.first);
            if (!cr.count(e.first)) { cr[e.first] = name; s << "      double " << name << " = 0.0;\n"; }
            s << "      " << name << " = fma(" << nu << " * " << lit(e.second - 1.0) << ", " << slot(sl.RM[j]) << ", " << name << ");\n";
          }
        }
      }
      for (auto& jn : rows[k]) {
        const int j = jn.first;
        s.fma(2 + (sl.RM[j] >= 0 ? 1 : 0) + (int)sl.Q[j].size());
        if (sl.RM[j] >= 0)
          for (auto& e : m.reactions[j].efficiencies) if (e.second != 1.0) s.fma();
      }
      s.mul(2); s.fma(N); s.mul(N);                  // fu, fj, dense fill
      // row factor: W_k (Jacobian of S = W omega), or -dt/(2 rho) W_k (Newton matrix)
      if (mode == JacMode::CN) s << "      const double F = -hh * " << lit(m.species[k].W) << ";\n";
      else s << "      const double F = " << lit(m.species[k].W) << ";\n";
      s << "      const double fu = F * u, fj = F * jt;\n";
      // a fresh opaque stride per row keeps the compiler from holding all N^2 offsets live
      if (mode != JacMode::CN) s << "      const i64 nr = opq(n);\n";
      s << "      double* Jr = Jp + (i64)" << k * N << " * nr;\n";
      s << "      #pragma unroll 1\n      for (int i = 0; i < NSP; ++i) Jr[(i64)i * nr] = fma(sE[i * BLKD + t], fu, fj * sA[i * BLKD + t]);\n";
      for (int i = 0; i < N; ++i) {
        std::string si = "sE" + sidx(i), ti = "sA" + sidx(i);
        std::string dst = "Jr[(i64)" + std::to_string(i) + " * nr]";
        bool hs = acc.count(i), hc = cr.count(i), diag = mode == JacMode::CN && i == k;
        if (hs || hc) {
          if (hc) s.fma();
          s.fma(2); s.mul();
          std::string tv = hc ? "fma(" + si + ", " + cr[i] + ", " + (hs ? acc[i] : std::string("0.0")) + ")" : acc[i];
          std::string base = diag ? "fma(F, " + tv + ", 1.0)" : "F * " + tv;
          s << "      " << dst << " = fma(" << si << ", fu, fma(fj, " << ti << ", " << base << "));\n";
        } else if (diag) {
          s << "      " << dst << " = fma(" << si << ", fu, fma(fj, " << ti << ", 1.0));\n";
        }
      }
      if (mode == JacMode::CN) {
        // right-hand side -F_k = c_k + (dt/2rho) W_k omega_k - Y_k (Eq. crank_nicol_rhs)
        s << "      { const double y = __ldg(Yp + (i64)" << k << " * n);\n"
             "        const double sk = (hh * " << lit(m.species[k].W) << ") * w;\n"
             "        double ck;\n"
             "        if (stp == 0) { ck = y + sk; g_c[(i64)" << k << " * cnt + p] = ck; } else { ck = g_c[(i64)" << k << " * cnt + p]; }\n"
             "        g_b[(i64)" << k << " * cnt + q] = (ck + sk) - y; }\n";
      }
      s << "    }\n";
    }
    s << "  }\n}\n";
    return;
  }
  // ---- phase 2: rows.  sL becomes s_i = rho/W_i, sA the Tdot column accumulators.
  // The barrier keeps the compiler from forwarding phase-1 values through registers.
  s << "    asm volatile(\"\" ::: \"memory\");\n";
  for (int i = 0; i < N; ++i)
    s << "    sE" << sidx(i) << " = rho * " << lit(1.0 / m.species[i].W) << "; sA" << sidx(i) << " = 0.0;\n";
  s << "    const double RT = " << lit((double)R_GAS) << " * T;\n";
  s.mul(N + 1);
  s << "    double sum_ew = 0.0, sum_cpw = 0.0, sum_ejt = 0.0, U = 0.0;\n";
  // per-species row lists
  std::vector<std::vector<std::pair<int, int>>> rows(N);
  for (int j = 0; j < M; ++j)
    for (auto& q : net_nu(m.reactions[j])) if (q.second) rows[q.first].push_back({j, q.second});
  if (table) {
    count_table_rows(s, m, sl, true);
    // rows by loops over the tables; the entries of row k accumulate in place and
    // each species term also feeds the Tdot column accumulator sA_i (weight e_k)
    s << "    #pragma unroll 1\n    for (int k = 0; k < NSP; ++k) {\n"
         "      const int re0 = __ldg(pyro_jr_ptr" << sfx << " + k), re1 = __ldg(pyro_jr_ptr" << sfx << " + k + 1);\n"
      << jac_table_row_sums(sfx) <<
         "      const double* cf = pyro_jsp" << sfx << " + 24 * k + (hi ? 13 : 2);\n"
         "      double hr = fma(T, __ldg(cf + 4), __ldg(cf + 3)); hr = fma(T, hr, __ldg(cf + 2)); "
         "hr = fma(T, hr, __ldg(cf + 1)); hr = fma(T, hr, __ldg(cf)); hr = fma(__ldg(cf + 5), invT, hr);\n"
         "      double cp = fma(T, __ldg(cf + 10), __ldg(cf + 9)); cp = fma(T, cp, __ldg(cf + 8)); "
         "cp = fma(T, cp, __ldg(cf + 7)); cp = fma(T, cp, __ldg(cf + 6));\n"
         "      const double eh = fma(RT, hr, -RT); const double cpm = " << lit((double)R_GAS) << " * (cp - 1.0);\n"
         "      sum_ew = fma(eh, w, sum_ew); sum_cpw = fma(cpm, w, sum_cpw); sum_ejt = fma(eh, jt, sum_ejt); U = fma(eh, u, U);\n"
         "      const i64 nr = n;\n      double* Jr = Jp + (i64)(k + 1) * " << NP << " * nr;\n      Jr[0] = jt;\n"
         "      #pragma unroll 1\n"
         "      for (int i = 0; i < NSP; ++i) Jr[(i64)(1 + i) * nr] = sE[i * BLKD + t] * u;\n"
      << jac_table_row_terms(sfx, "Jr[(i64)(1 + i) * nr] += v; sA[i * BLKD + t] = fma(eh, v, sA[i * BLKD + t]);") <<
         "    }\n";
  }
  for (int k = 0; k < (table ? 0 : N); ++k) {
    const SpeciesCoef& c = C[k];
    for (auto& jn : rows[k]) {
      const int j = jn.first;
      s.fma(2 + (sl.RM[j] >= 0 ? 1 : 0) + (int)sl.Q[j].size());
      if (sl.RM[j] >= 0)
        for (auto& e : m.reactions[j].efficiencies) if (e.second != 1.0) s.fma();
    }
    s.fma(5 + 4 + 1 + 4); s.add(); s.mul(1 + N);   // h/RT, cp/R, e_k, 4 sums, cpm, dense fill
    s << "    { // row of species " << k << "\n      double w = 0.0, jt = 0.0, u = 0.0;\n";
    std::map<int, std::string> acc, cr;
    for (auto& jn : rows[k]) {
      int j = jn.first;
      std::string nu = lit((double)jn.second);
      s << "      w = fma(" << nu << ", " << slot(sl.R[j]) << ", w); jt = fma(" << nu << ", " << slot(sl.Rt[j]) << ", jt);";
      if (sl.RM[j] >= 0) s << " u = fma(" << nu << ", " << slot(sl.RM[j]) << ", u);";
      s << "\n";
      for (auto& qi : sl.Q[j]) {
        std::string name = "q" + std::to_string(qi.first);
        if (!acc.count(qi.first)) { acc[qi.first] = name; s << "      double " << name << " = 0.0;\n"; }
        s << "      " << name << " = fma(" << nu << ", " << slot(qi.second) << ", " << name << ");\n";
      }
      if (sl.RM[j] >= 0) {
        for (auto& e : m.reactions[j].efficiencies) {
          if (e.second == 1.0) continue;
          std::string name = "c" + std::to_string(e.first);
          if (!cr.count(e.first)) { cr[e.first] = name; s << "      double " << name << " = 0.0;\n"; }
          s << "      " << name << " = fma(" << nu << " * " << lit(e.second - 1.0) << ", " << slot(sl.RM[j]) << ", " << name << ");\n";
        }
      }
    }
    double h4[2] = {c.h[0][4], c.h[1][4]}, h3[2] = {c.h[0][3], c.h[1][3]}, h2[2] = {c.h[0][2], c.h[1][2]};
    double h1[2] = {c.h[0][1], c.h[1][1]}, h0[2] = {c.h[0][0], c.h[1][0]}, h5[2] = {c.h[0][5], c.h[1][5]};
    double p4[2] = {c.cp[0][4], c.cp[1][4]}, p3[2] = {c.cp[0][3], c.cp[1][3]}, p2[2] = {c.cp[0][2], c.cp[1][2]};
    double p1[2] = {c.cp[0][1], c.cp[1][1]}, p0[2] = {c.cp[0][0], c.cp[1][0]};
    s << "      double hr = fma(T, " << sel(h4) << ", " << sel(h3) << "); hr = fma(T, hr, " << sel(h2)
      << "); hr = fma(T, hr, " << sel(h1) << "); hr = fma(T, hr, " << sel(h0) << "); hr = fma(" << sel(h5) << ", invT, hr);\n";
    s << "      double cp = fma(T, " << sel(p4) << ", " << sel(p3) << "); cp = fma(T, cp, " << sel(p2)
      << "); cp = fma(T, cp, " << sel(p1) << "); cp = fma(T, cp, " << sel(p0) << ");\n";
    s << "      const double eh = fma(RT, hr, -RT); const double cpm = " << lit((double)R_GAS) << " * (cp - 1.0);\n";
    s << "      sum_ew = fma(eh, w, sum_ew); sum_cpw = fma(cpm, w, sum_cpw); sum_ejt = fma(eh, jt, sum_ejt); U = fma(eh, u, U);\n";
    s << "      const i64 nr = opq(n);\n      double* Jr = Jp + (i64)" << (k + 1) * NP << " * nr;\n      Jr[0] = jt;\n";
    s << "      #pragma unroll 1\n      for (int i = 0; i < NSP; ++i) Jr[(i64)(1 + i) * nr] = sE[i * BLKD + t] * u;\n";
    for (int i = 0; i < N; ++i) {
      std::string si = "sE" + sidx(i);
      std::string dst = "Jr[(i64)" + std::to_string(1 + i) + " * nr]";
      bool hs = acc.count(i), hc = cr.count(i);
      if (hs || hc) {
        s.fma(2 + (hc ? 1 : 0));
        std::string tv = hc ? "fma(" + si + ", " + cr[i] + ", " + (hs ? acc[i] : std::string("0.0")) + ")" : acc[i];
        s << "      { const double tv = " << tv << "; " << dst << " = fma(" << si << ", u, tv); sA" << sidx(i)
          << " = fma(eh, tv, sA" << sidx(i) << "); }\n";
      }
    }
    s << "    }\n";
  }
  // Tdot row
  s << "    double cv = 0.0, cvT = 0.0;\n";
  for (int k = 0; k < N; ++k) {
    const SpeciesCoef& c = C[k];
    double p4[2] = {c.cp[0][4], c.cp[1][4]}, p3[2] = {c.cp[0][3], c.cp[1][3]}, p2[2] = {c.cp[0][2], c.cp[1][2]};
    double p1[2] = {c.cp[0][1], c.cp[1][1]}, p0[2] = {c.cp[0][0], c.cp[1][0]};
    double q3[2] = {c.cpd[0][3], c.cpd[1][3]}, q2[2] = {c.cpd[0][2], c.cpd[1][2]}, q1[2] = {c.cpd[0][1], c.cpd[1][1]};
    double q0[2] = {c.cpd[0][0], c.cpd[1][0]};
    s << "    { const double yw = __ldg(Yp + (i64)" << k << " * n) * " << lit((double)R_GAS / m.species[k].W) << ";\n";
    s << "      double cp = fma(T, " << sel(p4) << ", " << sel(p3) << "); cp = fma(T, cp, " << sel(p2)
      << "); cp = fma(T, cp, " << sel(p1) << "); cp = fma(T, cp, " << sel(p0) << ");\n";
    s << "      double cd = fma(T, " << sel(q3) << ", " << sel(q2) << "); cd = fma(T, cd, " << sel(q1) << "); cd = fma(T, cd, " << sel(q0) << ");\n";
    s << "      cv = fma(yw, cp - 1.0, cv); cvT = fma(yw, cd, cvT); }\n";
    s.mul(); s.fma(4 + 3 + 2); s.add();
  }
  s << "    const double rcv = pdm::rcp(rho * cv);\n    const double Tdot = -sum_ew * rcv;\n"
       "    const double tcv = Tdot * pdm::rcp(cv);\n"
       "    Jp[0] = fma(-(sum_cpw + sum_ejt), rcv, -tcv * cvT);\n";
  s.mul(4); s.rcp_(); s.rcp_(); s.add(); s.fma();
  // Tdot row: d c_v/dY_i = (cp_i/R - 1) R/W_i recomputed per entry
  for (int k = 0; k < N; ++k) {
    const SpeciesCoef& c = C[k];
    double p4[2] = {c.cp[0][4], c.cp[1][4]}, p3[2] = {c.cp[0][3], c.cp[1][3]}, p2[2] = {c.cp[0][2], c.cp[1][2]};
    double p1[2] = {c.cp[0][1], c.cp[1][1]}, p0[2] = {c.cp[0][0], c.cp[1][0]};
    s << "    { double cp = fma(T, " << sel(p4) << ", " << sel(p3) << "); cp = fma(T, cp, " << sel(p2)
      << "); cp = fma(T, cp, " << sel(p1) << "); cp = fma(T, cp, " << sel(p0) << ");\n"
      << "      Jp[(i64)" << 1 + k << " * opq(n)] = fma(-fma(sE" << sidx(k) << ", U, sA" << sidx(k) << "), rcv, -tcv * ((cp - 1.0) * "
      << lit((double)R_GAS / m.species[k].W) << ")); }\n";
    s.fma(4 + 2); s.add(); s.mul(2);
  }
  s << "  }\n}\n";
}

// ---------------------------------------------------------------------------
// Mixture-averaged transport (Sec. A.2): mu (Eq. mixavg_viscosity, Wilke's
// Phi), kappa (Eq. mixavg_conductivity, Eq. species_cond) and the mixture
// diffusivities D_km (Eq. diff_mix_rule), one thread per state.
//
// Arithmetic (exact up to rounding):
//  * mu_k = sqrt(T) P_k^2 with P_k = |sum_m b_km ln^m T|, so sqrt(mu_k/mu_j) =
//    P_k/P_j and Wilke's Phi_kj = c_kj (1 + P_k w_kj / P_j)^2 with the constants
//    c_kj = 1/sqrt(8 (1 + W_k/W_j)), w_kj = (W_j/W_k)^(1/4).  Expanding the square,
//      sum_j Phi_kj X_j = sum_j c_kj X_j + 2 P_k sum_j c_kj w_kj (X_j/P_j)
//                         + P_k^2 sum_j c_kj w_kj^2 (X_j/P_j^2),
//    three products with constant matrices and no per-pair square root or division.
//  * the common sqrt(T) of the species fits is factored out of every sum.
//  * D_km = (1 - Y_k) sqrt(T) / sum_{j != k} X_j / p_kj (W - X_k W_k = W (1 - Y_k)),
//    with one reciprocal per unordered pair {k, j} feeding both sums.
// ---------------------------------------------------------------------------
void emit_transport_kernel(Src& s, const Mechanism& m, int blk, bool gstore) {
  const int N = m.n_species();
  const TransportFits& tf = m.transport;
  auto W = [&](int k) { return (long double)m.species[k].W; };
  // constant tables (global memory, read with uniform addresses)
  s << "\n__device__ const double pyro_tr_wilke[" << 3 * N * N << "] = {";
  for (int t = 0; t < 3; ++t)
    for (int k = 0; k < N; ++k)
      for (int j = 0; j < N; ++j) {
        long double c = 1.0L / sqrtl(8.0L * (1.0L + W(k) / W(j)));
        long double w = powl(W(j) / W(k), 0.25L);
        long double v = t == 0 ? c : t == 1 ? c * w : c * w * w;
        s << ((t | k | j) ? "," : "") << lit((double)v);
      }
  s << "};\n";
  const int npair = N * (N - 1) / 2;
  s << "__device__ const double pyro_tr_pair[" << std::max(1, 5 * npair) << "] = {";
  int q = 0;
  for (int k = 0; k < N; ++k)
    for (int j = k + 1; j < N; ++j)
      for (int i = 0; i < 5; ++i) s << (q++ ? "," : "") << lit(tf.diff[((size_t)k * N + j) * 5 + i]);
  if (q == 0) s << "0.0";
  s << "};\n";
  s << "__device__ const double pyro_tr_visc[" << 5 * N << "] = {";
  for (int k = 0; k < N; ++k)
    for (int i = 0; i < 5; ++i) s << ((k | i) ? "," : "") << lit(tf.visc[(size_t)k * 5 + i]);
  s << "};\n";
  s << "\n// mu, kappa, D_km of the mixture-averaged model (each output nullable)\n";
  s << "extern \"C\" __global__ void __launch_bounds__(" << blk << ") pyro_transport(i64 n, const double* __restrict__ g_T,\n"
       "    const double* __restrict__ g_Y, double* __restrict__ g_mu, double* __restrict__ g_kappa,\n"
       "    double* __restrict__ g_Dm, double* __restrict__ g_store) {\n"
       "  __shared__ double s_exp[512];\n  __shared__ double s_log[256];\n  extern __shared__ double s_dyn[];\n"
       "  double* sX = " << (gstore ? "g_store + (i64)blockIdx.x * 3 * NSP * BLKD" : "s_dyn") << ";\n"
       "  double* sV = sX + NSP * BLKD; double* sW = sV + NSP * BLKD;\n"
       "  pyro_load_tables(s_exp, s_log);\n  __syncthreads();\n  const int t = threadIdx.x;\n"
       "  for (i64 p = (i64)blockIdx.x * BLKD + t; p < n; p += (i64)gridDim.x * BLKD) {\n"
       "    const double* Yp = g_Y + p;\n"
       "    const double T = g_T[p];\n    const double L = pdm::log(T, s_log);\n    const double sqT = sqrt(T);\n"
       "    double ys = 0.0;\n";
  for (int k = 0; k < N; ++k) s << "    ys = fma(__ldg(Yp + (i64)" << k << " * n), " << lit(1.0 / m.species[k].W) << ", ys);\n";
  s << "    const double rys = pdm::rcp(ys);\n    double ka = 0.0, kh = 0.0;\n";
  for (int k = 0; k < N; ++k) {
    const double* b = &tf.visc[(size_t)k * 5];
    const double* c = &tf.cond[(size_t)k * 5];
    s << "    { const double x = __ldg(Yp + (i64)" << k << " * n) * (" << lit(1.0 / m.species[k].W) << " * rys);\n"
      << "      double P = fma(L, " << lit(b[4]) << ", " << lit(b[3]) << "); P = fma(L, P, " << lit(b[2])
      << "); P = fma(L, P, " << lit(b[1]) << "); P = fabs(fma(L, P, " << lit(b[0]) << "));\n"
      << "      double K = fma(L, " << lit(c[4]) << ", " << lit(c[3]) << "); K = fma(L, K, " << lit(c[2])
      << "); K = fma(L, K, " << lit(c[1]) << "); K = fma(L, K, " << lit(c[0]) << ");\n"
      << "      const double qv = pdm::rcp(P) * x;\n"
      << "      sX" << sidx(k) << " = x; sV" << sidx(k) << " = qv; sW" << sidx(k) << " = qv * pdm::rcp(P);\n"
      << "      ka = fma(x, K, ka); kh = fma(x, pdm::rcp(K), kh); }\n";
  }
  s << "    if (g_kappa) g_kappa[p] = 0.5 * sqT * (ka + pdm::rcp(kh));\n";
  s << R"(    if (g_mu) {
      double mu = 0.0;
      // two rows k, k+1 per pass: each X_j, X_j/P_j, X_j/P_j^2 load feeds six
      // independent FMA chains (the three Wilke products of both rows)
      int k = 0;
      #pragma unroll 1
      for (; k + 1 < NSP; k += 2) {
        const double* c0 = pyro_tr_wilke + k * NSP;
        const double* c1 = c0 + NSP * NSP;
        const double* c2 = c1 + NSP * NSP;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, b0 = 0.0, b1 = 0.0, b2 = 0.0;
        #pragma unroll 2
        for (int j = 0; j < NSP; ++j) {
          const double xj = sX[j * BLKD + t], vj = sV[j * BLKD + t], wj = sW[j * BLKD + t];
          a0 = fma(__ldg(c0 + j), xj, a0);
          a1 = fma(__ldg(c1 + j), vj, a1);
          a2 = fma(__ldg(c2 + j), wj, a2);
          b0 = fma(__ldg(c0 + NSP + j), xj, b0);
          b1 = fma(__ldg(c1 + NSP + j), vj, b1);
          b2 = fma(__ldg(c2 + NSP + j), wj, b2);
        }
        #pragma unroll
        for (int r = 0; r < 2; ++r) {
          const double* bk = pyro_tr_visc + 5 * (k + r);
          double Pk = fma(L, __ldg(bk + 4), __ldg(bk + 3));
          Pk = fma(L, Pk, __ldg(bk + 2)); Pk = fma(L, Pk, __ldg(bk + 1)); Pk = fabs(fma(L, Pk, __ldg(bk)));
          const double den = r == 0 ? fma(Pk, fma(Pk, a2, 2.0 * a1), a0) : fma(Pk, fma(Pk, b2, 2.0 * b1), b0);
          mu = fma(sX[(k + r) * BLKD + t] * (Pk * Pk), pdm::rcp(den), mu);
        }
      }
      if (k < NSP) {
        const double* c0 = pyro_tr_wilke + k * NSP;
        const double* c1 = c0 + NSP * NSP;
        const double* c2 = c1 + NSP * NSP;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int j = 0; j < NSP; ++j) {
          a0 = fma(__ldg(c0 + j), sX[j * BLKD + t], a0);
          a1 = fma(__ldg(c1 + j), sV[j * BLKD + t], a1);
          a2 = fma(__ldg(c2 + j), sW[j * BLKD + t], a2);
        }
        const double* bk = pyro_tr_visc + 5 * k;
        double Pk = fma(L, __ldg(bk + 4), __ldg(bk + 3));
        Pk = fma(L, Pk, __ldg(bk + 2)); Pk = fma(L, Pk, __ldg(bk + 1)); Pk = fabs(fma(L, Pk, __ldg(bk)));
        const double den = fma(Pk, fma(Pk, a2, 2.0 * a1), a0);
        mu = fma(sX[k * BLKD + t] * (Pk * Pk), pdm::rcp(den), mu);
      }
      g_mu[p] = sqT * mu;
    }
    if (g_Dm) {
      #pragma unroll 1
      for (int k = 0; k < NSP; ++k) sV[k * BLKD + t] = 0.0;
      // pairs {k, j}, j > k, in row order k: pyro_tr_pair + 5 (k (N-1) - k (k-1)/2 + j - k - 1);
      // rows k and k+1 are taken together so that each X_j load and each update
      // of the sum of species j serves two pairs
      int k = 0;
      #pragma unroll 1
      for (; k + 1 < NSP - 1; k += 2) {
        const double* a0p = pyro_tr_pair + 5 * (k * (NSP - 1) - k * (k - 1) / 2);   // pair (k, k+1)
        const double* a1p = a0p + 5 * (NSP - 1 - k);                                // pair (k+1, k+2)
        const double xk = sX[k * BLKD + t], xk1 = sX[(k + 1) * BLKD + t];
        double sk, sk1;
        {   // the pair (k, k+1)
          double pk = fma(L, __ldg(a0p + 4), __ldg(a0p + 3));
          pk = fma(L, pk, __ldg(a0p + 2)); pk = fma(L, pk, __ldg(a0p + 1)); pk = fma(L, pk, __ldg(a0p));
          const double r = pdm::rcp(pk);
          sk = fma(xk1, r, sV[k * BLKD + t]);
          sk1 = fma(xk, r, sV[(k + 1) * BLKD + t]);
        }
        const double* a = a0p + 5;
        const double* b = a1p;
        #pragma unroll 2
        for (int j = k + 2; j < NSP; ++j, a += 5, b += 5) {
          double pa = fma(L, __ldg(a + 4), __ldg(a + 3));
          double pb = fma(L, __ldg(b + 4), __ldg(b + 3));
          pa = fma(L, pa, __ldg(a + 2)); pb = fma(L, pb, __ldg(b + 2));
          pa = fma(L, pa, __ldg(a + 1)); pb = fma(L, pb, __ldg(b + 1));
          pa = fma(L, pa, __ldg(a));     pb = fma(L, pb, __ldg(b));
          const double ra = pdm::rcp(pa), rb = pdm::rcp(pb);
          const double xj = sX[j * BLKD + t];
          sk = fma(xj, ra, sk);
          sk1 = fma(xj, rb, sk1);
          sV[j * BLKD + t] = fma(xk, ra, fma(xk1, rb, sV[j * BLKD + t]));
        }
        sV[k * BLKD + t] = sk;
        sV[(k + 1) * BLKD + t] = sk1;
      }
      for (; k < NSP - 1; ++k) {     // a last single row
        const double* a = pyro_tr_pair + 5 * (k * (NSP - 1) - k * (k - 1) / 2);
        const double xk = sX[k * BLKD + t];
        double sk = sV[k * BLKD + t];
        for (int j = k + 1; j < NSP; ++j, a += 5) {
          double pk = fma(L, __ldg(a + 4), __ldg(a + 3));
          pk = fma(L, pk, __ldg(a + 2)); pk = fma(L, pk, __ldg(a + 1)); pk = fma(L, pk, __ldg(a));
          const double r = pdm::rcp(pk);
          sk = fma(sX[j * BLKD + t], r, sk);
          sV[j * BLKD + t] = fma(xk, r, sV[j * BLKD + t]);
        }
        sV[k * BLKD + t] = sk;
      }
      #pragma unroll 1
      for (int k = 0; k < NSP; ++k)
        g_Dm[(i64)k * n + p] = (1.0 - __ldg(Yp + (i64)k * n)) * sqT * pdm::rcp(sV[k * BLKD + t]);
    }
  }
}
)";
}

// ---------------------------------------------------------------------------
// Crank-Nicolson step (Sec. A.3.2, Eqs. crank_nicol_rhs to crank_nicol_jac):
// preparation, batched dense solve of the Newton system, completion.  The
// Newton system itself is assembled by the Jacobian kernel in mode CN.
// ---------------------------------------------------------------------------
void emit_cn_kernels(Src& s, const Mechanism& m, const std::vector<SpeciesCoef>& C) {
  int N = m.n_species();
  // preparation: e = e(T^m, Y^m) (Eq. int_energy), iterate Y <- Y^m, T <- T^m
  s << "\nextern \"C\" __global__ void __launch_bounds__(BLKD) pyro_cn_prep(i64 cnt, i64 n,\n"
       "    const double* __restrict__ g_Tin, const double* __restrict__ g_Yin, double* __restrict__ g_Tout,\n"
       "    double* __restrict__ g_Yout, double* __restrict__ g_e, int* __restrict__ g_state, int* __restrict__ g_it,\n"
       "    int* __restrict__ g_list, int* __restrict__ g_count) {\n"
       "  for (i64 p = (i64)blockIdx.x * BLKD + threadIdx.x; p < cnt; p += (i64)gridDim.x * BLKD) {\n"
       "    const double* Yp = g_Yin + p;\n    const double T = g_Tin[p];\n"
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
       "    if (g_Yout != g_Yin) {\n"
       "      #pragma unroll 1\n      for (int k = 0; k < NSP; ++k) g_Yout[(i64)k * n + p] = Yp[(i64)k * n];\n    }\n"
       "    g_Tout[p] = T;\n    g_state[p] = 0;\n    g_it[p] = 0;\n    g_list[p] = (int)p;\n  }\n"
       "  if (blockIdx.x == 0 && threadIdx.x == 0) *g_count = (int)cnt;\n}\n";

  // batched solve: one warp per state, CN_W states per block (matrices in groups of CN_G)
  s << R"(
// Newton update of one Crank-Nicolson iteration, one warp per state: solve
// (I - dt/(2 rho) J) dY = -F by LU with partial pivoting in FP32 and `refine`
// steps of iterative refinement whose residuals b - A x are formed in FP64 from
// the FP64 matrix; then Y += dY and the state's Newton bookkeeping (stop once
// max_k |dY_k| <= tol, after one further step: the rule of the temperature solve).
// Each row is scaled by a power of two that brings its largest entry into
// [0.5, 1) before it is rounded to FP32; row maxima, scaling and rounding (to
// nearest even) work on the bit patterns in integer arithmetic.  The trailing
// update of the factorisation spreads the submatrix over the lanes as a 16 x 2
// tile (rows l/2 mod 16, columns l mod 2), so with the leading dimension
// CN_LDA = 2 * odd the tile's shared-memory accesses are conflict-free.
#define CN_NJ ((NSP + 31) / 32)
#define CN_LDA (((NSP + 1) / 2) % 2 == 1 ? 2 * ((NSP + 1) / 2) : 2 * ((NSP + 1) / 2) + 2)

// |v| 2^-e rounded to FP32 (round to nearest even), with v's bits; 0 below FP32's normal range
__device__ __forceinline__ float pyro_scaled_f32(long long bits, int e) {
  const unsigned long long a = (unsigned long long)bits & 0x7fffffffffffffffull;
  const int ex = (int)(a >> 52);
  if (ex == 2047) return __int_as_float(0x7fc00000);   // Inf or NaN: NaN (the pivot search rejects it)
  int fe = ex - 1023 - e + 127;
  if (ex == 0 || fe <= 0) return 0.0f;
  unsigned long long mant = a & 0xfffffffffffffull;
  unsigned int m23 = (unsigned int)(mant >> 29);
  const unsigned int rem = (unsigned int)(mant & 0x1fffffffu);
  if (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) {
    ++m23;
    if (m23 == 0x800000u) { m23 = 0; ++fe; }
  }
  const unsigned int fb = ((unsigned int)(bits >> 32) & 0x80000000u) | ((unsigned int)min(fe, 255) << 23) |
                          (fe >= 255 ? 0u : m23);
  return __uint_as_float(fb);
}

// mode 0: factor the matrix of slot q.  mode 1 (chord, iterations that re-assemble):
// factor state p's matrix (at index p) and keep its FP32 factors, pivots and row
// exponents in g_fac.  mode 2 (chord, the iterations between): reuse state p's kept
// factors and refine against its kept FP64 matrix.
#define CN_FAC_WORDS (NSP * CN_LDA + 2 * NSP)
extern "C" __global__ void __launch_bounds__(CN_W * 32) pyro_cn_solve(i64 cnt, i64 n,
    const double* __restrict__ g_A, const double* __restrict__ g_b, double* __restrict__ g_Y,
    int* __restrict__ g_state, int* __restrict__ g_it, double tol, int max_newton, int refine,
    unsigned long long* __restrict__ g_fail, const int* __restrict__ g_list, const int* __restrict__ g_count,
    int* __restrict__ g_list_next, int* __restrict__ g_count_next, int mode, float* __restrict__ g_fac) {
  extern __shared__ double s_cn[];
  const int wi = threadIdx.x >> 5, l = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  double* sx = s_cn + wi * NSP;                       // solution (FP64)
  double* sr = s_cn + (CN_W + wi) * NSP;              // right-hand side / residual (FP64)
  float* fb = (float*)(s_cn + 2 * CN_W * NSP);
  float* sM = fb + wi * (NSP * CN_LDA);                                // scaled LU factors
  float* sv = fb + CN_W * NSP * CN_LDA + wi * NSP;                      // FP32 solve vector
  float* sq = fb + CN_W * NSP * CN_LDA + CN_W * NSP + wi * NSP;         // reciprocal pivots
  int* spiv = (int*)(fb + CN_W * NSP * CN_LDA + 2 * CN_W * NSP) + wi * NSP;   // pivot rows
  int* se = spiv + CN_W * NSP;                                          // row scale exponents
  const int tr = l >> 1, tc = l & 1;                  // lane's place in the 16 x 2 update tile
  const i64 na = *g_count;
  for (i64 q = ((i64)blockIdx.x * CN_W + wi); q < na; q += (i64)gridDim.x * CN_W) {
    const i64 p = g_list[q];
    const int st = g_state[p];
    if (st >= 3) continue;
    const i64 qa = mode == 0 ? q : p;             // where this state's FP64 matrix is
    const double* Ag = g_A + (qa / CN_G) * (i64)(NSP * NSP * CN_G) + (qa % CN_G);
    float* fac = g_fac + p * (i64)CN_FAC_WORDS;
    bool sing = false;
    if (mode == 2) {
      // kept factors: LU (rows of CN_LDA floats), pivots, row exponents
      for (int e = l; e < NSP * CN_LDA; e += 32) sM[e] = fac[e];
      for (int k = l; k < NSP; k += 32) {
        spiv[k] = __float_as_int(fac[NSP * CN_LDA + k]);
        se[k] = __float_as_int(fac[NSP * CN_LDA + NSP + k]);
        sq[k] = __frcp_rn(fac[k * CN_LDA + k]);
        sr[k] = g_b[(i64)k * cnt + q]; sx[k] = 0.0;
      }
      __syncwarp();
    } else {
    // scaled FP32 copy of the matrix, one row at a time
    #pragma unroll 2
    for (int i = 0; i < NSP; ++i) {
      long long v[CN_NJ];
      unsigned long long mx = 0;
      #pragma unroll
      for (int t = 0; t < CN_NJ; ++t) {
        const int j = l + 32 * t;
        v[t] = j < NSP ? __double_as_longlong(__ldg(Ag + (i64)(i * NSP + j) * CN_G)) : 0ll;
        const unsigned long long a = (unsigned long long)v[t] & 0x7fffffffffffffffull;
        mx = a > mx ? a : mx;
      }
      for (int o = 16; o; o >>= 1) {
        const unsigned long long om = __shfl_xor_sync(FULL, mx, o);
        mx = om > mx ? om : mx;
      }
      const int e = mx ? (int)(mx >> 52) - 1022 : 0;   // 2^(e-1) <= max |A_ij| < 2^e
      #pragma unroll
      for (int t = 0; t < CN_NJ; ++t) {
        const int j = l + 32 * t;
        if (j < NSP) sM[i * CN_LDA + j] = pyro_scaled_f32(v[t], e);
      }
      if (l == 0) se[i] = e;
    }
    for (int k = l; k < NSP; k += 32) { sr[k] = g_b[(i64)k * cnt + q]; sx[k] = 0.0; }
    __syncwarp();
    // LU factorisation with partial pivoting (row exchanges applied to the whole rows)
    for (int k = 0; k < NSP; ++k) {
      float bv = -1.0f;
      int bi = k;
      for (int i = k + l; i < NSP; i += 32) {
        const float v = fabsf(sM[i * CN_LDA + k]);
        if (v > bv) { bv = v; bi = i; }
      }
      for (int o = 16; o; o >>= 1) {
        const float ov = __shfl_xor_sync(FULL, bv, o);
        const int oi = __shfl_xor_sync(FULL, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (!(bv > 0.0f) || bv > 3.0e38f) { sing = true; break; }
      if (bi != k)
        for (int j = l; j < NSP; j += 32) {
          const float a = sM[k * CN_LDA + j];
          sM[k * CN_LDA + j] = sM[bi * CN_LDA + j];
          sM[bi * CN_LDA + j] = a;
        }
      if (l == 0) spiv[k] = bi;
      __syncwarp();
      const float inv = __frcp_rn(sM[k * CN_LDA + k]);
      if (l == 0) sq[k] = inv;
      for (int i = k + 1 + l; i < NSP; i += 32) sM[i * CN_LDA + k] *= inv;
      __syncwarp();
      // trailing update A[i][j] -= A[i][k] A[k][j], i, j > k, on the 16 x 2 tile
      const int m = NSP - 1 - k;
      float li[(NSP + 15) / 16];
      #pragma unroll
      for (int u = 0; u < (NSP + 15) / 16; ++u) {
        const int i = k + 1 + tr + 16 * u;
        li[u] = i < NSP ? sM[i * CN_LDA + k] : 0.0f;
      }
      for (int jj = tc; jj < m; jj += 2) {
        const int j = k + 1 + jj;
        const float uj = sM[k * CN_LDA + j];
        #pragma unroll
        for (int u = 0; u < (NSP + 15) / 16; ++u) {
          if (16 * u < m) {                          // uniform across the warp
            const int i = k + 1 + tr + 16 * u;
            if (i < NSP) sM[i * CN_LDA + j] = fmaf(-li[u], uj, sM[i * CN_LDA + j]);
          }
        }
      }
      __syncwarp();
    }
    if (mode == 1 && !sing) {
      for (int e = l; e < NSP * CN_LDA; e += 32) fac[e] = sM[e];
      for (int k = l; k < NSP; k += 32) {
        fac[NSP * CN_LDA + k] = __int_as_float(spiv[k]);
        fac[NSP * CN_LDA + NSP + k] = __int_as_float(se[k]);
      }
    }
    }   // factorisation (modes 0, 1)
    double dmax = 0.0;
    if (!sing) {
      for (int pass = 0; pass <= refine; ++pass) {
        if (pass > 0) {   // residual r = b - A x in FP64, one row per lane
          for (int i = l; i < NSP; i += 32) {
            const double* Ai = Ag + (i64)(i * NSP) * CN_G;
            double acc0 = g_b[(i64)i * cnt + q], acc1 = 0.0;
            int j = 0;
            for (; j + 1 < NSP; j += 2) {
              acc0 = fma(-__ldg(Ai + (i64)j * CN_G), sx[j], acc0);
              acc1 = fma(-__ldg(Ai + (i64)(j + 1) * CN_G), sx[j + 1], acc1);
            }
            if (j < NSP) acc0 = fma(-__ldg(Ai + (i64)j * CN_G), sx[j], acc0);
            sr[i] = acc0 + acc1;
          }
          __syncwarp();
        }
        for (int k = l; k < NSP; k += 32) sv[k] = __double2float_rn(ldexp(sr[k], -se[k]));   // row scaling
        __syncwarp();
        if (l == 0)
          for (int k = 0; k < NSP; ++k) {
            const int pk = spiv[k];
            if (pk != k) { const float a = sv[k]; sv[k] = sv[pk]; sv[pk] = a; }
          }
        __syncwarp();
        for (int k = 0; k < NSP - 1; ++k) {        // unit lower triangle
          const float vk = sv[k];
          for (int i = k + 1 + l; i < NSP; i += 32) sv[i] = fmaf(-sM[i * CN_LDA + k], vk, sv[i]);
          __syncwarp();
        }
        for (int k = NSP - 1; k >= 0; --k) {       // upper triangle
          const float vk = sv[k] * sq[k];
          __syncwarp();
          if (l == 0) sv[k] = vk;
          for (int i = l; i < k; i += 32) sv[i] = fmaf(-sM[i * CN_LDA + k], vk, sv[i]);
          __syncwarp();
        }
        for (int k = l; k < NSP; k += 32) sx[k] += (double)sv[k];
        __syncwarp();
      }
      for (int k = l; k < NSP; k += 32) {
        const double dx = sx[k];
        g_Y[(i64)k * n + p] += dx;
        const double a = fabs(dx);
        dmax = (a > dmax || a != a) ? a : dmax;
      }
      for (int o = 16; o; o >>= 1) {
        const double od = __shfl_xor_sync(FULL, dmax, o);
        dmax = (od > dmax || od != od) ? od : dmax;
      }
    }
    if (l == 0) {
      const int it = g_it[p] + 1;
      g_it[p] = it;
      int ns;
      if (sing || !(dmax == dmax)) ns = 4;
      else if (st == 2) ns = 3;
      else if (dmax <= tol) ns = 2;
      else if (it >= max_newton) ns = 4;
      else ns = 1;
      g_state[p] = ns;
      if (ns == 4) atomicAdd(g_fail, 1ull);
      if (ns < 3) g_list_next[atomicAdd(g_count_next, 1)] = (int)p;
    }
    __syncwarp();
  }
}

// completion: T from (e, Y^{m+1}) and the Newton step counts (-1: failed)
extern "C" __global__ void __launch_bounds__(BLKD) pyro_cn_finish(i64 cnt, i64 n, const double* __restrict__ g_e,
    const double* __restrict__ g_Y, double* __restrict__ g_T, const int* __restrict__ g_state,
    const int* __restrict__ g_it, int* __restrict__ g_iters, int max_iter, double tol,
    unsigned long long* __restrict__ g_fail) {
  const float tolf = (float)tol;
  for (i64 p = (i64)blockIdx.x * BLKD + threadIdx.x; p < cnt; p += (i64)gridDim.x * BLKD) {
    int st = g_state[p];
    if (st == 3) {
      int tit;
      const double T = pyro_tsolve<false>(g_Y + p, n, g_e[p], g_T[p], max_iter, tolf, &tit);
      if (tit < 0) { st = 4; atomicAdd(g_fail, 1ull); } else { g_T[p] = T; }
    } else if (st != 4) {
      st = 4;
      atomicAdd(g_fail, 1ull);
    }
    if (g_iters) g_iters[p] = st == 3 ? g_it[p] : -1;
  }
}
)";
}

// Right-hand side only (the chord variant of the Crank-Nicolson Newton iteration
// keeps the matrix of its first iterate): T from (e, Y), omega by the forward
// path, -F = c + (dt/2rho) W omega - Y into slot q.  Same state/list protocol as
// pyro_cn_assemble.
void emit_cn_residual_kernel(Src& s, const Mechanism& m, const std::vector<SpeciesCoef>& C, bool acc_mem) {
  const int N = m.n_species();
  s << "\nextern \"C\" __global__ void __launch_bounds__(BLKD) pyro_cn_residual(i64 cnt, i64 n,\n"
       "    const double* __restrict__ g_rho, const double* __restrict__ g_e, const double* __restrict__ g_Y,\n"
       "    const double* __restrict__ g_c, double* __restrict__ g_T, int* __restrict__ g_state, double dt,\n"
       "    int max_iter, double tol, double* __restrict__ g_b, unsigned long long* __restrict__ g_fail,\n"
       "    const int* __restrict__ g_list, const int* __restrict__ g_count, int* __restrict__ g_count_next) {\n"
       "  __shared__ double s_exp[512];\n  __shared__ double s_log[256];\n  extern __shared__ double s_dyn[];\n"
       "  double* sL = s_dyn; double* sA = sL + NSP * BLKD;\n"
       "  pyro_load_tables(s_exp, s_log);\n  __syncthreads();\n  const int t = threadIdx.x;\n"
       "  const float tolf = (float)tol;\n  const i64 na = *g_count;\n"
       "  if (blockIdx.x == 0 && t == 0) *g_count_next = 0;\n"
       "  for (i64 q = (i64)blockIdx.x * BLKD + t; q < na; q += (i64)gridDim.x * BLKD) {\n"
       "    const i64 p = g_list[q];\n"
       "    const double* Yp = g_Y + p;\n    const double rho = g_rho[p];\n"
       "    int tit;\n"
       "    const double T = pyro_tsolve<false>(Yp, n, g_e[p], g_T[p], max_iter, tolf, &tit);\n"
       "    if (tit < 0) { g_state[p] = 4; atomicAdd(g_fail, 1ull); continue; }\n"
       "    g_T[p] = T;\n"
       "    const double lnT = pdm::log(T, s_log);\n    const double invT = pdm::rcp(T);\n"
       "    const bool hi = pdm::to_float_trunc(T) >= (float)TMID;\n";
  Src r;
  emit_species_forward(r, m, C);
  if (has_plog(m))
    r << "    const double lnp = lnT + pdm::log(rho * ysum, s_log) + " << lit((double)logl(R_GAS)) << ";\n";
  // large mechanisms: the species sums accumulate in the right-hand side itself
  g_acc.mem = acc_mem;
  g_acc.base = "Bq";
  g_acc.stride = "cnt";
  if (acc_mem) r << "    double* Bq = g_b + q;\n";
  emit_acc_init(r, "w", N);
  for (auto& grp : reaction_groups(m)) emit_reaction_group(r, m, grp);
  s << r.o.str();
  s << "    const double hh = 0.5 * dt * pdm::rcp(rho);\n";
  for (int k = 0; k < N; ++k)
    s << "    g_b[(i64)" << k << " * cnt + q] = (g_c[(i64)" << k << " * cnt + p] + (hh * " << lit(m.species[k].W)
      << ") * " << acc("w", k) << ") - __ldg(Yp + (i64)" << k << " * n);\n";
  s << "  }\n}\n";
  g_acc.mem = false;
  g_acc.stride = "n";
}

// ---------------------------------------------------------------------------
// learned initial guess: BF16 tensor-core MLP inference fused into the
// temperature kernel (mma.sync m16n8k16, FP32 accumulation)
// ---------------------------------------------------------------------------
void emit_mlp(Src& s, const Mechanism& m) {
  int N = m.n_species();
  if (N + 1 > 64) return;       // the learned guess supports up to 63 species
  s << "\n#define MLP_D " << (N + 1) << "\n";
  s << R"(
// bf16 helpers on bit patterns (round to nearest even for finite values)
__device__ __forceinline__ unsigned pyro_f2bf(float f) {
  unsigned u = __float_as_uint(f);
  return (u + 0x7fffu + ((u >> 16) & 1u)) >> 16;
}
__device__ __forceinline__ float pyro_bf2f(unsigned h) { return __uint_as_float(h << 16); }
// SiLU z / (1 + e^-z) with the hardware exp2 and reciprocal (a few ulp of FP32):
// the result is rounded to bf16 (8 significant bits) right after
__device__ __forceinline__ float pyro_silu(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

// one 16x8x16 BF16 MMA with FP32 accumulation
__device__ __forceinline__ void pyro_mma(float* c, unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};\n"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

#define MLP_LD 36   // 32-bit words per staged row (64 bf16 + 8 pad): conflict-free fragments

struct PyroMlpSmem {
  unsigned W1[64 * MLP_LD];     // [out][in] bf16 pairs
  unsigned W2[64 * MLP_LD];
  float b1[64], b2[64], w3[64];
  float b3, e_mean, e_inv, T_mean, T_std;
  unsigned act[BLK / 32][32 * MLP_LD];   // per warp: 32 points x 64 features (bf16 pairs)
};

__device__ __forceinline__ void pyro_mlp_load(PyroMlpSmem& S, const unsigned short* __restrict__ wb,
                                              const float* __restrict__ wf, const float* __restrict__ norm) {
  const int D = MLP_D;
  const int oW1 = 0, ob1 = 64 * D, oW2 = ob1 + 64, ob2 = oW2 + 64 * 64, ow3 = ob2 + 64, ob3 = ow3 + 64;
  for (int q = threadIdx.x; q < 64 * 32; q += blockDim.x) {
    int o = q >> 5, w = q & 31, i0 = 2 * w, i1 = 2 * w + 1;
    unsigned lo = i0 < D ? wb[oW1 + o * D + i0] : 0u, hi = i1 < D ? wb[oW1 + o * D + i1] : 0u;
    S.W1[o * MLP_LD + w] = lo | (hi << 16);
    S.W2[o * MLP_LD + w] = (unsigned)wb[oW2 + o * 64 + i0] | ((unsigned)wb[oW2 + o * 64 + i1] << 16);
  }
  for (int o = threadIdx.x; o < 64; o += blockDim.x) {
    S.b1[o] = wf[ob1 + o]; S.b2[o] = wf[ob2 + o]; S.w3[o] = pyro_bf2f(wb[ow3 + o]);
  }
  if (threadIdx.x == 0) {
    S.b3 = wf[ob3]; S.e_mean = norm[0]; S.e_inv = 1.0f / norm[1]; S.T_mean = norm[2]; S.T_std = norm[3];
  }
}

// one layer for the warp's 32 points: act (K = 64) -> act, y = bf16(silu(W act + b))
__device__ __forceinline__ void pyro_mlp_layer(unsigned* act, const unsigned* W, const float* b, int lane) {
  const int g = lane >> 2, t = lane & 3;
  float c[2][8][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) c[mt][nt][q] = 0.0f;
#pragma unroll
  for (int kt = 0; kt < 4; ++kt) {
    unsigned a[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const unsigned* r0 = act + (mt * 16 + g) * MLP_LD + kt * 8 + t;
      const unsigned* r1 = r0 + 8 * MLP_LD;
      a[mt][0] = r0[0]; a[mt][1] = r1[0]; a[mt][2] = r0[4]; a[mt][3] = r1[4];
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const unsigned* wr = W + (nt * 8 + g) * MLP_LD + kt * 8 + t;
      unsigned b0 = wr[0], b1 = wr[4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) pyro_mma(c[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
    }
  }
  __syncwarp();
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      int col = nt * 8 + 2 * t;
      float y0 = pyro_silu(c[mt][nt][0] + b[col]), y1 = pyro_silu(c[mt][nt][1] + b[col + 1]);
      float y2 = pyro_silu(c[mt][nt][2] + b[col]), y3 = pyro_silu(c[mt][nt][3] + b[col + 1]);
      act[(mt * 16 + g) * MLP_LD + nt * 4 + t] = pyro_f2bf(y0) | (pyro_f2bf(y1) << 16);
      act[(mt * 16 + g + 8) * MLP_LD + nt * 4 + t] = pyro_f2bf(y2) | (pyro_f2bf(y3) << 16);
    }
  __syncwarp();
}

// Network output y (normalised) for this lane's point; all 32 lanes must call.
__device__ __forceinline__ float pyro_mlp_eval(PyroMlpSmem& S, double e, const double* __restrict__ Yp, i64 n,
                                               bool valid) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned* act = S.act[warp];
  unsigned* row = act + lane * MLP_LD;
  float x0 = valid ? (float)((e - (double)S.e_mean) * (double)S.e_inv) : 0.0f;
  unsigned prev = pyro_f2bf(x0);
)";
  // features: x_0 = normalised e, x_{1+k} = Y_k; packed in bf16 pairs
  for (int i = 1; i < 64; ++i) {
    std::string v = i <= N ? "(valid ? pyro_f2bf(pdm::to_float_trunc(__ldg(Yp + (i64)" + std::to_string(i - 1) +
                                 " * n)) * " + std::to_string(N) + ".0f) : 0u)" : "0u";
    if (i % 2 == 1) s << "  row[" << (i / 2) << "] = prev | (" << v << " << 16);\n";
    else s << "  prev = " << v << ";\n";
  }
  s << R"(  __syncwarp();
  pyro_mlp_layer(act, S.W1, S.b1, lane);
  pyro_mlp_layer(act, S.W2, S.b2, lane);
  float y = S.b3;
#pragma unroll 8
  for (int w = 0; w < 32; ++w) {
    unsigned v = row[w];
    y = fmaf(S.w3[2 * w], pyro_bf2f(v & 0xffffu), y);
    y = fmaf(S.w3[2 * w + 1], pyro_bf2f(v >> 16), y);
  }
  __syncwarp();
  return y;
}

// Guess of the network alone (raw normalised output and the clipped temperature)
extern "C" __global__ void __launch_bounds__(BLK) pyro_mlp_guess(i64 n, const double* __restrict__ g_e,
    const double* __restrict__ g_Y, const unsigned short* __restrict__ wb, const float* __restrict__ wf,
    const float* __restrict__ norm, double* __restrict__ g_y, double* __restrict__ g_T) {
  __shared__ PyroMlpSmem S;
  pyro_mlp_load(S, wb, wf, norm);
  __syncthreads();
  for (i64 base = (i64)blockIdx.x * BLK; base < n; base += (i64)gridDim.x * BLK) {
    i64 p = base + threadIdx.x;
    bool valid = p < n;
    i64 pp = valid ? p : n - 1;
    float y = pyro_mlp_eval(S, g_e[pp], g_Y + pp, n, valid);
    if (valid) {
      g_y[p] = (double)y;
      g_T[p] = (double)fminf(fmaxf(fmaf(S.T_std, y, S.T_mean), 200.0f), 3500.0f);
    }
  }
}

// Temperature with the learned initial guess; falls back to 1200 K where the
// Newton iteration from the guess does not converge.
extern "C" __global__ void __launch_bounds__(BLK) pyro_temperature_mlp(i64 n, const double* __restrict__ g_e,
    const double* __restrict__ g_Y, const unsigned short* __restrict__ wb, const float* __restrict__ wf,
    const float* __restrict__ norm, int max_iter, double tol, double* __restrict__ g_T, int* __restrict__ g_iters,
    unsigned long long* __restrict__ g_fail) {
  __shared__ PyroMlpSmem S;
  pyro_mlp_load(S, wb, wf, norm);
  __syncthreads();
  const float tolf = (float)tol;
  for (i64 base = (i64)blockIdx.x * BLK; base < n; base += (i64)gridDim.x * BLK) {
    i64 p = base + threadIdx.x;
    bool valid = p < n;
    i64 pp = valid ? p : n - 1;
    double e = g_e[pp];
    float y = pyro_mlp_eval(S, e, g_Y + pp, n, valid);
    if (!valid) continue;
    double T0 = (double)fminf(fmaxf(fmaf(S.T_std, y, S.T_mean), 200.0f), 3500.0f);
    int it;
    double T = pyro_tsolve<false>(g_Y + p, n, e, T0, max_iter, tolf, &it);
    if (it < 0) {
      int it2;
      T = pyro_tsolve<false>(g_Y + p, n, e, 1200.0, max_iter, tolf, &it2);
      it = it2 < 0 ? -1 : it2 + max_iter + 1;
    }
    g_T[p] = T;
    if (g_iters) g_iters[p] = it;
    if (it < 0) atomicAdd(g_fail, 1ull);
  }
}
)";
}

}  // namespace

EmitResult emit_module(const Mechanism& m, const EmitOptions& opt) {
  // the emitters keep per-emission state in file-scope variables (accumulator
  // mode, folded sums, exponential flavour): one emission at a time, so that
  // handles loaded from several host threads stay independent
  static std::mutex emit_mu;
  std::lock_guard<std::mutex> lock(emit_mu);
  EmitResult out;
  g_exp_ops = opt.exp_ops;
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

  // ---- enthalpy and c_p (h_k = e_k + R T / W_k) --------------------------------
  s << "\nextern \"C\" __global__ void __launch_bounds__(BLK) pyro_enthalpy(i64 n, const double* __restrict__ g_T,\n"
       "    const double* __restrict__ g_Y, double* __restrict__ g_h, double* __restrict__ g_cp) {\n"
       "  for (i64 p = (i64)blockIdx.x * BLK + threadIdx.x; p < n; p += (i64)gridDim.x * BLK) {\n"
       "    const double* Yp = g_Y + p;\n    const double T = g_T[p];\n"
       "    const bool hi = pdm::to_float_trunc(T) >= (float)TMID;\n"
       "    double B0 = 0.0, B1 = 0.0, B2 = 0.0, B3 = 0.0, B4 = 0.0, B5 = 0.0;\n";
  for (int k = 0; k < N; ++k) {
    s << "    { double y = __ldg(Yp + (i64)" << k << " * n);";
    for (int q = 0; q < 6; ++q) {
      double v[2] = {C[k].d[0][q], C[k].d[1][q]};
      if (q == 1) { v[0] += 1.0 / m.species[k].W; v[1] += 1.0 / m.species[k].W; }
      s << " B" << q << " = fma(y, " << sel(v) << ", B" << q << ");";
    }
    s << " }\n";
  }
  s << "    g_h[p] = " << lit((double)R_GAS) << " * fma(T, fma(T, fma(T, fma(T, fma(T, B5, B4), B3), B2), B1), B0);\n"
       "    if (g_cp) g_cp[p] = " << lit((double)R_GAS)
    << " * fma(T, fma(T, fma(T, fma(T, 5.0 * B5, 4.0 * B4), 3.0 * B3), 2.0 * B2), B1);\n  }\n}\n";

  // ---- temperature --------------------------------------------------------------
  s << R"(
extern "C" __global__ void __launch_bounds__(BLK) pyro_temperature(i64 n, const double* __restrict__ g_e,
    const double* __restrict__ g_Y, const double* __restrict__ g_guess, double T_guess, int max_iter, double tol,
    double* __restrict__ g_T, int* __restrict__ g_iters, unsigned long long* __restrict__ g_fail) {
  const float tolf = (float)tol;
  for (i64 p = (i64)blockIdx.x * BLK + threadIdx.x; p < n; p += (i64)gridDim.x * BLK) {
    int it;
    double T = pyro_tsolve<false>(g_Y + p, n, g_e[p], g_guess ? g_guess[p] : T_guess, max_iter, tolf, &it);
    g_T[p] = T;
    if (g_iters) g_iters[p] = it;
    if (it < 0) atomicAdd(g_fail, 1ull);
  }
}

// Temperature from the mixture enthalpy (the enthalpy variant of the inversion)
extern "C" __global__ void __launch_bounds__(BLK) pyro_temperature_h(i64 n, const double* __restrict__ g_h,
    const double* __restrict__ g_Y, const double* __restrict__ g_guess, double T_guess, int max_iter, double tol,
    double* __restrict__ g_T, int* __restrict__ g_iters, unsigned long long* __restrict__ g_fail) {
  const float tolf = (float)tol;
  for (i64 p = (i64)blockIdx.x * BLK + threadIdx.x; p < n; p += (i64)gridDim.x * BLK) {
    int it;
    double T = pyro_tsolve<true>(g_Y + p, n, g_h[p], g_guess ? g_guess[p] : T_guess, max_iter, tolf, &it);
    g_T[p] = T;
    if (g_iters) g_iters[p] = it;
    if (it < 0) atomicAdd(g_fail, 1ull);
  }
}
)";

  // ---- learned initial guess (inference fused into the temperature kernel) --------
  emit_mlp(s, m);
  out.stats["mlp_supported"] = (N + 1 <= 64) ? 1 : 0;

  // ---- net production rates (Eq. production_rates) ------------------------------
  Src r;   // count the forward per-point path separately
  r << "\nextern \"C\" __global__ void __launch_bounds__(BLK, MINB) pyro_omega(i64 n, const double* __restrict__ g_rho,\n"
       "    const double* __restrict__ g_Tin, int energy_mode, const double* __restrict__ g_Y,\n"
       "    double* __restrict__ g_Tout, double* __restrict__ g_omega, double T_guess, int max_iter, double tol,\n"
       "    unsigned long long* __restrict__ g_fail, double* __restrict__ g_store) {\n"
       "  __shared__ double s_exp[512];\n  __shared__ double s_log[256];\n"
       "  extern __shared__ double s_dyn[];\n"
       "  double* sL = " << (opt.gstore ? "g_store + (i64)blockIdx.x * 2 * NSP * BLK" : "s_dyn") << ";\n"
       "  double* sA = sL + NSP * BLK;\n"
       "  pyro_load_tables(s_exp, s_log);\n  __syncthreads();\n"
       "  const int t = threadIdx.x;\n  const float tolf = (float)tol;\n"
       "  for (i64 p = (i64)blockIdx.x * BLK + t; p < n; p += (i64)gridDim.x * BLK) {\n"
       "    const double* Yp = g_Y + p;\n    const double rho = g_rho[p];\n"
       "    double T;\n"
       "    if (energy_mode) {\n      int it;\n"
       "      T = pyro_tsolve<false>(Yp, n, g_Tin[p], T_guess, max_iter, tolf, &it);\n"
       "      if (it < 0) atomicAdd(g_fail, 1ull);\n      if (g_Tout) g_Tout[p] = T;\n"
       "    } else {\n      T = g_Tin[p];\n    }\n"
       "    const double lnT = pdm::log(T, s_log);\n    const double invT = pdm::rcp(T);\n"
       "    const bool hi = pdm::to_float_trunc(T) >= (float)TMID;\n";
  r.log_(); r.rcp_();
  emit_species_forward(r, m, C);
  if (has_plog(m)) {
    // mixture pressure for the PLOG reactions: ln p = ln(R T rho sum_k Y_k/W_k) (Eq. eos)
    r << "    const double lnp = lnT + pdm::log(rho * ysum, s_log) + " << lit((double)logl(R_GAS)) << ";\n";
    r.log_(); r.mul(); r.add(2);
  }
  g_acc.mem = opt.acc_mem;
  g_acc.base = "Wp";
  if (opt.acc_mem) r << "    double* Wp = g_omega + p;\n";
  emit_acc_init(r, "w", N);
  for (auto& grp : reaction_groups(m)) emit_reaction_group(r, m, grp);
  if (!opt.acc_mem)
    for (int k = 0; k < N; ++k) r << "    g_omega[(i64)" << k << " * n + p] = w" << k << ";\n";
  g_acc.mem = false;
  r << "  }\n}\n";
  s << r.o.str();

  // ---- derivative kernels: separate translation units (compiled on first use) -------
  // the derivative translation units index shared memory with BLK as well, so
  // their prelude sets BLK to the derivative block size
  Src pre;
  EmitOptions dopt = opt;
  dopt.block = opt.deriv_block;
  emit_prelude(pre, m, dopt);
  pre << "#define BLKD " << opt.deriv_block << "\n";
  {
    Src d; d << pre.o.str(); emit_jvp_kernel(d, m, C, opt.deriv_block, opt); out.group_sources["jvp"] = d.o.str();
    out.stats["jvp_fp64_flops_per_point"] = d.flops();
    out.stats["jvp_fp64_ops_per_point"] = d.ops();
  }
  {
    Src d; d << pre.o.str(); emit_vjp_kernel(d, m, C, opt.deriv_block, opt); out.group_sources["vjp"] = d.o.str();
    out.stats["vjp_fp64_flops_per_point"] = d.flops();
    out.stats["vjp_fp64_ops_per_point"] = d.ops();
  }
  int nslots = 0;
  {
    Src d; d << pre.o.str();
    emit_jacobian_kernel(d, m, C, opt.deriv_block, &nslots, JacMode::TY, opt.dgstore, opt.jac_table);
    out.group_sources["jac"] = d.o.str();
    out.stats["jacobian_fp64_flops_per_point"] = d.flops();
    out.stats["jacobian_fp64_ops_per_point"] = d.ops();
  }
  // Jacobian-type kernels: two per-state species arrays, in shared memory or (large
  // mechanisms) after the slots in the per-block global scratch
  out.jac_slots = nslots;
  out.smem_dyn_bytes_jac = opt.dgstore ? 0 : 2 * N * opt.deriv_block * (int)sizeof(double);
  out.stats["jacobian_rows_from_tables"] = opt.jac_table ? 1 : 0;
  out.stats["jacobian_supported"] = common_tmid(m) ? 1 : 0;
  {
    int ns2 = 0;
    Src d; d << pre.o.str();
    emit_jacobian_kernel(d, m, C, opt.deriv_block, &ns2, JacMode::ADIA, opt.dgstore, opt.jac_table);
    out.group_sources["jad"] = d.o.str();
    out.stats["jacobian_adiabatic_fp64_flops_per_point"] = d.flops();
    out.stats["jacobian_adiabatic_fp64_ops_per_point"] = d.ops();
  }
  if (m.has_transport) {
    Src d;
    EmitOptions topt = opt;
    topt.block = kTransportBlock;
    emit_prelude(d, m, topt);
    d << "#define BLKD " << kTransportBlock << "\n";
    emit_transport_kernel(d, m, kTransportBlock, opt.dgstore);
    out.smem_dyn_bytes_transport = opt.dgstore ? 0 : 3 * N * kTransportBlock * (int)sizeof(double);
    out.group_sources["tr"] = d.o.str();
    const int npair = N * (N - 1) / 2;
    // FP64-pipe operations per state (rcp = 4, log = 7, sqrt counted as 1)
    out.stats["transport_fp64_ops_per_point"] = 7 + 1 + N + 4 + N * 23.0 + 4 + 3.0 * N * N + 13.0 * N + 10.0 * npair + 6.0 * N;
  }
  out.stats["has_transport"] = m.has_transport ? 1 : 0;
  {
    // Crank-Nicolson: temperature solve + Newton-system assembly + batched solve
    int ns2 = 0;
    Src d; d << pre.o.str();
    // shared memory of one state of the batched solve; states per block: as many
    // as fit in 227 KB, at most kCnGroup (2 for 160 species)
    const int half = (N + 1) / 2, lda = half % 2 == 1 ? 2 * half : 2 * half + 2;   // CN_LDA
    const int per_warp = 2 * N * 8 + N * lda * 4 + 4 * N * 4;
    const int cnw = std::max(1, std::min(kCnGroup, (227 * 1024) / per_warp));
    d << "#define CN_G " << kCnGroup << "\n#define CN_W " << cnw << "\n#define opt_mixed "
      << (opt.mixed_newton ? 1 : 0) << "\n";
    std::map<std::string, double> dummy;
    emit_tsolve(d, m, C, opt, dummy);
    emit_jacobian_kernel(d, m, C, opt.deriv_block, &ns2, JacMode::CN, opt.dgstore, opt.jac_table);
    emit_cn_kernels(d, m, C);
    if (opt.cn_residual) emit_cn_residual_kernel(d, m, C, opt.acc_mem);
    out.stats["cn_residual_kernel"] = opt.cn_residual ? 1 : 0;
    out.group_sources["cn"] = d.o.str();
    out.cn_solve_warps = cnw;
    out.stats["cn_solve_warps"] = cnw;
    out.smem_dyn_bytes_cn_solve = cnw * per_warp;
  }
  out.smem_dyn_bytes_deriv = opt.dgstore ? 0 : 4 * N * opt.deriv_block * (int)sizeof(double);
  out.stats["jacobian_scratch_doubles_per_point"] = nslots;
  out.stats["deriv_warp_per_state"] = 0;
  std::string warp_why;
  if (warp_supported(m, &warp_why)) {
    // warp-per-state kernels (compiled on first use: variant=warp)
    WarpEmit w = emit_warp_units(m, opt);
    for (auto& kv : w.sources) out.group_sources[kv.first] = kv.second;
    for (auto& kv : w.stats) out.stats[kv.first] = kv.second;
    out.warp_wpb = w.wpb;
    out.smem_dyn_bytes_warp = w.smem;
    out.stats["deriv_warp_per_state"] = 1;
  }
  out.stats["deriv_block"] = opt.deriv_block;

  out.stats["omega_fp64_ops_per_point"] = r.ops();
  out.stats["omega_fp64_flops_per_point"] = r.flops();
  out.stats["omega_dfma_per_point"] = r.dfma;
  out.stats["omega_dadd_per_point"] = r.dadd;
  out.stats["omega_dmul_per_point"] = r.dmul;
  out.stats["n_species"] = N;
  out.stats["n_reactions"] = m.n_reactions();
  out.stats["block"] = opt.block;
  out.smem_dyn_bytes_omega = opt.gstore ? 0 : 2 * N * opt.block * (int)sizeof(double);
  out.stats["omega_store_global"] = opt.gstore ? 1 : 0;
  out.stats["deriv_store_global"] = opt.dgstore ? 1 : 0;
  out.stats["accumulators_in_memory"] = opt.acc_mem ? 1 : 0;
  out.source = s.o.str();
  out.group_sources["fwd"] = out.source;
  return out;
}

}  // namespace pyro
