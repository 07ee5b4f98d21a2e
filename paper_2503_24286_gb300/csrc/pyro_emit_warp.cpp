// Emitter of the warp-per-state kernels (large mechanisms): one warp evaluates
// one state, its 32 lanes splitting the species and the reactions.
//
// Layout per warp (shared memory): Y_k, L_k = ln(phi_k/W_k), the activities
// a_k = exp(L_k) rho Y_k (the activity form of Eq. equil_constants and
// Eq. reaction_rates used by every kernel of the library, see pyro_emit.cpp),
// one value per reaction (rate of progress, or its tangent), and the partial
// sums of the production rates.  Slot N of the species arrays is a unit
// factor (L = 0, a = 1, Y = 0) that pads short reactions.
//
// Work split, specialised to the mechanism at emit time:
//  * species: lane k handles species k, k + 32, ...; the Newton temperature
//    solve (energy input) collapses the species polynomials with one warp sum
//    per coefficient and iterates uniformly on every lane;
//  * reactions: sorted into classes (plain, third-body, Lindemann, Troe with
//    three or four constants, SRI, PLOG) and, inside a class, by shape; every
//    chunk of 32 consecutive reactions becomes one straight-line block in which
//    lane l evaluates reaction base + l with the chunk's largest shape (shorter
//    reactions read the unit slot), its constants read from emitted tables
//    with the reaction index fastest (coalesced);
//  * production rates (Eq. production_rates): the nonzero (species, reaction)
//    pairs, in species order, are cut into 32 runs of equal length; lane l
//    sums run l with its stoichiometric coefficients, flushing a partial sum at
//    each species boundary, and one pass over the species adds the (at most a
//    few) partial sums of each species.  Fixed order: results are
//    deterministic.
#include "pyro_emit_warp.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <set>
#include <sstream>
#include <tuple>

#include "pyro_emit_common.h"

namespace pyro {

namespace {
using namespace emitc;

enum WKind { WK_PLAIN = 0, WK_TB = 1, WK_LIND = 2, WK_TROE3 = 3, WK_TROE4 = 4, WK_SRI = 5, WK_PLOG = 6 };

int wkind(const Reaction& r) {
  if (r.kind == RX_ARRHENIUS) return WK_PLAIN;
  if (r.kind == RX_THREEBODY) return WK_TB;
  if (r.kind == RX_PLOG) return WK_PLOG;
  if (r.n_sri >= 3) return WK_SRI;
  if (r.n_troe == 4) return WK_TROE4;
  if (r.n_troe >= 3) return WK_TROE3;
  return WK_LIND;
}

struct WChunk {
  int kind = 0, base = 0, count = 0;
  int nf = 1, nr = 1;       // largest reactant / product factor counts
  bool rev = true;          // any reversible reaction in the chunk
  int neff = 0;             // largest number of efficiency terms (eps != 1)
  int nodes = 0;            // PLOG: largest node count
  int eoff = 0, foff = 0;   // offsets into the efficiency / falloff-constant tables
};

struct WPlan {
  int N = 0, M = 0;
  std::vector<int> order;   // slot -> reaction
  std::vector<int> slot;    // reaction -> slot
  std::vector<WChunk> chunks;
  // production-rate gather: [steps][32] packed entries, per species its segments
  int steps = 0, nseg = 0;
  std::vector<unsigned> gent;
  std::vector<int> seg_first, seg_count;
};

int n_eff(const Reaction& r) {
  int c = 0;
  for (auto& e : r.efficiencies) if (e.second != 1.0) ++c;
  return c;
}

int n_factors(const std::vector<std::pair<int, int>>& side) {
  int c = 0;
  for (auto& p : side) c += p.second;
  return c;
}

WPlan make_plan(const Mechanism& m) {
  WPlan P;
  P.N = m.n_species();
  P.M = m.n_reactions();
  const int M = P.M;
  std::vector<std::tuple<int, int, int, int, int, int>> key(M);
  for (int j = 0; j < M; ++j) {
    const Reaction& r = m.reactions[j];
    const int nodes = r.kind == RX_PLOG ? (int)r.plog.size() : 0;
    // class, then larger shapes first so every chunk is as uniform as possible
    key[j] = std::make_tuple(wkind(r), r.reversible ? 0 : 1, -(n_factors(r.reactants) * 4 + n_factors(r.products)),
                             -n_eff(r), -nodes, j);
  }
  std::vector<int> idx(M);
  for (int j = 0; j < M; ++j) idx[j] = j;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return key[a] < key[b]; });
  P.order = idx;
  P.slot.assign(M, 0);
  for (int s = 0; s < M; ++s) P.slot[P.order[s]] = s;
  int eoff = 0, foff = 0;
  for (int s = 0; s < M;) {
    const int kind = wkind(m.reactions[P.order[s]]);
    int e = s;
    while (e < M && e - s < 32 && wkind(m.reactions[P.order[e]]) == kind) ++e;
    WChunk c;
    c.kind = kind; c.base = s; c.count = e - s; c.rev = false; c.nf = 1; c.nr = 1;
    for (int q = s; q < e; ++q) {
      const Reaction& r = m.reactions[P.order[q]];
      c.nf = std::max(c.nf, n_factors(r.reactants));
      if (r.reversible) { c.rev = true; c.nr = std::max(c.nr, n_factors(r.products)); }
      c.neff = std::max(c.neff, n_eff(r));
      if (r.kind == RX_PLOG) c.nodes = std::max(c.nodes, (int)r.plog.size());
    }
    c.eoff = eoff;
    if (kind != WK_PLAIN && kind != WK_PLOG) eoff += 32 * c.neff;
    c.foff = foff;
    const int nfo = kind == WK_LIND ? 3 : kind == WK_TROE3 ? 7 : kind == WK_TROE4 ? 8 : kind == WK_SRI ? 8
                  : kind == WK_PLOG ? 4 * c.nodes + (c.nodes - 1) : 0;
    foff += 32 * nfo;
    P.chunks.push_back(c);
    s = e;
  }
  // gather: nonzero (species, slot, nu) in species order, cut into 32 equal runs
  std::vector<std::vector<std::pair<int, int>>> rows(P.N);
  for (int j = 0; j < M; ++j)
    for (auto& q : net_nu(m.reactions[j]))
      if (q.second) rows[q.first].push_back({P.slot[j], q.second});
  for (auto& r : rows) std::sort(r.begin(), r.end());
  std::vector<std::tuple<int, int, int>> ent;   // (species, slot, nu)
  for (int k = 0; k < P.N; ++k)
    for (auto& e : rows[k]) ent.push_back(std::make_tuple(k, e.first, e.second));
  const int nnz = (int)ent.size();
  P.steps = std::max(1, (nnz + 31) / 32);
  P.gent.assign((size_t)P.steps * 32, 0u);
  P.seg_first.assign(P.N, -1);
  P.seg_count.assign(P.N, 0);
  int seg = 0;
  for (int l = 0; l < 32; ++l) {
    const int a = l * P.steps, b = std::min(nnz, (l + 1) * P.steps);
    for (int q = a; q < b; ++q) {
      const int k = std::get<0>(ent[q]);
      const bool last = q + 1 == b || std::get<0>(ent[q + 1]) != k;
      unsigned e = (unsigned)std::get<1>(ent[q]) | ((unsigned)(std::get<2>(ent[q]) + 4) << 16);
      if (last) {
        if (P.seg_first[k] < 0) P.seg_first[k] = seg;
        P.seg_count[k]++;
        e |= (1u << 19) | ((unsigned)seg << 20);
        ++seg;
      }
      P.gent[(size_t)(q - a) * 32 + l] = e;
    }
  }
  P.nseg = seg;
  return P;
}

template <class T>
void emit_array(std::ostringstream& o, const char* type, const std::string& name, const std::vector<T>& v,
                bool as_lit) {
  o << "__device__ const " << type << " " << name << "[" << std::max<size_t>(v.size(), 1) << "] = {";
  if (v.empty()) o << "0";
  for (size_t i = 0; i < v.size(); ++i) {
    if (i) o << ",";
    if (as_lit) o << lit((double)v[i]);
    else o << v[i];
  }
  o << "};\n";
}

}  // namespace

namespace {

// Tables and device code shared by the warp-per-state kernels of one mechanism,
// and the reaction-phase code: per chunk, R_j (or its tangent) into sR[slot].
struct WarpCommon {
  WPlan P;
  std::string prelude, reaction_code;
};

WarpCommon emit_warp_common(const Mechanism& m, const EmitOptions& opt) {
  WarpCommon W;
  W.P = make_plan(m);
  const WPlan& P = W.P;
  const int N = P.N, M = P.M;
  std::vector<SpeciesCoef> C;
  for (auto& sp : m.species) C.push_back(species_coef(sp));
  std::ostringstream o;
  o << "// Generated for mechanism '" << m.name << "': " << N << " species, " << M
    << " reactions; warp-per-state kernels.\n";
  o << "#include \"pyro_device_math.cuh\"\ntypedef long long i64;\n";
  o << "#define PEXP(x, t) pdm::" << (opt.exp_ops == 4 ? "exp4" : "exp") << "((x), (t))\n";
  o << "#define NSP " << N << "\n#define NRX " << M << "\n#define TMID " << lit(m.species[0].t_mid) << "\n";
  o << "#define GSTEPS " << P.steps << "\n#define NSEG " << P.nseg << "\n";
  // species tables: L_k coefficients [2][7][N+1] (unit slot zero), 1/W, Newton collapse [2][6][N]
  std::vector<double> Lc(2 * 7 * (N + 1), 0.0), dc(2 * 6 * N), invW(N + 1, 0.0);
  std::vector<float> dcf(2 * 6 * N);
  for (int k = 0; k < N; ++k) {
    invW[k] = 1.0 / m.species[k].W;
    for (int r = 0; r < 2; ++r) {
      const double L[7] = {C[k].cl[r], C[k].ci[r], C[k].c0[r], C[k].c1[r], C[k].c2[r], C[k].c3[r], C[k].c4[r]};
      for (int q = 0; q < 7; ++q) Lc[(r * 7 + q) * (N + 1) + k] = L[q];
      for (int q = 0; q < 6; ++q) {
        dc[(r * 6 + q) * N + k] = C[k].d[r][q];
        dcf[(r * 6 + q) * N + k] = (float)C[k].d[r][q];
      }
    }
  }
  emit_array(o, "double", "w_Lc", Lc, true);
  emit_array(o, "double", "w_dc", dc, true);
  {
    o << "__device__ const float w_dcf[" << dcf.size() << "] = {";
    for (size_t i = 0; i < dcf.size(); ++i) o << (i ? "," : "") << litf(dcf[i]);
    o << "};\n";
  }
  emit_array(o, "double", "w_invW", invW, true);
  // reaction tables in slot order: ln A' (minus the reactants' ln W), b, -theta, packed factor indices
  std::vector<double> ta(M), tb(M), tt(M);
  std::vector<unsigned> tfr(M), tfp(M);
  for (int s = 0; s < M; ++s) {
    const Reaction& r = m.reactions[P.order[s]];
    long double lnA = logl((long double)r.A);
    std::vector<int> fr = side_factors(r.reactants), fp = side_factors(r.products);
    for (int i : fr) lnA -= logl((long double)m.species[i].W);
    ta[s] = (double)lnA; tb[s] = r.b; tt[s] = -r.theta;
    unsigned a = 0, b = 0;
    for (int q = 0; q < 3; ++q) {
      a |= (unsigned)(q < (int)fr.size() ? fr[q] : N) << (10 * q);
      b |= (unsigned)(q < (int)fp.size() && r.reversible ? fp[q] : N) << (10 * q);
    }
    tfr[s] = a; tfp[s] = b;
  }
  emit_array(o, "double", "w_lnA", ta, true);
  emit_array(o, "double", "w_b", tb, true);
  emit_array(o, "double", "w_mth", tt, true);
  emit_array(o, "unsigned", "w_fr", tfr, false);
  emit_array(o, "unsigned", "w_fp", tfp, false);
  // per-chunk efficiency terms [chunk][q][lane] and falloff / PLOG constants [chunk][field][lane]
  std::vector<unsigned short> ei;
  std::vector<double> ec, fo;
  for (auto& c : P.chunks) {
    if (c.kind != WK_PLAIN && c.kind != WK_PLOG) {
      std::vector<unsigned short> bi((size_t)32 * c.neff, (unsigned short)N);
      std::vector<double> bc((size_t)32 * c.neff, 0.0);
      for (int l = 0; l < c.count; ++l) {
        const Reaction& r = m.reactions[P.order[c.base + l]];
        int q = 0;
        for (auto& e : r.efficiencies) {
          if (e.second == 1.0) continue;
          bi[(size_t)q * 32 + l] = (unsigned short)e.first;
          bc[(size_t)q * 32 + l] = (e.second - 1.0) / m.species[e.first].W;
          ++q;
        }
      }
      ei.insert(ei.end(), bi.begin(), bi.end());
      ec.insert(ec.end(), bc.begin(), bc.end());
    }
    int nfo = 0;
    std::vector<double> f;
    if (c.kind == WK_LIND || c.kind == WK_TROE3 || c.kind == WK_TROE4 || c.kind == WK_SRI) {
      nfo = c.kind == WK_LIND ? 3 : c.kind == WK_TROE3 ? 7 : 8;
      f.assign((size_t)32 * nfo, 0.0);
      for (int l = 0; l < c.count; ++l) {
        const Reaction& r = m.reactions[P.order[c.base + l]];
        double v[8] = {(double)(logl((long double)r.A0) - logl((long double)r.A)), r.b0 - r.b, -(r.theta0 - r.theta),
                       0, 0, 0, 0, 0};
        if (c.kind == WK_TROE3 || c.kind == WK_TROE4) {
          v[3] = 1.0 - r.troe[0]; v[4] = -1.0 / r.troe[1]; v[5] = r.troe[0]; v[6] = -1.0 / r.troe[2];
          if (c.kind == WK_TROE4) v[7] = -r.troe[3];
        } else if (c.kind == WK_SRI) {
          v[3] = r.sri[0]; v[4] = -r.sri[1]; v[5] = -1.0 / r.sri[2];
          v[6] = r.n_sri >= 5 ? (double)logl((long double)r.sri[3]) : 0.0;
          v[7] = r.n_sri >= 5 ? r.sri[4] : 0.0;
        }
        for (int q = 0; q < nfo; ++q) f[(size_t)q * 32 + l] = v[q];
      }
      // unused lanes of a partial chunk: finite constants (their results are not stored)
      for (int l = c.count; l < 32; ++l)
        for (int q = 0; q < nfo; ++q) f[(size_t)q * 32 + l] = f[(size_t)q * 32];
    } else if (c.kind == WK_PLOG) {
      // per node q: lnA'_q, b_q, -theta_q, ln p_q (nodes beyond a reaction's own: ln p = +huge);
      // then per segment q: 1/(ln p_{q+1} - ln p_q)
      const int Q = c.nodes;
      nfo = 4 * Q + (Q - 1);
      f.assign((size_t)32 * nfo, 0.0);
      for (int l = 0; l < 32; ++l) {
        const Reaction& r = m.reactions[P.order[c.base + std::min(l, c.count - 1)]];
        long double lnWs = 0;
        for (auto& p : r.reactants) lnWs += p.second * logl((long double)m.species[p.first].W);
        const int n = (int)r.plog.size();
        for (int q = 0; q < Q; ++q) {
          const int qq = std::min(q, n - 1);
          f[(size_t)(4 * q + 0) * 32 + l] = (double)(logl((long double)r.plog[qq].A) - lnWs);
          f[(size_t)(4 * q + 1) * 32 + l] = r.plog[qq].b;
          f[(size_t)(4 * q + 2) * 32 + l] = -r.plog[qq].theta;
          f[(size_t)(4 * q + 3) * 32 + l] = q < n ? (double)logl((long double)r.plog[q].p) : 1e300;
        }
        for (int q = 0; q + 1 < Q; ++q)
          f[(size_t)(4 * Q + q) * 32 + l] =
              q + 1 < n ? (double)(1.0L / (logl((long double)r.plog[q + 1].p) - logl((long double)r.plog[q].p))) : 0.0;
      }
    }
    fo.insert(fo.end(), f.begin(), f.end());
  }
  {
    o << "__device__ const unsigned short w_ei[" << std::max<size_t>(ei.size(), 1) << "] = {";
    if (ei.empty()) o << "0";
    for (size_t i = 0; i < ei.size(); ++i) o << (i ? "," : "") << ei[i];
    o << "};\n";
  }
  emit_array(o, "double", "w_ec", ec, true);
  emit_array(o, "double", "w_fo", fo, true);
  emit_array(o, "unsigned", "w_gent", P.gent, false);
  emit_array(o, "int", "w_segf", P.seg_first, false);
  emit_array(o, "int", "w_segc", P.seg_count, false);
  o << "__constant__ double pyro_tab_exp[512] = {";
  for (int j = 0; j < 512; ++j) o << (j ? "," : "") << lit((double)exp2l((j + 0.5L) / 512.0L));
  o << "};\n__constant__ double pyro_tab_log[256] = {";
  for (int j = 0; j < 128; ++j) {
    long double c = 1.0L + (j + 0.5L) / 128.0L;
    o << (j ? "," : "") << lit((double)(1.0L / c)) << "," << lit((double)logl(c));
  }
  o << "};\n";
  o << R"(
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int q = 16; q > 0; q >>= 1) v += __shfl_xor_sync(0xffffffffu, v, q);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int q = 16; q > 0; q >>= 1) v += __shfl_xor_sync(0xffffffffu, v, q);
  return v;
}

// Newton inversion of e(T) = sum_k Y_k e_k(T) for the warp's state (Sec. A.3.1,
// Eq. delta_temp): the mixture polynomial's coefficients are warp sums over the
// lanes' species; every lane then iterates identically -- FP32 to |dT| <= 1e-5 T,
// then FP64 with the FP32 c_v as slope to |dT| <= tol T and one more step (the
// scheme of the thread-per-state kernels).  Returns T; *iters = steps or -1.
__device__ double wtsolve(const double* sY, double e, double T0, int max_iter, float tolf, int* iters, int lane) {
  const double eR = e * )" << lit((double)(1.0L / R_GAS)) << R"(;
  float bf[2][6];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int q = 0; q < 6; ++q) bf[r][q] = 0.f;
  for (int k = lane; k < NSP; k += 32) {
    const float y = pdm::to_float_trunc(sY[k]);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int q = 0; q < 6; ++q) bf[r][q] = fmaf(y, __ldg(w_dcf + (r * 6 + q) * NSP + k), bf[r][q]);
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int q = 0; q < 6; ++q) bf[r][q] = warp_sumf(bf[r][q]);
  float Tf = pdm::to_float_trunc(T0);
  const float eRf = pdm::to_float_trunc(eR);
  int it32 = 0;
  for (; it32 < 40;) {
    ++it32;
    const int h = Tf >= (float)TMID;
    const float* c = bf[h];
    const float ef = fmaf(Tf, fmaf(Tf, fmaf(Tf, fmaf(Tf, fmaf(Tf, c[5], c[4]), c[3]), c[2]), c[1]), c[0]);
    const float cvf = fmaf(Tf, fmaf(Tf, fmaf(Tf, fmaf(Tf, 5.f * c[5], 4.f * c[4]), 3.f * c[3]), 2.f * c[2]), c[1]);
    const float Tn = fminf(fmaxf(Tf + (eRf - ef) * __frcp_rn(cvf), 100.f), 5000.f);
    const bool conv = fabsf(Tn - Tf) <= 1e-5f * Tn;
    Tf = Tn;
    if (conv) break;
  }
  double T = pdm::to_double(Tf);
  int hi = pdm::to_float_trunc(T) >= (float)TMID;
  double B[6];
  auto collapse = [&](int r) {
    double pp[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int k = lane; k < NSP; k += 32) {
      const double y = sY[k];
#pragma unroll
      for (int q = 0; q < 6; ++q) pp[q] = fma(y, __ldg(w_dc + (r * 6 + q) * NSP + k), pp[q]);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) B[q] = warp_sum(pp[q]);
  };
  collapse(hi);
  int it64 = 0;
  bool flag = false, ok = false;
  for (int it = 0; it < max_iter + 1; ++it) {
    ++it64;
    const float Tcur = pdm::to_float_trunc(T);
    const int h2 = Tcur >= (float)TMID;
    if (h2 != hi) { hi = h2; collapse(hi); }
    const double e64 = fma(T, fma(T, fma(T, fma(T, fma(T, B[5], B[4]), B[3]), B[2]), B[1]), B[0]);
    const float* c = bf[hi];
    const float cvf = fmaf(Tcur, fmaf(Tcur, fmaf(Tcur, fmaf(Tcur, 5.f * c[5], 4.f * c[4]), 3.f * c[3]), 2.f * c[2]), c[1]);
    const double dT = (e64 - eR) * pdm::to_double(-__frcp_rn(cvf));
    double Tn = T + dT;
    const float Tnf = pdm::to_float_trunc(Tn);
    const bool clamped = !(Tnf >= 100.f && Tnf <= 5000.f);
    Tn = clamped ? (Tnf < 100.f ? 100.0 : 5000.0) : Tn;
    const bool conv = !clamped && fabsf(pdm::to_float_trunc(dT)) <= tolf * pdm::to_float_trunc(Tn);
    T = Tn;
    if (flag) { ok = true; break; }
    if (conv) flag = true;
    else if (it >= max_iter - 1) break;
  }
  *iters = ok ? it32 + it64 : -1;
  return T;
}
)";
  W.prelude = o.str();
  // chunk code: one block per chunk of 32 reactions, lane l on slot base + l
  std::ostringstream rc;
  Src cnt;   // tally only (the algorithmic counts are the thread-per-state kernel's)
  for (auto& c : P.chunks) {
    rc << "    { // reactions " << c.base << ".." << c.base + c.count - 1 << " (class " << c.kind << ", " << c.nf
       << "x" << c.nr << (c.rev ? "" : " irreversible") << ")\n";
    rc << "      const int s = " << c.base << " + lane;\n";
    if (c.count < 32) rc << "      if (lane < " << c.count << ") {\n";
    rc << "      const unsigned fr = __ldg(w_fr + s);\n";
    for (int q = 0; q < c.nf; ++q) rc << "      const int i" << q << " = (fr >> " << 10 * q << ") & 1023;\n";
    if (c.rev) {
      rc << "      const unsigned fq = __ldg(w_fp + s);\n";
      for (int q = 0; q < c.nr; ++q) rc << "      const int o" << q << " = (fq >> " << 10 * q << ") & 1023;\n";
    }
    // ---- exponent (the shared ln k~ form)
    if (c.kind == WK_PLOG) {
      const int Q = c.nodes;
      auto F = [&](int field) { return "__ldg(w_fo + " + std::to_string(c.foff) + " + " + std::to_string(field * 32) + " + lane)"; };
      rc << "      int qa = 0;\n";
      for (int q = 1; q + 1 < Q; ++q) rc << "      if (lnp >= " << F(4 * q + 3) << ") qa = " << q << ";\n";
      rc << "      const double* nd = w_fo + " << c.foff << " + lane;\n"
            "      const double pla = __ldg(nd + (4 * qa) * 32), pba = __ldg(nd + (4 * qa + 1) * 32), "
            "pta = __ldg(nd + (4 * qa + 2) * 32), plp = __ldg(nd + (4 * qa + 3) * 32);\n"
            "      const double plb = __ldg(nd + (4 * qa + 4) * 32), pbb = __ldg(nd + (4 * qa + 5) * 32), "
            "ptb = __ldg(nd + (4 * qa + 6) * 32);\n"
            "      const double pinv = __ldg(nd + (" << 4 * Q << " + qa) * 32);\n"
            "      const double pxa = fma(pta, invT, fma(pba, lnT, pla));\n"
            "      const double pxb = fma(ptb, invT, fma(pbb, lnT, plb));\n"
            "      const double pf = fmin(fmax((lnp - plp) * pinv, 0.0), 1.0);\n"
            "      double x = fma(pf, pxb - pxa, pxa);\n";
      cnt.fma(5); cnt.add(4 + std::max(0, Q - 2)); cnt.mul();   // as the thread kernel's PLOG count
    } else {
      rc << "      double x = fma(__ldg(w_b + s), lnT, __ldg(w_lnA + s));\n"
            "      x = fma(__ldg(w_mth + s), invT, x);\n";
      cnt.fma(2);
    }
    for (int q = 0; q < c.nf; ++q) rc << "      x -= sL[i" << q << "];\n";
    cnt.add(c.nf);
    rc << "      double kt = PEXP(x, s_exp);\n";
    cnt.exp_();
    if (c.kind != WK_PLAIN && c.kind != WK_PLOG) {
      rc << "      double mS = ysum;\n";
      for (int q = 0; q < c.neff; ++q)
        rc << "      mS = fma(sY[__ldg(w_ei + " << c.eoff + q * 32 << " + lane)], __ldg(w_ec + " << c.eoff + q * 32
           << " + lane), mS);\n";
      rc << "      const double M = rho * mS;\n";
      cnt.fma(c.neff); cnt.mul();
    }
    auto F = [&](int field) { return "__ldg(w_fo + " + std::to_string(c.foff + field * 32) + " + lane)"; };
    if (c.kind == WK_TB) {
      rc << "      kt *= M;\n";
      cnt.mul();
    } else if (c.kind == WK_LIND || c.kind == WK_TROE3 || c.kind == WK_TROE4 || c.kind == WK_SRI) {
      rc << "      const double lnPr = fma(" << F(1) << ", lnT, " << F(0) << ") + fma(" << F(2)
         << ", invT, pdm::log(M, s_log));\n"
            "      const double fpr = pdm::rcp(1.0 + PEXP(-lnPr, s_exp));\n";
      cnt.fma(2); cnt.add(2); cnt.log_(); cnt.exp_(); cnt.rcp_();
      if (c.kind == WK_TROE3 || c.kind == WK_TROE4) {
        rc << "      double fc = fma(" << F(3) << ", PEXP(T * " << F(4) << ", s_exp), " << F(5) << " * PEXP(T * "
           << F(6) << ", s_exp));\n";
        cnt.fma(); cnt.mul(3); cnt.exp_(); cnt.exp_();
        if (c.kind == WK_TROE4) { rc << "      fc += PEXP(" << F(7) << " * invT, s_exp);\n"; cnt.mul(); cnt.exp_(); cnt.add(); }
        const double inv_ln10 = (double)(1.0L / logl(10.0L));
        rc << "      const double lfc = pdm::log(fc, s_log) * " << lit(inv_ln10) << ";\n"
              "      const double cc = fma(-0.67, lfc, -0.4), nn = fma(-1.27, lfc, 0.75);\n"
              "      const double xx = fma(lnPr, " << lit(inv_ln10) << ", cc), den = fma(-0.14, xx, nn);\n"
              "      const double den2 = den * den;\n"
              "      const double lf = lfc * den2 * pdm::rcp(fma(xx, xx, den2));\n"
              "      kt *= fpr * PEXP(lf * " << lit((double)logl(10.0L)) << ", s_exp);\n";
        cnt.log_(); cnt.mul(); cnt.fma(4); cnt.mul(3); cnt.fma(); cnt.rcp_(); cnt.mul(); cnt.exp_(); cnt.mul(2);
      } else if (c.kind == WK_SRI) {
        const double inv_ln10 = (double)(1.0L / logl(10.0L));
        rc << "      const double su = lnPr * " << lit(inv_ln10) << ";\n"
              "      const double sX = pdm::rcp(fma(su, su, 1.0));\n"
              "      const double sS = fma(" << F(3) << ", PEXP(" << F(4) << " * invT, s_exp), PEXP(T * " << F(5)
           << ", s_exp));\n"
              "      kt *= fpr * PEXP(fma(sX, pdm::log(sS, s_log), fma(" << F(7) << ", lnT, " << F(6)
           << ")), s_exp);\n";
        cnt.mul(); cnt.fma(); cnt.rcp_(); cnt.mul(2); cnt.fma(); cnt.exp_(); cnt.exp_(); cnt.log_(); cnt.fma(2);
        cnt.exp_(); cnt.mul(2);
      } else {
        rc << "      kt *= fpr;\n";
        cnt.mul();
      }
    }
    rc << "      double Pf = sA[i0]";
    for (int q = 1; q < c.nf; ++q) rc << " * sA[i" << q << "]";
    rc << ";\n";
    cnt.mul(c.nf - 1);
    if (c.rev) {
      rc << "      double Pr = sA[o0]";
      for (int q = 1; q < c.nr; ++q) rc << " * sA[o" << q << "]";
      rc << ";\n      sR[s] = kt * (Pf - Pr);\n";
      cnt.mul(c.nr - 1); cnt.add(); cnt.mul();
    } else {
      rc << "      sR[s] = kt * Pf;\n";
      cnt.mul();
    }
    if (c.count < 32) rc << "      }\n";
    rc << "    }\n";
    // algorithmic count: the chunk's ops for each of its reactions (not the idle lanes)
  }
  W.reaction_code = rc.str();
  return W;
}

// Shared-memory words per warp: Y (N+1), L then the partial sums (max(N+1, NSEG)),
// a (N+1), one value per reaction.
int warp_words(const WPlan& P) { return (P.N + 1) + std::max(P.N + 1, P.nseg) + (P.N + 1) + P.M; }

// Warps per block: the most resident warps per SM that 227 KB of shared memory
// allows (registers are checked at load); ties go to the smaller block.
int pick_warps(int words) {
  int best = 4, best_w = 0;
  for (int w = 4; w <= 16; ++w) {
    const long bytes = 8L * (776 + (long)w * words);
    if (bytes > 227L * 1024) break;
    // 228 KB of shared memory per SM, 1 KB of it reserved per resident block
    const int blocks = (int)std::min<long>(std::min(32, 64 / w), (228L * 1024) / (bytes + 1024));
    if (blocks * w > best_w) { best_w = blocks * w; best = w; }
  }
  return best;
}

}  // namespace

WarpEmit emit_warp_units(const Mechanism& m, const EmitOptions& opt) {
  WarpEmit out;
  WarpCommon W = emit_warp_common(m, opt);
  const WPlan& P = W.P;
  const int N = P.N;
  const int words = warp_words(P);
  const int wpb = pick_warps(words);
  out.warps_per_block = wpb;
  out.smem_bytes = 8 * (776 + wpb * words);
  out.stats["warp_chunks"] = (double)P.chunks.size();
  out.stats["warp_gather_steps"] = P.steps;
  out.stats["warp_segments"] = P.nseg;
  out.stats["warp_warps_per_block"] = wpb;
  out.stats["warp_smem_bytes"] = out.smem_bytes;
  std::ostringstream k;
  k << W.prelude;
  k << "#define WPB " << wpb << "\n#define WWORDS " << words << "\n#define LSTRIDE " << std::max(N + 1, P.nseg) << "\n";
  const bool plog = has_plog(m);
  k << R"(
// Net production rates, one warp per state (see the emitter for the work split).
// Same arguments as pyro_omega; g_store is unused.
extern "C" __global__ void __launch_bounds__(WPB * 32) pyro_omega_warp(i64 n, const double* __restrict__ g_rho,
    const double* __restrict__ g_Tin, int energy_mode, const double* __restrict__ g_Y,
    double* __restrict__ g_Tout, double* __restrict__ g_omega, double T_guess, int max_iter, double tol,
    unsigned long long* __restrict__ g_fail, double* __restrict__ g_store) {
  extern __shared__ double smem[];
  double* s_exp = smem;
  double* s_log = s_exp + 512;
  double* s_nu = s_log + 256;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* sY = s_nu + 8 + warp * WWORDS;
  double* sL = sY + (NSP + 1);
  double* sP = sL;                      // partial sums of the production rates (after the reactions)
  double* sA = sL + LSTRIDE;
  double* sR = sA + (NSP + 1);
  for (int i = threadIdx.x; i < 512; i += blockDim.x) s_exp[i] = pyro_tab_exp[i];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) s_log[i] = pyro_tab_log[i];
  if (threadIdx.x < 8) s_nu[threadIdx.x] = threadIdx.x == 0 ? 0.0 : (double)((int)threadIdx.x - 4);
  __syncthreads();
  (void)g_store;
  const float tolf = (float)tol;
  for (i64 base = (i64)blockIdx.x * WPB; base < n; base += (i64)gridDim.x * WPB) {
    const i64 p = base + warp;
    if (p >= n) break;                  // warp-uniform; no block barrier below
    const double rho = g_rho[p];
    double ys = 0.0;
    for (int k = lane; k < NSP; k += 32) {
      const double y = g_Y[(i64)k * n + p];
      sY[k] = y;
      ys = fma(y, __ldg(w_invW + k), ys);
    }
    if (lane == 0) sY[NSP] = 0.0;
    const double ysum = warp_sum(ys);
    __syncwarp();
    double T;
    if (energy_mode) {
      int it;
      T = wtsolve(sY, g_Tin[p], T_guess, max_iter, tolf, &it, lane);
      if (lane == 0) {
        if (it < 0) atomicAdd(g_fail, 1ull);
        if (g_Tout) g_Tout[p] = T;
      }
    } else {
      T = g_Tin[p];
    }
    const double lnT = pdm::log(T, s_log), invT = pdm::rcp(T);
    const int hi = pdm::to_float_trunc(T) >= (float)TMID;
    const double* Lc = w_Lc + hi * 7 * (NSP + 1);
    for (int k = lane; k < NSP; k += 32) {
      double q = fma(T, __ldg(Lc + 6 * (NSP + 1) + k), __ldg(Lc + 5 * (NSP + 1) + k));
      q = fma(T, q, __ldg(Lc + 4 * (NSP + 1) + k));
      q = fma(T, q, __ldg(Lc + 3 * (NSP + 1) + k));
      q = fma(T, q, __ldg(Lc + 2 * (NSP + 1) + k));
      q = fma(__ldg(Lc + k), lnT, q);
      q = fma(__ldg(Lc + (NSP + 1) + k), invT, q);
      sL[k] = q;
      sA[k] = PEXP(q, s_exp) * (rho * sY[k]);
    }
    if (lane == 0) { sL[NSP] = 0.0; sA[NSP] = 1.0; }
)";
  if (plog)
    k << "    const double lnp = lnT + pdm::log(rho * ysum, s_log) + " << lit((double)logl(R_GAS)) << ";\n";
  k << "    __syncwarp();\n";
  k << W.reaction_code;
  k << R"(    __syncwarp();
    double acc = 0.0;
#pragma unroll 4
    for (int st = 0; st < GSTEPS; ++st) {
      const unsigned e = __ldg(w_gent + st * 32 + lane);
      acc = fma(s_nu[(e >> 16) & 7u], sR[e & 0xffffu], acc);
      if (e & (1u << 19)) { sP[e >> 20] = acc; acc = 0.0; }
    }
    __syncwarp();
    for (int k = lane; k < NSP; k += 32) {
      const int f = __ldg(w_segf + k), c = __ldg(w_segc + k);
      double w = c > 0 ? sP[f] : 0.0;
      for (int q = 1; q < c; ++q) w += sP[f + q];
      g_omega[(i64)k * n + p] = w;
    }
    __syncwarp();
  }
}
)";
  out.sources["wfwd"] = k.str();
  return out;
}

}  // namespace pyro
