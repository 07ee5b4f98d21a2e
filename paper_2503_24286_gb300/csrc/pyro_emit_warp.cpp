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
//
// The dense Jacobians (d(Tdot, omega)/d(T, Y) at fixed rho and dS/dY at fixed
// (rho, e)) run one block of 8 warps per state with the same reaction chunks
// spread over the warps, every per-reaction partial kept in shared memory, the
// rows assembled by block-wide balanced gathers and written once; blocks form
// clusters of 4 on consecutive states so that the write pass fills whole
// 32-byte output sectors from the 4 blocks' shared memory.
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
  int goff = 0;             // Jacobian kernels: first slot of the chunk's species partials
  int nf = 1, nr = 1;       // largest reactant / product factor counts
  bool rev = true;          // any reversible reaction in the chunk
  int neff = 0;             // largest number of efficiency terms (eps != 1)
  int nodes = 0;            // PLOG: largest node count
  int nrb = 0;              // largest number of species with nu != 0 (adjoint gather of the VJP)
  int eoff = 0, foff = 0, roff = 0;   // offsets into the efficiency / falloff / nu-list tables
};

struct WPlan {
  int N = 0, M = 0;
  std::vector<int> order;   // slot -> reaction
  std::vector<int> slot;    // reaction -> slot
  std::vector<WChunk> chunks;
  int nplain = 0;           // plain reactions occupy slots [0, nplain)
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
  P.nplain = 0;
  for (int j = 0; j < M; ++j) if (wkind(m.reactions[j]) == WK_PLAIN) ++P.nplain;
  int eoff = 0, foff = 0, roff = 0;
  for (int s = 0; s < M;) {
    const int kind = wkind(m.reactions[P.order[s]]);
    const bool rev = m.reactions[P.order[s]].reversible;
    // a chunk holds one class and one direction: the reverse product of an
    // irreversible reaction must be absent, not the unit slot's 1
    int e = s;
    while (e < M && e - s < 32 && wkind(m.reactions[P.order[e]]) == kind && m.reactions[P.order[e]].reversible == rev) ++e;
    WChunk c;
    c.kind = kind; c.base = s; c.count = e - s; c.rev = false; c.nf = 1; c.nr = 1;
    for (int q = s; q < e; ++q) {
      const Reaction& r = m.reactions[P.order[q]];
      c.nf = std::max(c.nf, n_factors(r.reactants));
      if (r.reversible) { c.rev = true; c.nr = std::max(c.nr, n_factors(r.products)); }
      c.neff = std::max(c.neff, n_eff(r));
      if (r.kind == RX_PLOG) c.nodes = std::max(c.nodes, (int)r.plog.size());
      int nnu = 0;
      for (auto& t : net_nu(r)) if (t.second) ++nnu;
      c.nrb = std::max(c.nrb, nnu);
    }
    c.eoff = eoff;
    if (kind != WK_PLAIN && kind != WK_PLOG) eoff += 32 * c.neff;
    c.foff = foff;
    const int nfo = kind == WK_LIND ? 3 : kind == WK_TROE3 ? 7 : kind == WK_TROE4 ? 8 : kind == WK_SRI ? 8
                  : kind == WK_PLOG ? 4 * c.nodes + (c.nodes - 1) : 0;
    foff += 32 * nfo;
    c.roff = roff;
    roff += 32 * c.nrb;
    P.chunks.push_back(c);
    s = e;
  }
  return P;
}

// Balanced gathers sum_{(k, e)} value(e) into per-species sums: every loop's
// entries (sorted by species) are cut into 32 runs of equal length, lane l
// walks run l and flushes a partial sum at each species boundary; the species
// pass then adds the partial sums (segments) of each species.
struct GItem {
  int k;          // species
  unsigned x, y;  // payload (y: bits 0..19)
  double c;       // payload coefficient (efficiency loops)
};
struct GLoop {
  int steps = 1;
  std::vector<unsigned> ent;   // [steps][32][2]
  std::vector<double> coef;    // [steps][32] (efficiency loops)
};
struct Gather {
  int lanes = 32;                      // threads that share the gather (a warp or a block)
  std::vector<GLoop> loops;
  int nseg = 0;
  std::vector<int> seg_ptr, seg_idx;   // per species: its segments
  double entries = 0;
};

Gather build_gather(int N, std::vector<std::vector<GItem>> items, int lanes = 32) {
  Gather G;
  G.lanes = lanes;
  std::vector<std::vector<int>> segs(N);
  for (auto& its : items) {
    std::stable_sort(its.begin(), its.end(), [](const GItem& a, const GItem& b) { return a.k < b.k; });
    GLoop L;
    const int nnz = (int)its.size();
    G.entries += nnz;
    L.steps = std::max(1, (nnz + lanes - 1) / lanes);
    L.ent.assign((size_t)L.steps * lanes * 2, 0u);
    L.coef.assign((size_t)L.steps * lanes, 0.0);
    for (int l = 0; l < lanes; ++l) {
      const int a = l * L.steps, b = std::min(nnz, (l + 1) * L.steps);
      for (int q = a; q < b; ++q) {
        const GItem& it = its[q];
        unsigned y = it.y;
        if (q + 1 == b || its[q + 1].k != it.k) {
          y |= (1u << 20) | ((unsigned)G.nseg << 21);
          segs[it.k].push_back(G.nseg++);
        }
        const size_t e = (size_t)(q - a) * lanes + l;
        L.ent[2 * e] = it.x;
        L.ent[2 * e + 1] = y;
        L.coef[e] = it.c;
      }
    }
    G.loops.push_back(L);
  }
  G.seg_ptr.push_back(0);
  for (int k = 0; k < N; ++k) {
    for (int v : segs[k]) G.seg_idx.push_back(v);
    G.seg_ptr.push_back((int)G.seg_idx.size());
  }
  return G;
}

// Gather into the nonzero entries of a block of Jacobian rows: keys 0..nkeys-1
// (every key has at least one item), items sorted by key and cut into `lanes`
// runs of equal length.  The keys of one run are consecutive, so lane l needs
// only its first key and advances one key per flush.  A key cut by a run
// boundary is written by the lane it starts in; the lanes that continue it
// write their partial sums to a carry slot (one per lane), and one fix-up
// record per cut key adds those in lane order.  Fixed order: deterministic.
struct NzItem {
  int key;
  unsigned slot;
  int nu;
};
struct NzGather {
  int steps = 1, nkeys = 0;
  std::vector<unsigned> ent;     // [steps][lanes]: slot | (nu + 4) << 16 | flush << 19
  std::vector<unsigned> lane0;   // [lanes]: first key | continues-a-key << 31
  std::vector<unsigned> fix;     // per cut key: key | first carrying lane << 16 | last << 24
};

NzGather build_nz_gather(std::vector<NzItem> its, int nkeys, int lanes, unsigned zero_slot) {
  NzGather G;
  G.nkeys = nkeys;
  std::stable_sort(its.begin(), its.end(), [](const NzItem& a, const NzItem& b) { return a.key < b.key; });
  const int n = (int)its.size();
  G.steps = std::max(1, (n + lanes - 1) / lanes);
  G.ent.assign((size_t)G.steps * lanes, zero_slot);   // padding: the zero slot times nu index 0
  G.lane0.assign(lanes, 0u);
  for (int l = 0; l < lanes; ++l) {
    const int a = l * G.steps, b = std::min(n, (l + 1) * G.steps);
    if (a >= b) continue;
    G.lane0[l] = (unsigned)its[a].key | ((a > 0 && its[a - 1].key == its[a].key) ? (1u << 31) : 0u);
    for (int q = a; q < b; ++q) {
      const bool flush = q + 1 == b || its[q + 1].key != its[q].key;
      G.ent[(size_t)(q - a) * lanes + l] = its[q].slot | ((unsigned)(its[q].nu + 4) << 16) | (flush ? (1u << 19) : 0u);
    }
  }
  for (int q = 0; q < n;) {
    int e = q;
    while (e < n && its[e].key == its[q].key) ++e;
    const int la = q / G.steps, lb = (e - 1) / G.steps;
    if (lb > la) G.fix.push_back((unsigned)its[q].key | ((unsigned)(la + 1) << 16) | ((unsigned)lb << 24));
    q = e;
  }
  return G;
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

enum WMode { W_FWD = 0, W_JVP = 1, W_VJP = 2, W_JAC = 3, W_JAD = 4 };

// Slots of a chunk's species partials in the Jacobian kernels: one per factor
// occurrence (reactants, then products of reversible chunks), then one per
// third-body efficiency term.
int chunk_occ(const WChunk& c) { return c.nf + (c.rev ? c.nr : 0); }
int chunk_gslots(const WChunk& c) {
  return 32 * (chunk_occ(c) + ((c.kind != WK_PLAIN && c.kind != WK_PLOG) ? c.neff : 0));
}

std::string gname(const char* base, int g) { return std::string(base) + std::to_string(g); }

// The gather's tables: entries, coefficients (if any), per-species segments.
void emit_gather_tables(std::ostringstream& o, const Gather& G, int g, bool coef) {
  for (size_t l = 0; l < G.loops.size(); ++l) {
    const auto& L = G.loops[l];
    o << "__device__ const uint2 " << gname("w_ge", g) << "_" << l << "[" << L.steps * G.lanes << "] = {";
    for (size_t e = 0; e < L.ent.size() / 2; ++e)
      o << (e ? "," : "") << "{" << L.ent[2 * e] << "u," << L.ent[2 * e + 1] << "u}";
    o << "};\n";
    if (coef) emit_array(o, "double", gname("w_gc", g) + "_" + std::to_string(l), L.coef, true);
  }
  emit_array(o, "int", gname("w_sp", g), G.seg_ptr, false);
  emit_array(o, "int", gname("w_si", g), G.seg_idx, false);
}

// One gather loop: lane l accumulates its run; `term` is the FP64 update of acc
// for entry e (uint2) and coefficient c.  `lane` names the thread's index among
// the gather's lanes.
// With sP2 given, a second accumulator acc2 flushes into sP2 alongside.
void emit_gather_loop(std::ostringstream& k, const Gather& G, int g, size_t l, const std::string& term, bool coef,
                      const std::string& sP, const std::string& lane = "lane", const std::string& sP2 = "") {
  const std::string at = " + st * " + std::to_string(G.lanes) + " + " + lane + ");\n";
  k << "    {\n      double acc = 0.0" << (sP2.empty() ? "" : ", acc2 = 0.0") << ";\n#pragma unroll 4\n"
    << "      for (int st = 0; st < " << G.loops[l].steps
    << "; ++st) {\n        const uint2 e = __ldg(" << gname("w_ge", g) << "_" << l << at;
  if (coef) k << "        const double c = __ldg(" << gname("w_gc", g) << "_" << l << at;
  k << "        " << term << "\n        if (e.y & (1u << 20)) { " << sP << "[e.y >> 21] = acc; acc = 0.0;";
  if (!sP2.empty()) k << " " << sP2 << "[e.y >> 21] = acc2; acc2 = 0.0;";
  k << " }\n      }\n    }\n";
}

// Per-species total of gather g (segments in sP): into the double variable `var`.
std::string gather_total(int g, const std::string& sP, const std::string& var) {
  return "      double " + var + " = 0.0;\n      for (int q = __ldg(" + gname("w_sp", g) + " + k); q < __ldg(" +
         gname("w_sp", g) + " + k + 1); ++q) " + var + " += " + sP + "[__ldg(" + gname("w_si", g) + " + q)];\n";
}

// Shared-memory words of one warp for a kernel mode.
struct WLayout {
  std::vector<std::pair<std::string, int>> arrays;   // name, words
  int words() const {
    int w = 0;
    for (auto& a : arrays) w += a.second;
    return w;
  }
};

// Warps per block: the most resident warps per SM that the shared memory allows
// (228 KB per SM, 1 KB reserved per block, 227 KB per block, at most 64 warps);
// registers are checked at load.  Ties go to the smaller block.
int pick_warps(int words) {
  int best = 4, best_w = 0;
  for (int w = 4; w <= 16; ++w) {
    const long bytes = 8L * (776 + (long)w * words);
    if (bytes > 227L * 1024) break;
    const int blocks = (int)std::min<long>(std::min(32, 64 / w), (228L * 1024) / (bytes + 1024));
    if (blocks * w > best_w) { best_w = blocks * w; best = w; }
  }
  return best;
}

// The reaction phase of one chunk (lane l: slot base + l) in the given mode.
//   FWD: sR[s] = R;  JVP: sR[s] = dR;  VJP: sDb[s] = Rb kk, sMb[s - NPLAIN] = Rb kM D and the
//   lane's partial sums of T_bar, the total [M] adjoint and its rho term.
void emit_chunk(std::ostringstream& rc, const WChunk& c, int mode) {
  const double inv_ln10 = (double)(1.0L / logl(10.0L));
  const std::string ln10 = lit((double)logl(10.0L));
  rc << "    { // reactions " << c.base << ".." << c.base + c.count - 1 << " (class " << c.kind << ", " << c.nf << "x"
     << c.nr << (c.rev ? "" : " irreversible") << ")\n";
  rc << "      const int s = " << c.base << " + lane;\n";
  if (c.count < 32) rc << "      if (lane < " << c.count << ") {\n";
  rc << "      const unsigned fr = __ldg(w_fr + s);\n";
  for (int q = 0; q < c.nf; ++q) rc << "      const int i" << q << " = (fr >> " << 10 * q << ") & 1023;\n";
  if (c.rev) {
    rc << "      const unsigned fq = __ldg(w_fp + s);\n";
    for (int q = 0; q < c.nr; ++q) rc << "      const int o" << q << " = (fq >> " << 10 * q << ") & 1023;\n";
  }
  auto F = [&](int field) { return "__ldg(w_fo + " + std::to_string(c.foff + field * 32) + " + lane)"; };
  const bool der = mode != W_FWD;
  // ---- exponent of k~ (and d/dT)
  if (c.kind == WK_PLOG) {
    const int Q = c.nodes;
    rc << "      int qa = 0;\n";
    for (int q = 1; q + 1 < Q; ++q) rc << "      if (lnp >= " << F(4 * q + 3) << ") qa = " << q << ";\n";
    rc << "      const double* nd = w_fo + " << c.foff << " + lane;\n"
          "      const double pla = __ldg(nd + (4 * qa) * 32), pba = __ldg(nd + (4 * qa + 1) * 32), "
          "pma = __ldg(nd + (4 * qa + 2) * 32), plp = __ldg(nd + (4 * qa + 3) * 32);\n"
          "      const double plb = __ldg(nd + (4 * qa + 4) * 32), pbb = __ldg(nd + (4 * qa + 5) * 32), "
          "pmb = __ldg(nd + (4 * qa + 6) * 32);\n"
          "      const double pinv = __ldg(nd + (" << 4 * Q << " + qa) * 32);\n"
          "      const double pxa = fma(pma, invT, fma(pba, lnT, pla));\n"
          "      const double pxb = fma(pmb, invT, fma(pbb, lnT, plb));\n"
          "      const double pfu = (lnp - plp) * pinv;\n"
          "      const double pf = fmin(fmax(pfu, 0.0), 1.0);\n"
          "      double x = fma(pf, pxb - pxa, pxa);\n";
    if (der)
      rc << "      const double pdx = (pfu > 0.0 && pfu < 1.0) ? (pxb - pxa) * pinv : 0.0;\n"
            "      const double pta_ = fma(pba, invT, -pma * invT2), ptb_ = fma(pbb, invT, -pmb * invT2);\n"
            "      double tau = fma(pdx, invT, fma(pf, ptb_ - pta_, pta_));\n";
  } else {
    rc << "      double x = fma(__ldg(w_b + s), lnT, __ldg(w_lnA + s));\n"
          "      x = fma(__ldg(w_mth + s), invT, x);\n";
    if (der) rc << "      double tau = fma(__ldg(w_b + s), invT, -__ldg(w_mth + s) * invT2);\n";
  }
  for (int q = 0; q < c.nf; ++q) rc << "      x -= sL[i" << q << "];\n";
  rc << "      const double kt = PEXP(x, s_exp);\n";
  // ---- [M] and the rate-constant factor
  const bool tb = c.kind != WK_PLAIN && c.kind != WK_PLOG;
  if (tb) {
    rc << "      double mS = ysum;\n";
    for (int q = 0; q < c.neff; ++q)
      rc << "      mS = fma(sY[__ldg(w_ei + " << c.eoff + q * 32 << " + lane)], __ldg(w_ec + " << c.eoff + q * 32
         << " + lane), mS);\n";
    rc << "      const double M = rho * mS;\n";
  } else if (c.kind == WK_PLOG && der) {
    rc << "      const double mS = ysum;\n      const double M = rho * mS;\n";
  }
  if (c.kind == WK_PLAIN) {
    rc << "      const double kk = kt;\n";
  } else if (c.kind == WK_PLOG) {
    rc << "      const double kk = kt;\n";
    if (der) rc << "      const double kM = kt * pdx * pdm::rcp(M);\n";
  } else if (c.kind == WK_TB) {
    rc << "      const double kk = kt * M;\n";
    if (der) rc << "      const double kM = kt;\n";
  } else {
    rc << "      const double lnPr = fma(" << F(1) << ", lnT, " << F(0) << ") + fma(" << F(2)
       << ", invT, pdm::log(M, s_log));\n"
          "      const double qpr = PEXP(-lnPr, s_exp);\n"
          "      const double fpr = pdm::rcp(1.0 + qpr);\n";
    if (der)
      rc << "      const double pT = fma(" << F(1) << ", invT, -" << F(2) << " * invT2);\n"
            "      const double cpr = qpr * fpr;   // 1 - Pr/(1+Pr) without cancellation\n";
    if (c.kind == WK_TROE3 || c.kind == WK_TROE4) {
      rc << "      const double t1 = " << F(3) << " * PEXP(T * " << F(4) << ", s_exp);\n"
            "      const double t2 = " << F(5) << " * PEXP(T * " << F(6) << ", s_exp);\n";
      if (c.kind == WK_TROE4) rc << "      const double t3 = PEXP(" << F(7) << " * invT, s_exp);\n";
      else rc << "      const double t3 = 0.0;\n";
      rc << "      const double fc = t1 + t2 + t3;\n"
            "      const double lfc = pdm::log(fc, s_log) * " << lit(inv_ln10) << ";\n"
            "      const double cc = fma(-0.67, lfc, -0.4), nn = fma(-1.27, lfc, 0.75);\n"
            "      const double xx = fma(lnPr, " << lit(inv_ln10) << ", cc), den = fma(-0.14, xx, nn);\n"
            "      const double den2 = den * den;\n";
      if (!der) {
        rc << "      const double lf = lfc * den2 * pdm::rcp(fma(xx, xx, den2));\n"
              "      const double kk = kt * (fpr * PEXP(lf * " << ln10 << ", s_exp));\n";
      } else {
        rc << "      const double rD = pdm::rcp(fma(xx, xx, den2));\n"
              "      const double f = den2 * rD;\n"
              "      const double Fb = PEXP(lfc * f * " << ln10 << ", s_exp);\n"
              "      const double rD2 = rD * rD;\n"
              "      const double Axx = lfc * (-2.0 * den2 * xx * rD2), Aden = lfc * (2.0 * den * xx * xx * rD2);\n"
              "      const double sPr = cpr + fma(-0.14, Aden, Axx);\n"
              "      const double sfc = fma(-0.67, Axx, fma(-1.1762, Aden, f));\n";
        if (c.kind == WK_TROE4)
          rc << "      const double dfc = fma(t1, " << F(4) << ", fma(t2, " << F(6) << ", -(t3 * " << F(7) << ") * invT2));\n";
        else
          rc << "      const double dfc = fma(t1, " << F(4) << ", t2 * " << F(6) << ");\n";
        rc << "      tau += fma(sPr, pT, sfc * dfc * pdm::rcp(fc));\n"
              "      const double kk = kt * fpr * Fb;\n";
      }
    } else if (c.kind == WK_SRI) {
      rc << "      const double su = lnPr * " << lit(inv_ln10) << ";\n"
            "      const double sX = pdm::rcp(fma(su, su, 1.0));\n"
            "      const double sea = " << F(3) << " * PEXP(" << F(4) << " * invT, s_exp);\n"
            "      const double seb = PEXP(T * " << F(5) << ", s_exp);\n"
            "      const double sS = sea + seb;\n"
            "      const double slS = pdm::log(sS, s_log);\n"
            "      const double Fb = PEXP(fma(sX, slS, fma(" << F(7) << ", lnT, " << F(6) << ")), s_exp);\n";
      if (der)
        rc << "      const double dlnF_dlnPr = slS * (-2.0 * su * sX * sX * " << lit(inv_ln10) << ");\n"
              "      const double dlnF_dT = fma(sX * fma(sea, -" << F(4) << " * invT2, seb * " << F(5)
           << "), pdm::rcp(sS), " << F(7) << " * invT);\n"
              "      const double sPr = cpr + dlnF_dlnPr;\n"
              "      tau += fma(sPr, pT, dlnF_dT);\n";
      rc << "      const double kk = kt * fpr * Fb;\n";
    } else {   // Lindemann
      if (der) rc << "      const double sPr = cpr;\n      tau += sPr * pT;\n";
      rc << "      const double kk = kt * fpr;\n";
    }
    if (der) rc << "      const double kM = kk * sPr * pdm::rcp(M);\n";
  }
  // ---- activity products
  rc << "      const double Pf = sA[i0]";
  for (int q = 1; q < c.nf; ++q) rc << " * sA[i" << q << "]";
  rc << ";\n";
  if (c.rev) {
    rc << "      const double Pr = sA[o0]";
    for (int q = 1; q < c.nr; ++q) rc << " * sA[o" << q << "]";
    rc << ";\n      const double D = Pf - Pr;\n";
  } else {
    rc << "      const double D = Pf;\n";
  }
  auto dprod = [&](const char* v, int nfac, const char* da) {
    std::string e;
    for (int q = 0; q < nfac; ++q) {
      std::string t = std::string(da) + "[" + v + std::to_string(q) + "]";
      for (int r = 0; r < nfac; ++r) if (r != q) t += " * sA[" + std::string(v) + std::to_string(r) + "]";
      e += (q ? " + " : "") + t;
    }
    return e;
  };
  if (mode == W_FWD) {
    rc << "      sR[s] = kk * D;\n";
  } else if (mode == W_JVP) {
    rc << "      double dx = tau * dT;\n";
    for (int q = 0; q < c.nf; ++q) rc << "      dx -= sdL[i" << q << "];\n";
    if (c.kind == WK_PLAIN) {
      rc << "      const double dkk = kk * dx;\n";
    } else {
      rc << "      double dmS = dysum;\n";
      if (tb)
        for (int q = 0; q < c.neff; ++q)
          rc << "      dmS = fma(sdY[__ldg(w_ei + " << c.eoff + q * 32 << " + lane)], __ldg(w_ec + " << c.eoff + q * 32
             << " + lane), dmS);\n";
      rc << "      const double dM = fma(drho, mS, rho * dmS);\n"
            "      const double dkk = fma(kk, dx, kM * dM);\n";
    }
    rc << "      const double dPf = " << dprod("i", c.nf, "sdA") << ";\n";
    if (c.rev) rc << "      const double dPr = " << dprod("o", c.nr, "sdA") << ";\n";
    rc << "      sR[s] = fma(dkk, D, kk * " << (c.rev ? "(dPf - dPr)" : "dPf") << ");\n";
  } else if (mode == W_JAC || mode == W_JAD) {
    // per-reaction partials of the dense Jacobian: dR/dT, the [M] term kM D rho,
    // and dR/dY_i at fixed (rho, T) per factor occurrence (the other factors'
    // product) and per efficiency term ((eps_i - 1)/W_i kM D rho)
    auto others = [&](const char* v, int nfac, int q) {
      std::string t;
      for (int r = 0; r < nfac; ++r) if (r != q) t += " * sA[" + std::string(v) + std::to_string(r) + "]";
      return t;
    };
    rc << "      const double R = kk * D;\n";
    if (c.rev) {
      rc << "      const double dS = sLp[i0]";
      for (int q = 1; q < c.nf; ++q) rc << " + sLp[i" << q << "]";
      for (int q = 0; q < c.nr; ++q) rc << " - sLp[o" << q << "]";
      rc << ";\n      const double Rt = kk * fma(D, tau, Pr * dS);\n";
    } else {
      rc << "      const double Rt = kk * (D * tau);\n";
    }
    rc << "      sRt[s] = Rt;\n";
    if (c.kind != WK_PLAIN) rc << "      const double RMr = kM * D * rho;\n      sRM[s] = RMr;\n";
    else rc << "      sRM[s] = 0.0;\n";
    for (int q = 0; q < c.nf; ++q)
      rc << "      sG[" << c.goff + q * 32 << " + lane] = kk * sEr[i" << q << "]" << others("i", c.nf, q) << ";\n";
    if (c.rev)
      for (int q = 0; q < c.nr; ++q)
        rc << "      sG[" << c.goff + (c.nf + q) * 32 << " + lane] = -kk * sEr[o" << q << "]" << others("o", c.nr, q)
           << ";\n";
    if (tb)
      for (int q = 0; q < c.neff; ++q)
        rc << "      sG[" << c.goff + (chunk_occ(c) + q) * 32 << " + lane] = __ldg(w_ec + " << c.eoff + q * 32
           << " + lane) * RMr;\n";
    if (mode == W_JAC) {
      // the reaction's internal-energy and heat-capacity changes (Tdot row)
      rc << "      double dE = 0.0, dC = 0.0;\n";
      for (int q = 0; q < c.nrb; ++q)
        rc << "      { const unsigned short b = __ldg(w_rb + " << c.roff + q * 32
           << " + lane); const double nu = s_nu[b >> 10]; dE = fma(nu, seh[b & 1023], dE); dC = fma(nu, scm[b & 1023], dC); }\n";
      rc << "      sDE[s] = dE;\n      pew = fma(dE, R, pew); pcw = fma(dC, R, pcw); pejt = fma(dE, Rt, pejt);\n";
      if (c.kind != WK_PLAIN) rc << "      pU = fma(dE, RMr, pU);\n";
    } else {
      rc << "      (void)R;\n";
    }
  } else {
    rc << "      double Rb = 0.0;\n";
    for (int q = 0; q < c.nrb; ++q)
      rc << "      { const unsigned short b = __ldg(w_rb + " << c.roff + q * 32
         << " + lane); Rb = fma(s_nu[b >> 10], sWb[b & 1023], Rb); }\n";
    rc << "      const double xb = Rb * (kk * D);\n      Tbp = fma(xb, tau, Tbp);\n";
    for (int q = 0; q < c.nf; ++q) rc << "      Tbp = fma(-xb, sLp[i" << q << "], Tbp);\n";
    rc << "      sDb[s] = Rb * kk;\n";
    if (c.kind != WK_PLAIN)
      rc << "      const double Mb = Rb * kM * D;\n      sMb[s - NPLAIN] = Mb;\n      Mtp += Mb;\n"
            "      rMp = fma(Mb, mS, rMp);\n";
  }
  if (c.count < 32) rc << "      }\n";
  rc << "    }\n";
}

}  // namespace

bool warp_supported(const Mechanism& m, std::string* why) {
  if (m.n_species() > kWarpMaxSpecies || m.n_reactions() > kWarpMaxReactions) {
    *why = "variant=warp supports up to " + std::to_string(kWarpMaxSpecies) + " species and " +
           std::to_string(kWarpMaxReactions) + " reactions";
    return false;
  }
  if (!common_tmid(m)) {
    *why = "variant=warp needs all species to share one NASA-7 T_mid";
    return false;
  }
  for (int j = 0; j < m.n_reactions(); ++j) {
    const Reaction& r = m.reactions[j];
    if (n_factors(r.reactants) > 3 || n_factors(r.products) > 3) {
      *why = "variant=warp supports at most three factors a side (reaction " + std::to_string(j) + ")";
      return false;
    }
  }
  return true;
}

WarpEmit emit_warp_units(const Mechanism& m, const EmitOptions& opt) {
  WarpEmit out;
  const WPlan P = make_plan(m);
  const int N = P.N, M = P.M, N1 = N + 1;
  std::vector<SpeciesCoef> C;
  for (auto& sp : m.species) C.push_back(species_coef(sp));
  // ---- gathers: production rates (forward, JVP) and the VJP's adjoints
  std::vector<GItem> fw;
  std::vector<GItem> adj1, adj2, effl;
  for (int j = 0; j < M; ++j) {
    const Reaction& r = m.reactions[j];
    const unsigned sl = (unsigned)P.slot[j];
    for (auto& q : net_nu(r))
      if (q.second) fw.push_back({q.first, sl | ((unsigned)(q.second + 4) << 16), 0u, 0.0});
    // d(prod a^nu)/d a_i: one entry per factor occurrence, with the other factors
    for (int side = 0; side < (r.reversible ? 2 : 1); ++side) {
      std::vector<int> f = side_factors(side == 0 ? r.reactants : r.products);
      for (size_t q = 0; q < f.size(); ++q) {
        std::vector<int> oth;
        for (size_t t = 0; t < f.size(); ++t) if (t != q) oth.push_back(f[t]);
        const unsigned x = sl | ((unsigned)side << 16);
        if (oth.size() <= 1) adj1.push_back({f[q], x, (unsigned)(oth.empty() ? N : oth[0]), 0.0});
        else adj2.push_back({f[q], x, (unsigned)oth[0] | ((unsigned)oth[1] << 10), 0.0});
      }
    }
    if (wkind(r) != WK_PLAIN && wkind(r) != WK_PLOG)
      for (auto& e : r.efficiencies)
        if (e.second != 1.0) effl.push_back({e.first, sl - (unsigned)P.nplain, 0u, (e.second - 1.0) / m.species[e.first].W});
  }
  const Gather gF = build_gather(N, {fw});
  const Gather gA = build_gather(N, {adj1, adj2});
  const Gather gC = build_gather(N, {effl});
  // ---- shared tables
  std::ostringstream o;
  o << "// Generated for mechanism '" << m.name << "': " << N << " species, " << M
    << " reactions; warp-per-state kernels.\n";
  o << "#include \"pyro_device_math.cuh\"\ntypedef long long i64;\n";
  o << "#define PEXP(x, t) pdm::" << (opt.warp_exp_ops == 4 ? "exp4" : "exp") << "((x), (t))\n";
  o << "#define NSP " << N << "\n#define NRX " << M << "\n#define NPLAIN " << P.nplain << "\n#define TMID "
    << lit(m.species[0].t_mid) << "\n";
  std::vector<double> Lc(2 * 7 * N1, 0.0), Hc(2 * 6 * N1, 0.0), dc(2 * 6 * N), invW(N1, 0.0);
  std::vector<float> dcf(2 * 6 * N);
  for (int k = 0; k < N; ++k) {
    invW[k] = 1.0 / m.species[k].W;
    for (int r = 0; r < 2; ++r) {
      const double L[7] = {C[k].cl[r], C[k].ci[r], C[k].c0[r], C[k].c1[r], C[k].c2[r], C[k].c3[r], C[k].c4[r]};
      for (int q = 0; q < 7; ++q) Lc[(r * 7 + q) * N1 + k] = L[q];
      for (int q = 0; q < 6; ++q) {
        Hc[(r * 6 + q) * N1 + k] = C[k].h[r][q];
        dc[(r * 6 + q) * N + k] = C[k].d[r][q];
        dcf[(r * 6 + q) * N + k] = (float)C[k].d[r][q];
      }
    }
  }
  emit_array(o, "double", "w_Lc", Lc, true);
  emit_array(o, "double", "w_Hc", Hc, true);
  emit_array(o, "double", "w_dc", dc, true);
  o << "__device__ const float w_dcf[" << dcf.size() << "] = {";
  for (size_t i = 0; i < dcf.size(); ++i) o << (i ? "," : "") << litf(dcf[i]);
  o << "};\n";
  emit_array(o, "double", "w_invW", invW, true);
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
  std::vector<unsigned short> ei, rb;
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
    {
      // net nu list of each reaction: species (10 bits) | (nu + 4) << 10; padding: the unit slot, nu 0
      std::vector<unsigned short> br((size_t)32 * c.nrb, (unsigned short)(N | (4 << 10)));
      for (int l = 0; l < c.count; ++l) {
        int q = 0;
        for (auto& t : net_nu(m.reactions[P.order[c.base + l]]))
          if (t.second) br[(size_t)(q++) * 32 + l] = (unsigned short)(t.first | ((t.second + 4) << 10));
      }
      rb.insert(rb.end(), br.begin(), br.end());
    }
    int nfo = 0;
    std::vector<double> f;
    if (c.kind == WK_LIND || c.kind == WK_TROE3 || c.kind == WK_TROE4 || c.kind == WK_SRI) {
      nfo = c.kind == WK_LIND ? 3 : c.kind == WK_TROE3 ? 7 : 8;
      f.assign((size_t)32 * nfo, 0.0);
      for (int l = 0; l < 32; ++l) {
        const Reaction& r = m.reactions[P.order[c.base + std::min(l, c.count - 1)]];
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
    } else if (c.kind == WK_PLOG) {
      // per node q: lnA'_q, b_q, -theta_q, ln p_q (nodes past a reaction's own: ln p = 1e300);
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
  o << "__device__ const unsigned short w_ei[" << std::max<size_t>(ei.size(), 1) << "] = {";
  if (ei.empty()) o << "0";
  for (size_t i = 0; i < ei.size(); ++i) o << (i ? "," : "") << ei[i];
  o << "};\n";
  o << "__device__ const unsigned short w_rb[" << std::max<size_t>(rb.size(), 1) << "] = {";
  if (rb.empty()) o << "0";
  for (size_t i = 0; i < rb.size(); ++i) o << (i ? "," : "") << rb[i];
  o << "};\n";
  emit_array(o, "double", "w_ec", ec, true);
  emit_array(o, "double", "w_fo", fo, true);
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
// Warp sums of eight values at once (every lane gets all eight): a reduce-scatter
// (halving the set at each of the first three exchanges: 4 + 2 + 1 adds), a
// butterfly on the remaining value (2 adds), then an all-gather by shuffles --
// 9 FP64 adds per lane instead of 8 x 5.
__device__ __forceinline__ void warp_sum8(double (&v)[8], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
  for (int q = 0; q < 4; ++q) {                 // keep v[0..3] (b4 = 0) or v[4..7] (b4 = 1)
    const double mine = b4 ? v[q + 4] : v[q], give = b4 ? v[q] : v[q + 4];
    v[q] = mine + __shfl_xor_sync(0xffffffffu, give, 16);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double mine = b3 ? v[q + 2] : v[q], give = b3 ? v[q] : v[q + 2];
    v[q] = mine + __shfl_xor_sync(0xffffffffu, give, 8);
  }
  {
    const double mine = b2 ? v[1] : v[0], give = b2 ? v[0] : v[1];
    v[0] = mine + __shfl_xor_sync(0xffffffffu, give, 4);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  // lane l now holds the total of value 4 b4 + 2 b3 + b2; gather all eight
  const double t = v[0];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __shfl_sync(0xffffffffu, t, ((q >> 2) & 1) * 16 + ((q >> 1) & 1) * 8 + (q & 1) * 4);
}
// the block's exp/log tables and the stoichiometric coefficients -4..3 (index nu + 4;
// index 0 is the gather's padding and holds 0)
__device__ __forceinline__ void wload_tables(double* s_exp, double* s_log, double* s_nu) {
  for (int i = threadIdx.x; i < 512; i += blockDim.x) s_exp[i] = pyro_tab_exp[i];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) s_log[i] = pyro_tab_log[i];
  if (threadIdx.x < 8) s_nu[threadIdx.x] = threadIdx.x == 0 ? 0.0 : (double)((int)threadIdx.x - 4);
}
)";
  // Newton temperature solve (forward kernel only)
  std::ostringstream nw;
  nw << R"(
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
    double pp[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int k = lane; k < NSP; k += 32) {
      const double y = sY[k];
#pragma unroll
      for (int q = 0; q < 6; ++q) pp[q] = fma(y, __ldg(w_dc + (r * 6 + q) * NSP + k), pp[q]);
    }
    warp_sum8(pp, lane);
#pragma unroll
    for (int q = 0; q < 6; ++q) B[q] = pp[q];
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
  const bool plog = has_plog(m);
  const std::string lnR = lit((double)logl(R_GAS));
  // species thermo of lane k: q = L_k; with H: hr = h_k/RT and Lp = L'_k = (1 - h_k/RT)/T
  auto species_L = [&](bool H) {
    std::string t =
        "      const double* Lc = w_Lc + hi * 7 * (NSP + 1);\n"
        "      double q = fma(T, __ldg(Lc + 6 * (NSP + 1) + k), __ldg(Lc + 5 * (NSP + 1) + k));\n"
        "      q = fma(T, q, __ldg(Lc + 4 * (NSP + 1) + k));\n"
        "      q = fma(T, q, __ldg(Lc + 3 * (NSP + 1) + k));\n"
        "      q = fma(T, q, __ldg(Lc + 2 * (NSP + 1) + k));\n"
        "      q = fma(__ldg(Lc + k), lnT, q);\n"
        "      q = fma(__ldg(Lc + (NSP + 1) + k), invT, q);\n";
    if (H)
      t += "      const double* Hc = w_Hc + hi * 6 * (NSP + 1);\n"
           "      double hr = fma(T, __ldg(Hc + 4 * (NSP + 1) + k), __ldg(Hc + 3 * (NSP + 1) + k));\n"
           "      hr = fma(T, hr, __ldg(Hc + 2 * (NSP + 1) + k));\n"
           "      hr = fma(T, hr, __ldg(Hc + (NSP + 1) + k));\n"
           "      hr = fma(T, hr, __ldg(Hc + k));\n"
           "      hr = fma(__ldg(Hc + 5 * (NSP + 1) + k), invT, hr);\n"
           "      const double Lp = fma(-hr, invT, invT);\n";
    return t;
  };
  auto kernel_head = [&](std::ostringstream& k, const WLayout& L, const char* sig) {
    int words = L.words();
    const int wpb = pick_warps(words);
    k << "\n#undef WPB\n#define WPB " << wpb << "\n" << sig << " {\n"
      << "  extern __shared__ double smem[];\n  double* s_exp = smem;\n  double* s_log = s_exp + 512;\n"
      << "  double* s_nu = s_log + 256;\n  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;\n"
      << "  double* wbase = s_nu + 8 + warp * " << words << ";\n";
    int off = 0;
    for (auto& a : L.arrays) {
      k << "  double* " << a.first << " = wbase + " << off << ";\n";
      off += a.second;
    }
    k << "  wload_tables(s_exp, s_log, s_nu);\n  __syncthreads();\n";
    return std::make_pair(wpb, 8 * (776 + wpb * words));
  };
  // ===================== forward =====================
  {
    WLayout L;
    L.arrays = {{"sY", N1}, {"sL", std::max(N1, gF.nseg)}, {"sA", N1}, {"sR", M}};
    std::ostringstream k;
    k << o.str() << nw.str();
    emit_gather_tables(k, gF, 0, false);
    auto wp = kernel_head(k, L,
        "// Net production rates, one warp per state (Eq. production_rates); arguments as pyro_omega.\n"
        "extern \"C\" __global__ void __launch_bounds__(WPB * 32) pyro_omega_warp(i64 n, const double* __restrict__ g_rho,\n"
        "    const double* __restrict__ g_Tin, int energy_mode, const double* __restrict__ g_Y,\n"
        "    double* __restrict__ g_Tout, double* __restrict__ g_omega, double T_guess, int max_iter, double tol,\n"
        "    unsigned long long* __restrict__ g_fail, double* __restrict__ g_store)");
    k << "  double* sP = sL;   // partial sums of the production rates (after the reactions)\n"
         "  (void)g_store;\n  const float tolf = (float)tol;\n"
         "  for (i64 base = (i64)blockIdx.x * WPB; base < n; base += (i64)gridDim.x * WPB) {\n"
         "    const i64 p = base + warp;\n    if (p >= n) break;   // warp-uniform; no block barrier below\n"
         "    const double rho = g_rho[p];\n    double ys = 0.0;\n"
         "    for (int k = lane; k < NSP; k += 32) {\n      const double y = g_Y[(i64)k * n + p];\n"
         "      sY[k] = y;\n      ys = fma(y, __ldg(w_invW + k), ys);\n    }\n"
         "    if (lane == 0) sY[NSP] = 0.0;\n    const double ysum = warp_sum(ys);\n    __syncwarp();\n"
         "    double T;\n    if (energy_mode) {\n      int it;\n"
         "      T = wtsolve(sY, g_Tin[p], T_guess, max_iter, tolf, &it, lane);\n"
         "      if (lane == 0) {\n        if (it < 0) atomicAdd(g_fail, 1ull);\n        if (g_Tout) g_Tout[p] = T;\n      }\n"
         "    } else {\n      T = g_Tin[p];\n    }\n"
         "    const double lnT = pdm::log(T, s_log), invT = pdm::rcp(T);\n"
         "    const int hi = pdm::to_float_trunc(T) >= (float)TMID;\n"
         "    for (int k = lane; k < NSP; k += 32) {\n" << species_L(false) <<
         "      sL[k] = q;\n      sA[k] = PEXP(q, s_exp) * (rho * sY[k]);\n    }\n"
         "    if (lane == 0) { sL[NSP] = 0.0; sA[NSP] = 1.0; }\n";
    if (plog) k << "    const double lnp = lnT + pdm::log(rho * ysum, s_log) + " << lnR << ";\n";
    k << "    __syncwarp();\n";
    for (auto& c : P.chunks) emit_chunk(k, c, W_FWD);
    k << "    __syncwarp();\n";
    emit_gather_loop(k, gF, 0, 0, "acc = fma(s_nu[(e.x >> 16) & 7u], sR[e.x & 0xffffu], acc);", false, "sP");
    k << "    __syncwarp();\n    for (int k = lane; k < NSP; k += 32) {\n" << gather_total(0, "sP", "w")
      << "      g_omega[(i64)k * n + p] = w;\n    }\n    __syncwarp();\n  }\n}\n";
    out.sources["wfwd"] = k.str();
    out.stats["warp_fwd_warps_per_block"] = wp.first;
    out.smem["wfwd"] = wp.second;
    out.wpb["wfwd"] = wp.first;
  }
  // ===================== JVP =====================
  {
    WLayout L;
    L.arrays = {{"sY", N1}, {"sdY", N1}, {"sL", std::max(N1, gF.nseg)}, {"sA", N1}, {"sdA", N1}, {"sdL", N1}, {"sR", M}};
    std::ostringstream k;
    k << o.str();
    emit_gather_tables(k, gF, 0, false);
    auto wp = kernel_head(k, L,
        "// JVP of the net production rates, one warp per state; arguments as pyro_jvp.  Per reaction the\n"
        "// tangent dR = dkk D + kk (dP' - dP'') of the forward kernel's expression, intermediates recomputed.\n"
        "extern \"C\" __global__ void __launch_bounds__(WPB * 32) pyro_jvp_warp(i64 n, const double* __restrict__ g_rho,\n"
        "    const double* __restrict__ g_T, const double* __restrict__ g_Y, const double* __restrict__ g_drho,\n"
        "    const double* __restrict__ g_dT, const double* __restrict__ g_dY, double* __restrict__ g_dw,\n"
        "    double* __restrict__ g_store)");
    k << "  double* sP = sL;\n  (void)g_store;\n"
         "  for (i64 base = (i64)blockIdx.x * WPB; base < n; base += (i64)gridDim.x * WPB) {\n"
         "    const i64 p = base + warp;\n    if (p >= n) break;\n"
         "    const double rho = g_rho[p], T = g_T[p], drho = g_drho[p], dT = g_dT[p];\n"
         "    const double lnT = pdm::log(T, s_log), invT = pdm::rcp(T), invT2 = invT * invT;\n"
         "    const double drr = drho * pdm::rcp(rho);\n"
         "    const int hi = pdm::to_float_trunc(T) >= (float)TMID;\n"
         "    double ys = 0.0, dys = 0.0;\n"
         "    for (int k = lane; k < NSP; k += 32) {\n"
         "      const double y = g_Y[(i64)k * n + p], dy = g_dY[(i64)k * n + p];\n"
         "      sY[k] = y; sdY[k] = dy;\n"
         "      ys = fma(y, __ldg(w_invW + k), ys); dys = fma(dy, __ldg(w_invW + k), dys);\n"
      << species_L(true) <<
         "      const double E = PEXP(q, s_exp);\n      const double a = E * (rho * y);\n"
         "      sL[k] = q; sA[k] = a;\n"
         "      sdA[k] = fma(a, fma(Lp, dT, drr), E * (rho * dy)); sdL[k] = Lp * dT;\n    }\n"
         "    if (lane == 0) { sY[NSP] = 0.0; sdY[NSP] = 0.0; sL[NSP] = 0.0; sA[NSP] = 1.0; sdA[NSP] = 0.0; sdL[NSP] = 0.0; }\n"
         "    const double ysum = warp_sum(ys), dysum = warp_sum(dys);\n";
    if (plog) k << "    const double lnp = lnT + pdm::log(rho * ysum, s_log) + " << lnR << ";\n";
    k << "    __syncwarp();\n";
    for (auto& c : P.chunks) emit_chunk(k, c, W_JVP);
    k << "    __syncwarp();\n";
    emit_gather_loop(k, gF, 0, 0, "acc = fma(s_nu[(e.x >> 16) & 7u], sR[e.x & 0xffffu], acc);", false, "sP");
    k << "    __syncwarp();\n    for (int k = lane; k < NSP; k += 32) {\n" << gather_total(0, "sP", "w")
      << "      g_dw[(i64)k * n + p] = w;\n    }\n    __syncwarp();\n  }\n}\n";
    out.sources["wjvp"] = k.str();
    out.stats["warp_jvp_warps_per_block"] = wp.first;
    out.smem["wjvp"] = wp.second;
    out.wpb["wjvp"] = wp.first;
  }
  // ===================== VJP =====================
  {
    WLayout L;
    L.arrays = {{"sY", std::max(N1, gA.nseg)}, {"sWb", std::max(N1, gC.nseg)}, {"sL", N1}, {"sA", N1}, {"sLp", N1},
                {"sDb", M}, {"sMb", std::max(1, M - P.nplain)}};
    std::ostringstream k;
    k << o.str();
    emit_gather_tables(k, gA, 1, false);
    emit_gather_tables(k, gC, 2, true);
    auto wp = kernel_head(k, L,
        "// VJP (reverse mode) of the net production rates, one warp per state; arguments as pyro_vjp.\n"
        "// Per reaction the adjoint R_bar = sum_k nu_kj omega_bar_k; the species adjoints of the\n"
        "// activity products and of [M] are gathered per species afterwards (nothing stored\n"
        "// between calls; the per-reaction intermediates are recomputed).\n"
        "extern \"C\" __global__ void __launch_bounds__(WPB * 32) pyro_vjp_warp(i64 n, const double* __restrict__ g_rho,\n"
        "    const double* __restrict__ g_T, const double* __restrict__ g_Y, const double* __restrict__ g_wb,\n"
        "    double* __restrict__ g_rhob, double* __restrict__ g_Tb, double* __restrict__ g_Yb,\n"
        "    double* __restrict__ g_store)");
    k << "  double* sPa = sY;    // partial sums of the activity adjoints (after the reactions)\n"
         "  double* sPc = sWb;   // partial sums of the efficiency adjoints\n  (void)g_store;\n"
         "  for (i64 base = (i64)blockIdx.x * WPB; base < n; base += (i64)gridDim.x * WPB) {\n"
         "    const i64 p = base + warp;\n    if (p >= n) break;\n"
         "    const double rho = g_rho[p], T = g_T[p];\n"
         "    const double lnT = pdm::log(T, s_log), invT = pdm::rcp(T), invT2 = invT * invT;\n"
         "    const int hi = pdm::to_float_trunc(T) >= (float)TMID;\n"
         "    double ys = 0.0;\n"
         "    for (int k = lane; k < NSP; k += 32) {\n"
         "      const double y = g_Y[(i64)k * n + p];\n"
         "      sY[k] = y; sWb[k] = g_wb[(i64)k * n + p];\n"
         "      ys = fma(y, __ldg(w_invW + k), ys);\n"
      << species_L(true) <<
         "      sL[k] = q; sA[k] = PEXP(q, s_exp) * (rho * y); sLp[k] = Lp;\n    }\n"
         "    if (lane == 0) { sY[NSP] = 0.0; sWb[NSP] = 0.0; sL[NSP] = 0.0; sA[NSP] = 1.0; sLp[NSP] = 0.0; }\n"
         "    const double ysum = warp_sum(ys);\n";
    if (plog) k << "    const double lnp = lnT + pdm::log(rho * ysum, s_log) + " << lnR << ";\n";
    k << "    double Tbp = 0.0, Mtp = 0.0, rMp = 0.0;\n    __syncwarp();\n";
    for (auto& c : P.chunks) emit_chunk(k, c, W_VJP);
    k << "    __syncwarp();\n    const double Mtot = warp_sum(Mtp);\n";
    // activity adjoints: entries with one other factor, then with two (sign bit 16 of x: product side)
    emit_gather_loop(k, gA, 1, 0,
        "const double db = sDb[e.x & 0xffffu]; acc = (e.x >> 16) & 1u ? fma(-db, sA[e.y & 1023u], acc) : "
        "fma(db, sA[e.y & 1023u], acc);", false, "sPa");
    emit_gather_loop(k, gA, 1, 1,
        "const double db = sDb[e.x & 0xffffu]; const double pa = sA[e.y & 1023u] * sA[(e.y >> 10) & 1023u]; "
        "acc = (e.x >> 16) & 1u ? fma(-db, pa, acc) : fma(db, pa, acc);", false, "sPa");
    emit_gather_loop(k, gC, 2, 0, "acc = fma(sMb[e.x & 0xffffu], c, acc);", true, "sPc");
    k << "    __syncwarp();\n    double rbp = 0.0;\n"
         "    for (int k = lane; k < NSP; k += 32) {\n" << gather_total(1, "sPa", "ab") << gather_total(2, "sPc", "sc") <<
         "      const double ta = ab * sA[k];\n      Tbp = fma(ta, sLp[k], Tbp);\n      rbp += ta;\n"
         "      g_Yb[(i64)k * n + p] = fma(ab, PEXP(sL[k], s_exp) * rho, rho * fma(Mtot, __ldg(w_invW + k), sc));\n"
         "    }\n"
         "    const double Tb = warp_sum(Tbp), rhob = warp_sum(rbp), rhobM = warp_sum(rMp);\n"
         "    if (lane == 0) { g_Tb[p] = Tb; g_rhob[p] = fma(rhob, pdm::rcp(rho), rhobM); }\n"
         "    __syncwarp();\n  }\n}\n";
    out.sources["wvjp"] = k.str();
    out.stats["warp_vjp_warps_per_block"] = wp.first;
    out.smem["wvjp"] = wp.second;
    out.wpb["wvjp"] = wp.first;
  }
  // ===================== dense Jacobians, one block of 8 warps per state =====================
  // Phase A (threads over species): thermo, activities, c_v.  Phase B (warps over
  // chunks of 32 reactions, balanced by an operation estimate): per reaction
  // dR/dT, the [M] term and one partial per factor occurrence and efficiency term
  // (slots of sG).  Phase C: balanced gathers over the block's 256 threads -- the
  // column of dT (sum nu dR/dT), the [M] rank-one factor u_k = sum nu kM D rho,
  // the Tdot row's column sums -- then, per group of rows, the nonzero species
  // entries (sum nu partial) into shared memory and every entry of the rows
  // written once (u_k/W_i plus the nonzero part).
  auto cta_jac = [&](bool ty) -> bool {
    const int LN = 256, NW = 8, NB = (N + 31) / 32;
    const int CL = kJacCluster, CB16 = (N + 15) / 16;   // blocks per cluster (states), 16-column blocks
    std::vector<WChunk> ch = P.chunks;
    int gtot = 0;
    for (auto& c : ch) { c.goff = gtot; gtot += chunk_gslots(c); }
    const unsigned GZ = (unsigned)gtot;   // zero slot (gather padding)
    if (gtot + 1 > 65536 || M >= (1 << 20)) return false;
    // every reaction slot's partials: (species, slot of sG)
    std::vector<std::vector<std::pair<int, unsigned>>> part(M);
    for (auto& c : ch)
      for (int l = 0; l < c.count; ++l) {
        const int s = c.base + l;
        const Reaction& r = m.reactions[P.order[s]];
        std::vector<int> fr = side_factors(r.reactants);
        for (size_t q = 0; q < fr.size(); ++q) part[s].push_back({fr[q], (unsigned)(c.goff + q * 32 + l)});
        if (c.rev) {
          std::vector<int> fp = side_factors(r.products);
          for (size_t q = 0; q < fp.size(); ++q) part[s].push_back({fp[q], (unsigned)(c.goff + (c.nf + q) * 32 + l)});
        }
        if (c.kind != WK_PLAIN && c.kind != WK_PLOG) {
          int q = 0;
          for (auto& e : r.efficiencies) {
            if (e.second == 1.0) continue;
            part[s].push_back({e.first, (unsigned)(c.goff + (chunk_occ(c) + q) * 32 + l)});
            ++q;
          }
        }
      }
    // gathers: dT column and [M] factor (the production-rate pairs), Tdot column sums
    const Gather gJ = build_gather(N, {fw}, LN);
    std::vector<GItem> td;
    if (ty)
      for (int s = 0; s < M; ++s)
        for (auto& pi : part[s]) td.push_back({pi.first, pi.second, (unsigned)s, 0.0});
    const Gather gT = build_gather(N, {td}, LN);
    // nonzero pattern of the species block and its terms
    std::vector<std::map<int, std::vector<std::pair<unsigned, int>>>> rowt(N);
    for (int s = 0; s < M; ++s)
      for (auto& kn : net_nu(m.reactions[P.order[s]]))
        if (kn.second)
          for (auto& pi : part[s]) rowt[kn.first][pi.first].push_back({pi.second, kn.second});
    // row groups: the nonzero sums of a group (and 256 carries) reuse the
    // reaction arrays dR/dT, [M] term and energy change (3 M doubles)
    const int region = std::max(3 * M, 1280), cap = region - LN;
    struct RGroup { int r0, r1, nnz; };
    std::vector<RGroup> groups;
    for (int k = 0; k < N;) {
      RGroup g{k, k, 0};
      while (g.r1 < N && g.nnz + (int)rowt[g.r1].size() <= cap) g.nnz += (int)rowt[g.r1++].size();
      groups.push_back(g);
      k = g.r1;
    }
    std::vector<unsigned> jm((size_t)2 * N * NB, 0u);   // per (row, 32-column block): mask, group-local base
    std::vector<NzGather> nzg;
    double nz_terms = 0, nnz_total = 0;
    for (auto& g : groups) {
      std::vector<NzItem> its;
      int key = 0;
      for (int k = g.r0; k < g.r1; ++k) {
        for (int b = 0; b < NB; ++b) jm[2 * ((size_t)k * NB + b) + 1] = (unsigned)key;   // base before the block's first
        int bprev = -1;
        for (auto& it : rowt[k]) {
          const int i = it.first, b = i / 32;
          if (b != bprev) { jm[2 * ((size_t)k * NB + b) + 1] = (unsigned)key; bprev = b; }
          jm[2 * ((size_t)k * NB + b)] |= 1u << (i % 32);
          for (auto& t : it.second) its.push_back({key, t.first, t.second});
          ++key;
        }
      }
      nz_terms += its.size();
      nnz_total += key;
      nzg.push_back(build_nz_gather(its, key, LN, GZ));
    }
    // ---- source
    std::ostringstream k;
    k << o.str();
    std::vector<double> cpt(2 * 5 * N1, 0.0), cdt(2 * 4 * N1, 0.0);
    for (int q = 0; q < N; ++q)
      for (int r = 0; r < 2; ++r) {
        for (int t = 0; t < 5; ++t) cpt[(r * 5 + t) * N1 + q] = C[q].cp[r][t];
        for (int t = 0; t < 4; ++t) cdt[(r * 4 + t) * N1 + q] = C[q].cpd[r][t];
      }
    emit_array(k, "double", "w_Cp", cpt, true);
    if (ty) emit_array(k, "double", "w_Cd", cdt, true);
    if (!ty) {
      std::vector<double> Wt(N);
      for (int q = 0; q < N; ++q) Wt[q] = m.species[q].W;
      emit_array(k, "double", "w_W", Wt, true);
    }
    emit_gather_tables(k, gJ, 3, false);
    if (ty) emit_gather_tables(k, gT, 4, false);
    k << "__device__ const uint2 w_jm[" << N * NB << "] = {";
    for (int q = 0; q < N * NB; ++q) k << (q ? "," : "") << "{" << jm[2 * q] << "u," << jm[2 * q + 1] << "u}";
    k << "};\n";
    for (size_t g = 0; g < nzg.size(); ++g) {
      emit_array(k, "unsigned", "w_jz" + std::to_string(g), nzg[g].ent, false);
      emit_array(k, "unsigned", "w_jl" + std::to_string(g), nzg[g].lane0, false);
      emit_array(k, "unsigned", "w_jf" + std::to_string(g), nzg[g].fix, false);
    }
    k << R"(
// Thread-block cluster of CL blocks (consecutive states): rank, barrier over the
// cluster's threads (release/acquire: shared-memory writes before it are visible
// to every block of the cluster after it), and a load from another block's
// shared memory at the address of the same variable.
__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}
__device__ __forceinline__ double ld_dsmem(const double* q, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(q);
  unsigned ra;
  double v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra));
  return v;
}
// warp sums of four values at once (every lane gets all four): 6 FP64 adds per lane
__device__ __forceinline__ void warp_sum4(double (&v)[4], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double mine = b4 ? v[q + 2] : v[q], give = b4 ? v[q] : v[q + 2];
    v[q] = mine + __shfl_xor_sync(0xffffffffu, give, 16);
  }
  {
    const double mine = b3 ? v[1] : v[0], give = b3 ? v[0] : v[1];
    v[0] = mine + __shfl_xor_sync(0xffffffffu, give, 8);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 4);
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  const double t = v[0];
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = __shfl_sync(0xffffffffu, t, ((q >> 1) & 1) * 16 + (q & 1) * 8);
}
// block sums of four values (every thread gets all four); sRed: 36 doubles
__device__ __forceinline__ void cta_sum4(double (&v)[4], double* sRed, int warp, int lane) {
  warp_sum4(v, lane);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) sRed[warp * 4 + q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += sRed[w * 4 + threadIdx.x];
    sRed[32 + threadIdx.x] = t;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = sRed[32 + q];
}
)";
    // shared memory (doubles)
    std::vector<std::pair<std::string, int>> arr = {
        {"s_exp", 512}, {"s_log", 256}, {"s_nu", 8}, {"sRed", 80},
        {"sY", N1}, {"sL", N1}, {"sA", N1}, {"sEr", N1}, {"sLp", N1}, {"seh", N1}, {"scm", N1},
        {"sjt", N1}, {"su", N1}, {"sX", N1},
        // (dS/dY: after phase C2, sPj..sPu hold the cluster's jt_k and sPt its dT/dY_i)
        {"sPj", ty ? std::max(1, gJ.nseg) : std::max(gJ.nseg, 2 * N)},
        {"sPu", ty ? std::max(1, gJ.nseg) : std::max(gJ.nseg, 2 * N)},
        {"sPt", ty ? std::max(1, gT.nseg) : CL * N},
        {"sG", gtot + 1}, {"sR3", region}, {"sIW", N1}, {"sJMw", N * NB}};
    int words = 0;
    for (auto& a : arr) words += a.second;
    const long bytes = 8L * words;
    if (bytes > 227L * 1024) return false;
    const std::string kname = ty ? "pyro_jacobian_cta" : "pyro_jacobian_adiabatic_cta";
    k << "\n// " << (ty ? "Dense Jacobian d(Tdot, omega)/d(T, Y) at fixed rho (arguments and layout as pyro_jacobian)"
                        : "dS/dY at fixed (rho, e), S = W omega (arguments and layout as pyro_jacobian_adiabatic)")
      << ",\n// one block of " << NW << " warps per state.\n"
      << "extern \"C\" __global__ void __cluster_dims__(" << CL << ", 1, 1) __launch_bounds__(" << LN << ", 2) " << kname
      << "(i64 n, const double* __restrict__ g_rho,\n"
         "    const double* __restrict__ g_T, const double* __restrict__ g_Y, double* __restrict__ g_J,\n"
         "    double* __restrict__ g_scratch) {\n"
         "  extern __shared__ double smem[];\n  (void)g_scratch;\n";
    int off = 0;
    for (auto& a : arr) {
      k << "  double* " << a.first << " = smem + " << off << ";\n";
      off += a.second;
    }
    k << "  double* sRt = sR3;\n  double* sRM = sR3 + " << M << ";\n  double* sDE = sR3 + " << 2 * M << ";\n"
      << "  double* sU4 = sY;           // the cluster's u_k, [state][species] (during the row groups)\n"
      << (ty ? "" : "  double* sJT4 = sPj;         // the cluster's W_k jt_k and dT/dY_i (dS/dY, during the row groups)\n"
                    "  double* sX4 = sPt;\n")
      << "  // 16-byte stores of two adjacent states need an even state count and a 16-byte aligned J\n"
      << "  const bool vec2 = (n & 1) == 0 && (reinterpret_cast<unsigned long long>(g_J) & 15ull) == 0;\n"
      << "  (void)vec2;\n"
      << "  double* sP = sR3;            // nonzero sums of a row group (after the gathers)\n"
      << "  double* sC = sR3 + " << cap << ";   // carries of the row-group gathers\n"
      << "  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;\n"
      << "  uint2* sJM = reinterpret_cast<uint2*>(sJMw);   // (mask, base) of every (row, 32-column block)\n"
      << "  wload_tables(s_exp, s_log, s_nu);\n  if (tid == 0) sG[" << GZ << "] = 0.0;\n"
      << "  for (int q = tid; q < NSP; q += " << LN << ") sIW[q] = __ldg(w_invW + q);\n"
      << "  for (int q = tid; q < " << N * NB << "; q += " << LN << ") sJM[q] = __ldg(w_jm + q);\n"
      << "  __syncthreads();\n"
      << "  // the cluster's blocks take the consecutive states pb .. pb + CL - 1 (a block past\n"
         "  // the end evaluates the last state again and writes nothing of its own)\n"
         "  const unsigned crank = cl_rank();\n"
         "  for (i64 pb = (i64)(blockIdx.x - crank); pb < n; pb += gridDim.x) {\n"
         "    const bool act = pb + crank < n;\n    const i64 p = act ? pb + crank : n - 1;\n"
      << "    const double rho = g_rho[p], T = g_T[p];\n"
         "    const double lnT = pdm::log(T, s_log), invT = pdm::rcp(T), invT2 = invT * invT;\n"
         "    const double RT = " << lit((double)R_GAS) << " * T;\n"
         "    const int hi = pdm::to_float_trunc(T) >= (float)TMID;\n"
         "    double red[4] = {0.0, 0.0, 0.0, 0.0};   // sum Y/W, c_v, dc_v/dT\n"
         "    for (int k = tid; k < NSP; k += " << LN << ") {\n"
         "      const double y = g_Y[(i64)k * n + p];\n"
      << species_L(true) <<
         "      const double E = PEXP(q, s_exp);\n"
         "      sY[k] = y; sL[k] = q; sA[k] = E * (rho * y); sEr[k] = E * rho; sLp[k] = Lp;\n"
         "      seh[k] = fma(RT, hr, -RT);\n"
         "      const double* Cp = w_Cp + hi * 5 * (NSP + 1);\n"
         "      double cp = fma(T, __ldg(Cp + 4 * (NSP + 1) + k), __ldg(Cp + 3 * (NSP + 1) + k));\n"
         "      cp = fma(T, cp, __ldg(Cp + 2 * (NSP + 1) + k));\n"
         "      cp = fma(T, cp, __ldg(Cp + (NSP + 1) + k));\n"
         "      cp = fma(T, cp, __ldg(Cp + k));\n"
         "      const double yw = y * __ldg(w_invW + k), ywR = yw * " << lit((double)R_GAS) << ";\n"
         "      red[0] += yw;\n      red[1] = fma(ywR, cp - 1.0, red[1]);\n";
    if (ty)
      k << "      scm[k] = " << lit((double)R_GAS) << " * (cp - 1.0);\n"
           "      const double* Cd = w_Cd + hi * 4 * (NSP + 1);\n"
           "      double cd = fma(T, __ldg(Cd + 3 * (NSP + 1) + k), __ldg(Cd + 2 * (NSP + 1) + k));\n"
           "      cd = fma(T, cd, __ldg(Cd + (NSP + 1) + k));\n"
           "      cd = fma(T, cd, __ldg(Cd + k));\n"
           "      red[2] = fma(ywR, cd, red[2]);\n";
    k << "    }\n"
         "    if (tid == 0) { sY[NSP] = 0.0; sL[NSP] = 0.0; sA[NSP] = 1.0; sEr[NSP] = 0.0; sLp[NSP] = 0.0; seh[NSP] = 0.0; "
         "scm[NSP] = 0.0; }\n"
         "    cta_sum4(red, sRed, warp, lane);\n"
         "    const double ysum = red[0], cv = red[1], cvT = red[2];\n    (void)cvT;\n";
    if (plog) k << "    const double lnp = lnT + pdm::log(rho * ysum, s_log) + " << lnR << ";\n";
    // phase B: chunks to warps, largest estimated cost first, to the least loaded warp
    // cost of a chunk: the FP64 operations of its emitted code (fma, binary + - *,
    // and the device exponential / logarithm / reciprocal at their operation counts)
    auto count = [](const std::string& t, const std::string& pat) {
      double c = 0;
      for (size_t at = t.find(pat); at != std::string::npos; at = t.find(pat, at + pat.size())) ++c;
      return c;
    };
    std::vector<double> cost(ch.size());
    for (size_t c = 0; c < ch.size(); ++c) {
      std::ostringstream t;
      emit_chunk(t, ch[c], ty ? W_JAC : W_JAD);
      const std::string x = t.str();
      cost[c] = count(x, "fma(") + count(x, " * ") + count(x, " + ") + count(x, " - ") +
                opt.warp_exp_ops * count(x, "PEXP(") + 7 * count(x, "pdm::log(") + 4 * count(x, "pdm::rcp(");
    }
    std::vector<int> ordc(ch.size());
    for (size_t c = 0; c < ch.size(); ++c) ordc[c] = (int)c;
    std::stable_sort(ordc.begin(), ordc.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<std::vector<int>> own(NW);
    std::vector<double> load(NW, 0.0);
    for (int c : ordc) {
      const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      own[w].push_back(c);
      load[w] += cost[c];
    }
    {
      double mx = 0, sum = 0;
      for (double l : load) { mx = std::max(mx, l); sum += l; }
      out.stats[std::string(ty ? "wjac" : "wjad") + "_reaction_phase_imbalance"] = sum > 0 ? mx * NW / sum : 1.0;
    }
    k << "    double pew = 0.0, pcw = 0.0, pejt = 0.0, pU = 0.0;   // sums over reactions (Tdot row)\n";
    for (int w = 0; w < NW; ++w) {
      std::sort(own[w].begin(), own[w].end());
      k << "    if (warp == " << w << ") {\n";
      for (int c : own[w]) emit_chunk(k, ch[c], ty ? W_JAC : W_JAD);
      k << "    }\n";
    }
    k << "    __syncthreads();\n";
    // phase C1: gathers
    emit_gather_loop(k, gJ, 3, 0,
        "const double nu = s_nu[(e.x >> 16) & 7u]; const unsigned s = e.x & 0xffffu; "
        "acc = fma(nu, sRt[s], acc); acc2 = fma(nu, sRM[s], acc2);", false, "sPj", "tid", "sPu");
    if (ty) {
      emit_gather_loop(k, gT, 4, 0, "acc = fma(sDE[e.y & 0xfffffu], sG[e.x], acc);", false, "sPt", "tid");
      k << "    double r4[4] = {pew, pcw, pejt, pU};\n    cta_sum4(r4, sRed + 40, warp, lane);\n"
           "    const double rcv = pdm::rcp(rho * cv), Tdot = -r4[0] * rcv, tcv = Tdot * pdm::rcp(cv);\n"
           "    if (tid == 0 && act) g_J[p] = fma(-(r4[1] + r4[2]), rcv, -tcv * cvT);\n";
    } else {
      k << "    __syncthreads();\n    const double mrcv = -pdm::rcp(cv);\n";
    }
    // phase C2: per-species totals, the dT column (ty) and the Tdot row (ty)
    k << "    for (int k = tid; k < NSP; k += " << LN << ") {\n" << gather_total(3, "sPj", "jt")
      << gather_total(3, "sPu", "u");
    if (ty) {
      k << gather_total(4, "sPt", "td") <<
           "      sjt[k] = jt; su[k] = u;\n"
           "      const double iw = __ldg(w_invW + k);\n"
           "      if (act) {\n"
           "        g_J[(i64)(1 + k) * " << N1 << " * n + p] = jt;\n"
           "        g_J[(i64)(1 + k) * n + p] = fma(-fma(iw, r4[3], td), rcv, -tcv * (scm[k] * iw));\n"
           "      }\n";
    } else {
      k << "      const double Wk = __ldg(w_W + k);\n"
           "      sjt[k] = Wk * jt; su[k] = Wk * u;\n"
           "      sX[k] = (seh[k] * __ldg(w_invW + k)) * mrcv;   // dT/dY_k at fixed e\n";
    }
    k << "    }\n    __syncthreads();\n";
    // phase C3: row groups
    for (size_t g = 0; g < groups.size(); ++g) {
      const RGroup& G = groups[g];
      const NzGather& Z = nzg[g];
      const std::string gs = std::to_string(g);
      k << "    { // rows " << G.r0 << ".." << G.r1 - 1 << ": " << G.nnz << " nonzero species entries\n"
           "      const unsigned l0 = __ldg(w_jl" << gs << " + tid);\n"
           "      int key = (int)(l0 & 0x7fffffffu);\n      bool carry = (l0 >> 31) != 0u;\n"
           "      double acc = 0.0;\n#pragma unroll 4\n"
           "      for (int st = 0; st < " << Z.steps << "; ++st) {\n"
           "        const unsigned e = __ldg(w_jz" << gs << " + st * " << LN << " + tid);\n"
           "        acc = fma(s_nu[(e >> 16) & 7u], sG[e & 0xffffu], acc);\n"
           "        if (e & (1u << 19)) { if (carry) { sC[tid] = acc; carry = false; } else { sP[key] = acc; } ++key; acc = 0.0; }\n"
           "      }\n    }\n    __syncthreads();\n";
      if (!Z.fix.empty())
        k << "    if (tid < " << Z.fix.size() << ") {\n"
             "      const unsigned f = __ldg(w_jf" << gs << " + tid);\n"
             "      const int K = (int)(f & 0xffffu);\n      double v = sP[K];\n"
             "      for (int l = (int)((f >> 16) & 255u); l <= (int)(f >> 24); ++l) v += sC[l];\n"
             "      sP[K] = v;\n    }\n";
      // every block's sums of this row group complete and visible to the cluster
      k << "    cl_sync();\n";
      // the cluster's u_k (and for dS/dY jt_k and dT/dY_i), written in phase C2 of
      // every block and so complete now, copied once per state into arrays of this
      // block that are free by then (species arrays, gather segments)
      if (g == 0) {
        k << "    for (int q = tid; q < " << CL * N << "; q += " << LN << ") {\n"
             "      const unsigned r = (unsigned)(q / NSP);\n      const int c = q % NSP;\n"
             "      sU4[q] = ld_dsmem(su + c, r);\n";
        if (!ty) k << "      sJT4[q] = ld_dsmem(sjt + c, r);\n      sX4[q] = ld_dsmem(sX + c, r);\n";
        k << "    }\n    __syncthreads();\n";
      }
      // the rows of the group for the cluster's CL states: each (row, 16-column block)
      // item is one warp instruction, lane 2c + h holding column 16 cb + c of states
      // 2h and 2h + 1 (one 16-byte store; two lanes fill one 32-byte sector of J); the
      // other blocks' nonzero sums are read from their shared memory
      k << "    for (int q = (int)crank * " << NW << " + warp; q < " << (G.r1 - G.r0) * CB16 << "; q += " << NW * CL << ") {\n"
           "      const int k = " << G.r0 << " + q / " << CB16 << ", i = (q % " << CB16 << ") * 16 + (lane >> 1);\n"
           "      const unsigned s0 = (lane & 1u) * 2u;\n";
      if (N % 16) k << "      if (i < NSP) {\n";
      else k << "      {\n";
      k << "        const uint2 mb = sJM[k * " << NB << " + (i >> 5)];\n"
           "        const int bit = i & 31;\n"
           "        const bool nz = (mb.x >> bit) & 1u;\n"
           "        const double* sPi = sP + mb.y + __popc(mb.x & ((1u << bit) - 1u));\n"
           "        const double t0 = nz ? ld_dsmem(sPi, s0) : 0.0, t1 = nz ? ld_dsmem(sPi, s0 + 1u) : 0.0;\n"
           "        const double iw = sIW[i];\n";
      if (ty)
        k << "        const double v0 = fma(sU4[s0 * NSP + k], iw, t0), v1 = fma(sU4[(s0 + 1u) * NSP + k], iw, t1);\n"
             "        double* dst = g_J + ((i64)(1 + k) * " << N1 << " + 1 + i) * n + pb + s0;\n";
      else
        k << "        const double Wk = __ldg(w_W + k);\n"
             "        double v0 = fma(sJT4[s0 * NSP + k], sX4[s0 * NSP + i], sU4[s0 * NSP + k] * iw);\n"
             "        double v1 = fma(sJT4[(s0 + 1u) * NSP + k], sX4[(s0 + 1u) * NSP + i], sU4[(s0 + 1u) * NSP + k] * iw);\n"
             "        if (nz) { v0 = fma(Wk, t0, v0); v1 = fma(Wk, t1, v1); }\n"
             "        double* dst = g_J + ((i64)k * " << N << " + i) * n + pb + s0;\n";
      k << "        if (vec2 && pb + s0 + 1 < n) {\n"
           "          *reinterpret_cast<double2*>(dst) = make_double2(v0, v1);\n"
           "        } else {\n"
           "          if (pb + s0 < n) dst[0] = v0;\n"
           "          if (pb + s0 + 1 < n) dst[1] = v1;\n"
           "        }\n";
      k << "      }\n    }\n    cl_sync();   // before the next group's gather overwrites the sums\n";
    }
    k << "  }\n}\n";
    const std::string key = ty ? "wjac" : "wjad";
    out.sources[key] = k.str();
    out.wpb[key] = NW;
    out.smem[key] = (int)bytes;
    out.stats[key + "_row_groups"] = (double)groups.size();
    out.stats[key + "_nonzeros"] = nnz_total;
    out.stats[key + "_terms"] = nz_terms;
    out.stats[key + "_partial_slots"] = gtot;
    return true;
  };
  out.stats["jacobian_cta"] = cta_jac(true) ? 1 : 0;
  out.stats["jacobian_adiabatic_cta"] = cta_jac(false) ? 1 : 0;
  out.stats["warp_chunks"] = (double)P.chunks.size();
  out.stats["warp_gather_steps"] = gF.loops[0].steps;
  out.stats["warp_segments"] = gF.nseg;
  out.stats["warp_warps_per_block"] = out.wpb["wfwd"];
  out.stats["warp_smem_bytes"] = out.smem["wfwd"];
  out.warps_per_block = out.wpb["wfwd"];
  out.smem_bytes = out.smem["wfwd"];
  return out;
}

}  // namespace pyro
