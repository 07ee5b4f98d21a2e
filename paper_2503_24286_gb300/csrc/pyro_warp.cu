// Warp-per-point net production rates, table-driven (no JIT compilation).
//
// One warp evaluates one state: its 32 lanes split the species (thermo, the
// activities a_k = exp(L_k) rho Y_k) and the reactions (one exponential per
// reaction of the same activity formulation as the emitted kernels), stage
// L_k, a_k and R_j in the warp's shared memory, then split the species again to
// gather omega_k = sum_j nu_kj R_j through a CSR table of the stoichiometry
// (Sec. A.1 Eq. production_rates, Eq. reaction_rates, Eq. equil_constants).
// Reactions are grouped into classes of equal shape (kind, reactant and product
// factor counts) so the lanes of a warp run the same code; per-reaction
// constants and species indices come from tables in global memory.  The
// temperature (energy input) is solved per warp with the same FP32-then-FP64
// Newton on collapsed mixture polynomials as the emitted kernels, with the
// species sums reduced across lanes.
//
// This layout keeps the per-state species arrays in shared memory for any
// mechanism size (12.6 KB per warp for 160 species / 1100 reactions) and needs
// no mechanism-specialised compilation; the emitted thread-per-point kernels are
// the alternative it is measured against.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "pyro.h"
#include "pyro_device_math.cuh"
#include "pyro_internal.h"
#include "pyro_mech.h"

namespace {

typedef long long i64;

constexpr int WARPS = 8;               // states per block iteration (one per warp)
constexpr int MAXC = 40;               // reaction classes
constexpr int NEFF = 8;                // third-body efficiency slots per reaction
constexpr int NFO = 12;                // falloff constants per reaction

struct ClassTab {
  int n;
  int kind[MAXC], nf[MAXC], nr[MAXC], rev[MAXC], start[MAXC], count[MAXC];
};

struct Tabs {
  int N, M, nnz;
  double tmid;
  const double* Lc;     // [2][7][N]: cl, ci, c0, c1, c2, c3, c4
  const double* dc;     // [2][6][N]
  const float* dcf;     // [2][6][N]
  const double* invW;   // [N]
  const double* rx;     // [M][3]: lnA', b, theta   (class order)
  const short* fac;     // [M][6]: reactant factors then product factors (class order)
  const short* effi;    // [M][NEFF]
  const double* effc;   // [M][NEFF]: (eps - 1)/W
  const double* fo;     // [M][NFO]: falloff constants
  const int* rowptr;    // [N+1] CSR of nu (rows: species in lane order)
  const int* col;       // [nnz] reaction slot
  const double* val;    // [nnz] nu
  const int* sperm;     // [N] species of CSR row r
  const double* tab;    // [512 exp table][256 log table]
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Newton inversion of e (per warp, uniform across lanes) -- Sec. A.3.1 Eq. delta_temp
__device__ double warp_tsolve(const Tabs& t, const double* sY, double e, int max_iter, float tolf, int* iters,
                              int lane) {
  const int N = t.N;
  const double eR = e * (1.0 / 8314.462618);
  float bf[2][6];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int q = 0; q < 6; ++q) bf[r][q] = 0.f;
  for (int k = lane; k < N; k += 32) {
    float y = pdm::to_float_trunc(sY[k]);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int q = 0; q < 6; ++q) bf[r][q] = fmaf(y, t.dcf[(r * 6 + q) * N + k], bf[r][q]);
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int q = 0; q < 6; ++q) bf[r][q] = warp_sumf(bf[r][q]);
  float Tf = 1200.f;
  const float eRf = pdm::to_float_trunc(eR);
  const float tmf = (float)t.tmid;
  int it32 = 0;
  for (; it32 < 40;) {
    ++it32;
    int h = Tf >= tmf;
    const float* c = bf[h];
    float ef = fmaf(Tf, fmaf(Tf, fmaf(Tf, fmaf(Tf, fmaf(Tf, c[5], c[4]), c[3]), c[2]), c[1]), c[0]);
    float cvf = fmaf(Tf, fmaf(Tf, fmaf(Tf, fmaf(Tf, 5.f * c[5], 4.f * c[4]), 3.f * c[3]), 2.f * c[2]), c[1]);
    float Tn = fminf(fmaxf(Tf + (eRf - ef) * __frcp_rn(cvf), 100.f), 5000.f);
    bool conv = fabsf(Tn - Tf) <= 1e-5f * Tn;
    Tf = Tn;
    if (conv) break;
  }
  double T = pdm::to_double(Tf);
  int hi = pdm::to_float_trunc(T) >= tmf;
  double B[6];
  auto collapse = [&](int r) {
    double p[6] = {0, 0, 0, 0, 0, 0};
    for (int k = lane; k < N; k += 32) {
      double y = sY[k];
#pragma unroll
      for (int q = 0; q < 6; ++q) p[q] = fma(y, t.dc[(r * 6 + q) * N + k], p[q]);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) B[q] = warp_sum(p[q]);
  };
  collapse(hi);
  int it64 = 0;
  bool flag = false, ok = false;
  for (int it = 0; it < max_iter + 1; ++it) {
    ++it64;
    float Tcur = pdm::to_float_trunc(T);
    int h2 = Tcur >= tmf;
    if (h2 != hi) { hi = h2; collapse(hi); }
    double e64 = fma(T, fma(T, fma(T, fma(T, fma(T, B[5], B[4]), B[3]), B[2]), B[1]), B[0]);
    const float* c = bf[hi];
    float cvf = fmaf(Tcur, fmaf(Tcur, fmaf(Tcur, fmaf(Tcur, 5.f * c[5], 4.f * c[4]), 3.f * c[3]), 2.f * c[2]), c[1]);
    double dT = (e64 - eR) * pdm::to_double(-__frcp_rn(cvf));
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

// One class of reactions, lanes over its members: R_j into sR (slot = class-order index).
template <int KIND, int NF, int NR>
__device__ __forceinline__ void eval_class(const Tabs& t, int start, int count, int rev, const double* sL,
                                           const double* sA, const double* sY, double* sR, double T, double lnT,
                                           double invT, double rho, double ysum, const double* se,
                                           const double* sl, int lane) {
  for (int j = start + lane; j < start + count; j += 32) {
    const double* c = t.rx + (i64)j * 3;
    const short* f = t.fac + (i64)j * 6;
    double x = fma(c[1], lnT, c[0]);
    x = fma(-c[2], invT, x);
    double Pf = 1.0, Pr = 0.0;
#pragma unroll
    for (int q = 0; q < NF; ++q) { int i = f[q]; x -= sL[i]; Pf = q ? Pf * sA[i] : sA[i]; }
    double kt = pdm::exp(x, se);
    if (rev) {
      Pr = sA[f[3]];
#pragma unroll
      for (int q = 1; q < NR; ++q) Pr *= sA[f[3 + q]];
    }
    if (KIND != 0) {
      const short* ei = t.effi + (i64)j * NEFF;
      const double* ec = t.effc + (i64)j * NEFF;
      double mS = ysum;
#pragma unroll
      for (int q = 0; q < NEFF; ++q) mS = fma(sY[ei[q]], ec[q], mS);
      double M = rho * mS;
      if (KIND == 1) {
        kt *= M;
      } else {
        const double* o = t.fo + (i64)j * NFO;
        // o: q0, db, dth, one_minus_a, -1/T3, a, -1/T1, -T2, f3 (T2 present), troe (1/0)
        double lnPr = fma(o[1], lnT, o[0]) + fma(o[2], invT, pdm::log(M, sl));
        double fpr = pdm::rcp(1.0 + pdm::exp(-lnPr, se));
        double kf = fpr;
        if (o[9] != 0.0) {
          double fc = fma(o[3], pdm::exp(T * o[4], se), fma(o[5], pdm::exp(T * o[6], se), o[8] * pdm::exp(o[7] * invT, se)));
          const double il10 = 0.43429448190325182765;
          double lfc = pdm::log(fc, sl) * il10;
          double cc = fma(-0.67, lfc, -0.4), nn = fma(-1.27, lfc, 0.75);
          double xx = fma(lnPr, il10, cc), den = fma(-0.14, xx, nn);
          double den2 = den * den;
          double lf = lfc * den2 * pdm::rcp(fma(xx, xx, den2));
          kf *= pdm::exp(lf * 2.30258509299404568402, se);
        }
        kt *= kf;
      }
    }
    sR[j] = kt * (Pf - Pr);
  }
}

__device__ __forceinline__ void dispatch_class(int kind, int nf, int nr, const Tabs& t, int start, int count, int rev,
                                               const double* sL, const double* sA, const double* sY, double* sR,
                                               double T, double lnT, double invT, double rho, double ysum,
                                               const double* se, const double* sl, int lane) {
#define PYRO_CASE(K, F, R)                                                                              \
  if (kind == K && nf == F && nr == R) {                                                                \
    eval_class<K, F, R>(t, start, count, rev, sL, sA, sY, sR, T, lnT, invT, rho, ysum, se, sl, lane);  \
    return;                                                                                             \
  }
#define PYRO_CASES_K(K) \
  PYRO_CASE(K, 1, 1) PYRO_CASE(K, 1, 2) PYRO_CASE(K, 1, 3) PYRO_CASE(K, 2, 1) PYRO_CASE(K, 2, 2) \
  PYRO_CASE(K, 2, 3) PYRO_CASE(K, 3, 1) PYRO_CASE(K, 3, 2) PYRO_CASE(K, 3, 3)
  PYRO_CASES_K(0) PYRO_CASES_K(1) PYRO_CASES_K(2)
#undef PYRO_CASES_K
#undef PYRO_CASE
}

__global__ void __launch_bounds__(WARPS * 32) pyro_omega_warp_kernel(
    i64 n, const double* __restrict__ g_rho, const double* __restrict__ g_Tin, int energy_mode,
    const double* __restrict__ g_Y, double* __restrict__ g_Tout, double* __restrict__ g_omega, Tabs t,
    ClassTab ct, int max_iter, double tol, unsigned long long* __restrict__ g_fail) {
  extern __shared__ double smem[];
  double* se = smem;               // 512 exp table
  double* sl = se + 512;           // 256 log table
  const int N = t.N, M = t.M;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* sY = sl + 256 + (size_t)warp * (3 * N + M);
  double* sL = sY + N;
  double* sA = sL + N;
  double* sR = sA + N;
  for (int i = threadIdx.x; i < 768; i += blockDim.x) se[i] = t.tab[i];
  __syncthreads();
  const float tolf = (float)tol;
  for (i64 base = (i64)blockIdx.x * WARPS; base < n; base += (i64)gridDim.x * WARPS) {
    i64 p = base + warp;
    if (p >= n) continue;                         // warp-uniform
    const double rho = g_rho[p];
    double ys = 0.0;
    for (int k = lane; k < N; k += 32) {
      double y = g_Y[(i64)k * n + p];
      sY[k] = y;
      ys = fma(y, t.invW[k], ys);
    }
    const double ysum = warp_sum(ys);
    __syncwarp();
    double T;
    if (energy_mode) {
      int it;
      T = warp_tsolve(t, sY, g_Tin[p], max_iter, tolf, &it, lane);
      if (lane == 0) {
        if (it < 0) atomicAdd(g_fail, 1ull);
        if (g_Tout) g_Tout[p] = T;
      }
    } else {
      T = g_Tin[p];
    }
    const double lnT = pdm::log(T, sl), invT = pdm::rcp(T);
    const int hi = pdm::to_float_trunc(T) >= (float)t.tmid;
    const double* L = t.Lc + (size_t)hi * 7 * N;
    for (int k = lane; k < N; k += 32) {
      double q = fma(T, L[6 * N + k], L[5 * N + k]);
      q = fma(T, q, L[4 * N + k]); q = fma(T, q, L[3 * N + k]); q = fma(T, q, L[2 * N + k]);
      q = fma(L[0 * N + k], lnT, q); q = fma(L[1 * N + k], invT, q);
      sL[k] = q;
      sA[k] = pdm::exp(q, se) * (rho * sY[k]);
    }
    __syncwarp();
    for (int c = 0; c < ct.n; ++c)
      dispatch_class(ct.kind[c], ct.nf[c], ct.nr[c], t, ct.start[c], ct.count[c], ct.rev[c], sL, sA, sY, sR, T, lnT,
                     invT, rho, ysum, se, sl, lane);
    __syncwarp();
    for (int r = lane; r < N; r += 32) {
      double w = 0.0;
      for (int q = t.rowptr[r]; q < t.rowptr[r + 1]; ++q) w = fma(t.val[q], sR[t.col[q]], w);
      g_omega[(i64)t.sperm[r] * n + p] = w;
    }
    __syncwarp();
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host: tables from the mechanism, launch
// ---------------------------------------------------------------------------
namespace pyro {

struct WarpTables {
  Tabs t;
  ClassTab ct;
  void* buf = nullptr;
  int smem = 0;
  int blocks_per_sm = 0;
  std::map<std::string, double> stats;
};

void warp_free(WarpTables* w) {
  if (!w) return;
  cudaFree(w->buf);
  delete w;
}

static int wfail(const char* what, cudaError_t e) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return internal_fail(PYRO_ECUDA, m.c_str());
}

int warp_build(const Mechanism& m, int num_sms, WarpTables** out) {
  const int N = m.n_species(), M = m.n_reactions();
  const long double R = 8314.462618L, P0 = 101325.0L;
  auto* w = new WarpTables();
  // ---- reaction classes
  std::map<std::tuple<int, int, int, int>, std::vector<int>> cls;
  for (int j = 0; j < M; ++j) {
    const Reaction& r = m.reactions[j];
    int nf = 0, nr = 0;
    for (auto& p : r.reactants) nf += p.second;
    for (auto& p : r.products) nr += p.second;
    if (nf < 1 || nf > 3 || nr < 1 || nr > 3 || (int)r.efficiencies.size() > NEFF) {
      delete w;
      return internal_fail(PYRO_EINVAL, "warp variant: reactions need 1-3 factors a side and at most 8 efficiencies");
    }
    cls[std::make_tuple((int)r.kind, nf, nr, r.reversible ? 1 : 0)].push_back(j);
  }
  if ((int)cls.size() > MAXC) { delete w; return internal_fail(PYRO_EINVAL, "warp variant: too many reaction classes"); }
  std::vector<int> order;   // class-order index -> reaction
  ClassTab ct{};
  for (auto& kv : cls) {
    int c = ct.n++;
    ct.kind[c] = std::get<0>(kv.first); ct.nf[c] = std::get<1>(kv.first); ct.nr[c] = std::get<2>(kv.first);
    ct.rev[c] = std::get<3>(kv.first); ct.start[c] = (int)order.size(); ct.count[c] = (int)kv.second.size();
    for (int j : kv.second) order.push_back(j);
  }
  std::vector<int> slot(M);
  for (int q = 0; q < M; ++q) slot[order[q]] = q;
  // ---- species tables
  std::vector<double> Lc(2 * 7 * N), dc(2 * 6 * N), invW(N);
  std::vector<float> dcf(2 * 6 * N);
  for (int k = 0; k < N; ++k) {
    const Species& s = m.species[k];
    long double lnRp0 = logl(R / P0), lnW = logl((long double)s.W), W = s.W;
    invW[k] = (double)(1.0L / W);
    for (int r = 0; r < 2; ++r) {
      const double* a = r ? s.high : s.low;
      double L[7] = {(double)(1.0L - a[0]), a[5], (double)((long double)a[0] - a[6] + lnRp0 - lnW),
                     (double)(-(long double)a[1] / 2), (double)(-(long double)a[2] / 6),
                     (double)(-(long double)a[3] / 12), (double)(-(long double)a[4] / 20)};
      for (int q = 0; q < 7; ++q) Lc[(r * 7 + q) * N + k] = L[q];
      double d[6] = {(double)(a[5] / W), (double)((a[0] - 1.0L) / W), (double)(a[1] / (2 * W)),
                     (double)(a[2] / (3 * W)), (double)(a[3] / (4 * W)), (double)(a[4] / (5 * W))};
      for (int q = 0; q < 6; ++q) { dc[(r * 6 + q) * N + k] = d[q]; dcf[(r * 6 + q) * N + k] = (float)d[q]; }
    }
  }
  // ---- reaction tables (class order)
  std::vector<double> rx(3 * M), effc((size_t)NEFF * M, 0.0), fo((size_t)NFO * M, 0.0);
  std::vector<short> fac(6 * M, 0), effi((size_t)NEFF * M, 0);
  for (int q = 0; q < M; ++q) {
    const Reaction& r = m.reactions[order[q]];
    long double lnA = logl((long double)r.A);
    int f = 0;
    for (auto& p : r.reactants)
      for (int i = 0; i < p.second; ++i) { fac[6 * q + f++] = (short)p.first; lnA -= logl((long double)m.species[p.first].W); }
    int g = 3;
    for (auto& p : r.products)
      for (int i = 0; i < p.second; ++i) fac[6 * q + g++] = (short)p.first;
    rx[3 * q] = (double)lnA; rx[3 * q + 1] = r.b; rx[3 * q + 2] = r.theta;
    int e = 0;
    for (auto& ef : r.efficiencies) {
      effi[NEFF * q + e] = (short)ef.first;
      effc[NEFF * q + e] = (ef.second - 1.0) / m.species[ef.first].W;
      ++e;
    }
    if (r.kind == RX_FALLOFF) {
      double* o = &fo[(size_t)NFO * q];
      o[0] = (double)(logl((long double)r.A0) - logl((long double)r.A));
      o[1] = r.b0 - r.b;
      o[2] = -(r.theta0 - r.theta);
      if (r.n_troe >= 3) {
        o[3] = 1.0 - r.troe[0]; o[4] = -1.0 / r.troe[1]; o[5] = r.troe[0]; o[6] = -1.0 / r.troe[2];
        o[7] = r.n_troe == 4 ? -r.troe[3] : 0.0; o[8] = r.n_troe == 4 ? 1.0 : 0.0; o[9] = 1.0;
      }
    }
  }
  // ---- CSR of nu by species (rows sorted by length so lanes of a round do similar work)
  std::vector<std::vector<std::pair<int, double>>> rows(N);
  for (int j = 0; j < M; ++j) {
    std::map<int, int> nu;
    for (auto& p : m.reactions[j].products) nu[p.first] += p.second;
    for (auto& p : m.reactions[j].reactants) nu[p.first] -= p.second;
    for (auto& q : nu) if (q.second) rows[q.first].push_back({slot[j], (double)q.second});
  }
  std::vector<int> sperm(N);
  for (int k = 0; k < N; ++k) sperm[k] = k;
  std::stable_sort(sperm.begin(), sperm.end(), [&](int a, int b) { return rows[a].size() > rows[b].size(); });
  std::vector<int> rowptr(N + 1, 0), col;
  std::vector<double> val;
  for (int r = 0; r < N; ++r) {
    for (auto& e : rows[sperm[r]]) { col.push_back(e.first); val.push_back(e.second); }
    rowptr[r + 1] = (int)col.size();
  }
  // ---- exp / log tables (Tang's table points, as in the emitted kernels)
  std::vector<double> tab(768);
  for (int j = 0; j < 512; ++j) tab[j] = (double)exp2l((j + 0.5L) / 512.0L);
  for (int j = 0; j < 128; ++j) {
    long double c = 1.0L + (j + 0.5L) / 128.0L;
    tab[512 + 2 * j] = (double)(1.0L / c);
    tab[512 + 2 * j + 1] = (double)logl(c);
  }
  // ---- one device buffer
  std::vector<char> host;
  auto put = [&](const void* p, size_t bytes) {
    size_t off = (host.size() + 255) & ~size_t(255);
    host.resize(off + bytes);
    if (bytes) std::memcpy(host.data() + off, p, bytes);
    return off;
  };
  size_t oLc = put(Lc.data(), Lc.size() * 8), odc = put(dc.data(), dc.size() * 8), odcf = put(dcf.data(), dcf.size() * 4);
  size_t oiw = put(invW.data(), invW.size() * 8), orx = put(rx.data(), rx.size() * 8), ofac = put(fac.data(), fac.size() * 2);
  size_t oei = put(effi.data(), effi.size() * 2), oec = put(effc.data(), effc.size() * 8), ofo = put(fo.data(), fo.size() * 8);
  size_t orp = put(rowptr.data(), rowptr.size() * 4), ocol = put(col.data(), col.size() * 4 + 4);
  size_t oval = put(val.data(), val.size() * 8 + 8), osp = put(sperm.data(), sperm.size() * 4), otab = put(tab.data(), tab.size() * 8);
  cudaError_t e = cudaMalloc(&w->buf, host.size());
  if (e) { delete w; return wfail("warp tables", e); }
  e = cudaMemcpy(w->buf, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e) { warp_free(w); return wfail("warp tables", e); }
  char* b = (char*)w->buf;
  Tabs& t = w->t;
  t.N = N; t.M = M; t.nnz = (int)col.size(); t.tmid = m.species[0].t_mid;
  t.Lc = (const double*)(b + oLc); t.dc = (const double*)(b + odc); t.dcf = (const float*)(b + odcf);
  t.invW = (const double*)(b + oiw); t.rx = (const double*)(b + orx); t.fac = (const short*)(b + ofac);
  t.effi = (const short*)(b + oei); t.effc = (const double*)(b + oec); t.fo = (const double*)(b + ofo);
  t.rowptr = (const int*)(b + orp); t.col = (const int*)(b + ocol); t.val = (const double*)(b + oval);
  t.sperm = (const int*)(b + osp); t.tab = (const double*)(b + otab);
  w->ct = ct;
  w->smem = (int)(sizeof(double) * (768 + (size_t)WARPS * (3 * N + M)));
  if (w->smem > 227 * 1024) {
    warp_free(w);
    return internal_fail(PYRO_EINVAL, "warp variant: per-state arrays of this mechanism exceed shared memory");
  }
  e = cudaFuncSetAttribute(pyro_omega_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, w->smem);
  if (e) { warp_free(w); return wfail("warp kernel shared memory", e); }
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pyro_omega_warp_kernel, WARPS * 32, w->smem);
  if (e || nb < 1) { warp_free(w); return wfail("warp kernel occupancy", e); }
  w->blocks_per_sm = nb;
  w->stats["warp_blocks_per_sm"] = nb;
  w->stats["warp_classes"] = ct.n;
  w->stats["warp_smem_bytes"] = w->smem;
  (void)num_sms;
  *out = w;
  return PYRO_OK;
}

int warp_launch_omega(const WarpTables* w, int num_sms, int64_t n, const double* rho, const double* T_or_e,
                      int energy, const double* Y, double* T_out, double* omega, unsigned long long* fail,
                      cudaStream_t st) {
  i64 need = (n + WARPS - 1) / WARPS;
  i64 cap = (i64)num_sms * w->blocks_per_sm;
  unsigned grid = (unsigned)std::min(need, cap);
  if (!grid) return PYRO_OK;
  pyro_omega_warp_kernel<<<grid, WARPS * 32, w->smem, st>>>(n, rho, T_or_e, energy, Y, T_out, omega, w->t, w->ct, 50,
                                                            1e-10, fail);
  cudaError_t e = cudaGetLastError();
  return e ? wfail("warp kernel launch", e) : PYRO_OK;
}

double warp_stat(const WarpTables* w, const std::string& k) {
  auto it = w->stats.find(k);
  return it == w->stats.end() ? -1.0 : it->second;
}

}  // namespace pyro
