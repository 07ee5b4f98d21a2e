// Device math for FP64-pipe-bound kernels on sm_103a.
//
// On GB300 the FP64 pipe retires 2 lanes/clk/SM while FP32 retires 128 and
// INT 64, and every instruction that touches a double in the FP64 unit --
// DFMA/DADD/DMUL, DSETP, and the F2F/I2F/F2I conversions -- costs one FP64 slot.
// These routines therefore keep only the steps that need 53-bit precision on
// the FP64 pipe and do range reduction, table indexing, exponent arithmetic and
// the small polynomial tails in INT and FP32.
//
// Methods (constants derived from the mathematics, tables built on the host):
//  * exp:  table-driven reduction (P.T.P. Tang, "Table-driven implementation of
//          the exponential function in IEEE floating-point arithmetic", ACM TOMS
//          15(2), 1989) with 512 table points 2^((j+1/2)/512); the Taylor tail
//          r^3/6 + r^4/24 (|r| <= 7.1e-4) is evaluated in FP32 and folded into
//          the table value by an integer add on its mantissa.  4 FP64 ops.
//  * log:  table-driven reduction (P.T.P. Tang, "Table-driven implementation of
//          the logarithm function in IEEE floating-point arithmetic", ACM TOMS
//          16(4), 1990) with 128 centres c_j = 1 + (j+1/2)/128; Taylor series of
//          ln(1+r), |r| <= 3.9e-3, with the r^4..r^7 terms in FP32.  7 FP64 ops.
//  * rcp:  FP32 reciprocal of the mantissa, two FP64 Newton-Raphson steps
//          y <- y + y(1 - m y), exponent applied by integer arithmetic.  4 FP64 ops.
// Conversions between float, int and double are done on bit patterns (INT pipe).
// Out-of-range arguments take a rarely executed branch to the CUDA math library.
#pragma once

namespace pdm {

#define PDM_INLINE __device__ __forceinline__

constexpr double LN2 = 0.6931471805599453094;              // ln 2 rounded to double
constexpr double EXP_C = 0.0013538030870311431;             // (ln 2)/512 rounded to double
constexpr float EXP_C_LO = 4.5293884e-20f;                  // (ln 2)/512 - EXP_C
constexpr float EXP_K = 738.65985f;                          // 512/ln 2
constexpr int EXP_TAB = 512;                                 // 2^((j+1/2)/512), j < 512
constexpr int LOG_TAB = 128;                                 // pairs (1/c_j, ln c_j)

// double -> float by truncation of the bit pattern (normal doubles; tiny -> 0, huge -> inf)
PDM_INLINE float to_float_trunc(double x) {
  int h = __double2hiint(x);
  unsigned l = (unsigned)__double2loint(x);
  int e = ((h >> 20) & 0x7ff) - 896;
  unsigned s = (unsigned)h & 0x80000000u;
  unsigned bits = s | ((unsigned)e << 23) | (((unsigned)h & 0xfffffu) << 3) | (l >> 29);
  bits = (e <= 0) ? s : bits;
  bits = (e >= 255) ? (s | 0x7f800000u) : bits;
  return __uint_as_float(bits);
}

// float -> double exactly (normal floats and zero; float subnormals map to zero)
PDM_INLINE double to_double(float f) {
  unsigned b = __float_as_uint(f);
  unsigned s = b & 0x80000000u;
  unsigned mag = b & 0x7fffffffu;
  unsigned h = s | ((mag >> 3) + 0x38000000u);
  unsigned l = mag << 29;
  bool z = mag < 0x00800000u;
  return __hiloint2double((int)(z ? s : h), (int)(z ? 0u : l));
}

// k/2 as double for odd k (|k| < 2^31), exactly, by integer arithmetic
PDM_INLINE double half_odd_to_double(int k) {
  unsigned s = (unsigned)k & 0x80000000u;
  unsigned a = k < 0 ? (unsigned)(-k) : (unsigned)k;
  int lz = __clz(a);
  unsigned u = (a << lz) << 1;                 // drop the leading one
  unsigned e = (unsigned)(1023 + 31 - lz - 1); // exponent of a/2
  unsigned h = s | (e << 20) | (u >> 12);
  unsigned l = u << 20;
  return __hiloint2double((int)h, (int)l);
}

// m as double exactly (|m| < 2^31) by integer arithmetic
PDM_INLINE double int_to_double(int m) {
  unsigned s = (unsigned)m & 0x80000000u;
  unsigned a = m < 0 ? (unsigned)(-m) : (unsigned)m;
  int lz = __clz(a);
  unsigned u = (a << (lz & 31)) << 1;
  unsigned e = (unsigned)(1023 + 31 - lz);
  unsigned h = s | (e << 20) | (u >> 12);
  unsigned l = u << 20;
  bool z = a == 0u;
  return __hiloint2double((int)(z ? 0u : h), (int)(z ? 0u : l));
}

__device__ __noinline__ double exp_slow(double x) { return ::exp(x); }
__device__ __noinline__ double log_slow(double x) { return ::log(x); }
__device__ __noinline__ double rcp_slow(double x) { return 1.0 / x; }

// e^x.  tab = 512 doubles 2^((j+1/2)/512) (shared memory).  Max error ~3 ulp.
PDM_INLINE double exp(double x, const double* __restrict__ tab) {
  float xf = to_float_trunc(x);
  float y = fmaf(xf, EXP_K, -0.5f);                         // ~ x*512/ln2 - 1/2
  int m = __float_as_int(y + 12582912.0f) - 0x4B400000;     // round -> ~floor(x*512/ln2)
  if (m < -520000 || m > 520000) return exp_slow(x);        // |x| > ~704: subnormal/overflow
  int k = 2 * m + 1;
  double mh = half_odd_to_double(k);                        // m + 1/2
  double r = fma(-mh, EXP_C, x);                            // FP64 #1   (x - (m+1/2) C_hi)
  float mhf = 0.5f * (__int_as_float(0x4B400000 + k) - 12582912.0f);
  float delta = mhf * EXP_C_LO;                             // (m+1/2) C_lo  (|.| < 1e-14)
  float rf = to_float_trunc(r);
  float tau = rf * rf * rf * fmaf(rf, 1.0f / 24.0f, 1.0f / 6.0f) - delta * (1.0f + rf);
  int j = m & (EXP_TAB - 1);
  int nexp = m >> 9;
  double Tj = tab[j];
  float corr = to_float_trunc(Tj) * tau * 4503599627370496.0f;   // T_j tau 2^52, |.| < 2^20
  int kc = __float_as_int(corr + 12582912.0f) - 0x4B400000;
  double B = __longlong_as_double(__double_as_longlong(Tj) + (long long)kc);  // T_j (1 + tau)
  double q = fma(r, 0.5, 1.0);                              // FP64 #2
  double u = Tj * r;                                        // FP64 #3
  double v = fma(u, q, B);                                  // FP64 #4: T_j e^r
  return __hiloint2double(__double2hiint(v) + (nexp << 20), __double2loint(v));
}

// ln x for positive normal x.  tab = 128 pairs (1/c_j, ln c_j).  Max error ~2 ulp
// (absolute error <= 3e-16 (1 + |exponent|/16)).
PDM_INLINE double log(double x, const double* __restrict__ tab) {
  int h = __double2hiint(x);
  int l = __double2loint(x);
  if (h < 0x00100000 || h >= 0x7ff00000) return log_slow(x);   // <= 0, subnormal, inf, nan
  int e = (h >> 20) - 1023;
  int j = (h >> 13) & (LOG_TAB - 1);
  double m = __hiloint2double((h & 0x000fffff) | 0x3ff00000, l);
  double c = __hiloint2double(0x3ff00000 | (j << 13) | (1 << 12), 0);
  double f = m - c;                                         // FP64 #1 (exact)
  double r = f * tab[2 * j];                                // FP64 #2
  float rf = to_float_trunc(r);
  float s = fmaf(rf, fmaf(rf, fmaf(rf, 1.0f / 7.0f, -1.0f / 6.0f), 0.2f), -0.25f);
  double t = fma(r, to_double(s), 1.0 / 3.0);               // FP64 #3
  t = fma(r, t, -0.5);                                      // FP64 #4
  t = fma(r, t, 1.0);                                       // FP64 #5: ln(1+r) = r t
  double A = fma(int_to_double(e), LN2, tab[2 * j + 1]);    // FP64 #6
  return fma(r, t, A);                                      // FP64 #7
}

// 1/x for positive normal x with 2^-1000 < x < 2^1000.  Max error ~1 ulp.
PDM_INLINE double rcp(double x) {
  int h = __double2hiint(x);
  int l = __double2loint(x);
  int eb = (h >> 20) & 0x7ff;
  if (eb < 24 || eb > 2022 || h < 0) return rcp_slow(x);
  double m = __hiloint2double((h & 0x000fffff) | 0x3ff00000, l);   // [1, 2)
  float mf = __uint_as_float(0x3f800000u | (((unsigned)h & 0xfffffu) << 3) | ((unsigned)l >> 29));
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(mf));
  double y = to_double(yf);
  double t = fma(-m, y, 1.0);                                // FP64 #1
  y = fma(y, t, y);                                          // FP64 #2
  t = fma(-m, y, 1.0);                                       // FP64 #3
  y = fma(y, t, y);                                          // FP64 #4
  int e = eb - 1023;
  return __hiloint2double(__double2hiint(y) - (e << 20), __double2loint(y));
}

// a/b = a * (1/b) for positive normal b
PDM_INLINE double div(double a, double b) { return a * rcp(b); }

// |x| as float, cheap (for tolerance tests off the FP64 pipe)
PDM_INLINE float absf(double x) { return fabsf(to_float_trunc(x)); }

}  // namespace pdm
