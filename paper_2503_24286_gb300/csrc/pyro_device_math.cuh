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
//          15(2), 1989) with 512 table points 2^((j+1/2)/512); the Taylor terms
//          beyond first order, r^2/2 + r^3/6 + r^4/24 (|r| <= 7.1e-4), are formed
//          in FP32 pairs (Dekker products) and folded into the table value by an
//          integer add on its mantissa, so only the reduction and the final
//          T_j r + T_j (1 + s) use the FP64 pipe.  2 FP64 ops, ~75 other
//          instructions.  exp4 keeps 1 + r + r^2/2 in FP64 (4 FP64 ops, ~30
//          other instructions); it is the kernels' default because the
//          straight-line kernels are bounded by instruction fetch as well as by
//          the FP64 pipe once exp grows (measured on the 53-species workload).
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

// float pair (hi, lo) with hi = x truncated to 24 significant bits and lo the
// rest (rounded to float; |lo| < 2^-23 |hi|), by integer arithmetic.
PDM_INLINE void split(double x, float& hi, float& lo) {
  hi = to_float_trunc(x);
  // x - hi: the low 29 mantissa bits of x, scaled; exact in double, rounded to float
  long long bx = __double_as_longlong(x);
  long long rem = bx & 0x1FFFFFFFll;                       // bits below the float's mantissa
  int e = (int)((bx >> 52) & 0x7ff) - 1023 - 52;           // value of mantissa bit 0 is 2^e
  // rem as a float (truncated to 24 bits) by integer normalisation, times 2^e
  unsigned v = (unsigned)rem;
  int lz = __clz(v | 1u);
  unsigned mant = ((v << lz) >> 8) & 0x7fffffu;            // drop the leading one
  int fe = 158 - lz + e;                                    // biased exponent of rem * 2^e
  float r = __uint_as_float(((unsigned)fe << 23) | mant);
  lo = (rem == 0 || fe < 1) ? 0.0f : ((bx < 0) ? -r : r);
}

// e^x.  tab = 512 doubles 2^((j+1/2)/512) (shared memory).  Max error ~2 ulp.
// FP64 pipe: 2 instructions (the reduction and the final fused multiply-add).
PDM_INLINE double exp(double x, const double* __restrict__ tab) {
  float xf = to_float_trunc(x);
  float y = fmaf(xf, EXP_K, -0.5f);                         // ~ x*512/ln2 - 1/2
  int m = __float_as_int(y + 12582912.0f) - 0x4B400000;     // round -> ~floor(x*512/ln2)
  if (m < -520000 || m > 520000) return exp_slow(x);        // |x| > ~704: subnormal/overflow
  int k = 2 * m + 1;
  double mh = half_odd_to_double(k);                        // m + 1/2
  double r = fma(-mh, EXP_C, x);                            // FP64 #1: x - (m+1/2) C_hi, |r| < 7.1e-4
  float mhf = 0.5f * (__int_as_float(0x4B400000 + k) - 12582912.0f);
  float delta = mhf * EXP_C_LO;                             // (m+1/2) C_lo (|.| < 1e-14)
  // s = e^(r - delta) - 1 - r  =  r^2/2 + r^3/6 + r^4/24 - delta (1 + r)   as a float pair
  float rh, rl;
  split(r, rh, rl);
  float p = rh * rh;
  float pe = fmaf(rh, rh, -p);                              // rh^2 = p + pe exactly
  float sh = 0.5f * p;
  float sl = fmaf(0.5f, pe, rh * rl) + p * rh * fmaf(rh, 1.0f / 24.0f, 1.0f / 6.0f) - delta * (1.0f + rh);
  int j = m & (EXP_TAB - 1);
  int nexp = m >> 9;
  double Tj = tab[j];
  float th, tl;
  split(Tj, th, tl);
  // K = round(Tj s 2^52) as a 64-bit integer, |K| < 2^32
  float q = th * sh;
  float qe = fmaf(th, sh, -q);
  float ql = fmaf(th, sl, fmaf(tl, sh, qe));
  float q52 = q * 4503599627370496.0f;                      // exact (power of two), < 2^32
  int qe_b = ((__float_as_int(q52) >> 23) & 0xff) - 127;   // exponent of q52
  long long mq = (long long)((__float_as_int(q52) & 0x7fffff) | 0x800000);
  long long Kh = qe_b >= 23 ? (mq << (qe_b - 23))
                            : (qe_b < 0 ? 0ll : ((mq + (1ll << (22 - qe_b))) >> (23 - qe_b)));
  Kh = (q52 == 0.0f) ? 0ll : (__float_as_int(q52) < 0 ? -Kh : Kh);
  float l52 = ql * 4503599627370496.0f;                     // |.| < 2^10
  int Kl = __float_as_int(l52 + 12582912.0f) - 0x4B400000;
  double B = __longlong_as_double(__double_as_longlong(Tj) + Kh + (long long)Kl);   // Tj (1 + s)
  double v = fma(Tj, r, B);                                 // FP64 #2: Tj e^r
  return __hiloint2double(__double2hiint(v) + (nexp << 20), __double2loint(v));
}

// e^x with 4 FP64 operations (fewer integer/FP32 instructions than exp): the
// tail r^3/6 + r^4/24 in FP32 folded into the table value, 1 + r + r^2/2 in FP64.
PDM_INLINE double exp4(double x, const double* __restrict__ tab) {
  float xf = to_float_trunc(x);
  float y = fmaf(xf, EXP_K, -0.5f);
  int m = __float_as_int(y + 12582912.0f) - 0x4B400000;
  if (m < -520000 || m > 520000) return exp_slow(x);
  int k = 2 * m + 1;
  double mh = half_odd_to_double(k);
  double r = fma(-mh, EXP_C, x);                            // FP64 #1
  float mhf = 0.5f * (__int_as_float(0x4B400000 + k) - 12582912.0f);
  float delta = mhf * EXP_C_LO;
  float rf = to_float_trunc(r);
  float tau = rf * rf * rf * fmaf(rf, 1.0f / 24.0f, 1.0f / 6.0f) - delta * (1.0f + rf);
  int j = m & (EXP_TAB - 1);
  int nexp = m >> 9;
  double Tj = tab[j];
  float corr = to_float_trunc(Tj) * tau * 4503599627370496.0f;
  int kc = __float_as_int(corr + 12582912.0f) - 0x4B400000;
  double B = __longlong_as_double(__double_as_longlong(Tj) + (long long)kc);
  double q = fma(r, 0.5, 1.0);                              // FP64 #2
  double u = Tj * r;                                        // FP64 #3
  double v = fma(u, q, B);                                  // FP64 #4
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
