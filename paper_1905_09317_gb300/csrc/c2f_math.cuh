// c2f_math.cuh -- device elementary functions, Philox4x32-10 and the ROS
// perturbation draw.
//
// Every exp / log / sin / cos on the fire-growth path is computed here from
// IEEE-754 primitives (correctly rounded +, *, /, sqrt and fused multiply-add,
// with no compiler contraction: the library is built with --fmad=false and
// the fused steps are explicit __fma_rn calls), so that a CPU build of the
// same construction reproduces every bit.  Constructions:
//   series forms (dexp_series, dlog_series), which fill the tables below:
//     exp   x = k ln2 + r (Cody-Waite, 29-bit head of ln2), Taylor to r^13, 2^k
//     log   x = 2^e m, m in [sqrt(1/2), sqrt(2)], 2 atanh((m-1)/(m+1)) to s^21
//   table forms (Tang's method), used everywhere else:
//     exp   x = (64k + j) ln2/64 + r: 2^k T_j (1 + p(r)), T_j = 2^(j/64),
//           p = Taylor of exp(r) - 1 to r^5
//     log   x = 2^e m, m in [1, 2), j = top 8 fraction bits, V_j = 1/(1 + j/256)
//           rounded, r = m V_j - 1 (one fused rounding):
//           e ln2 - log V_j + (Taylor of log(1 + r) to r^6)
//   sin/cos of degrees: exact reduction by multiples of 90, Taylor to t^17/t^18
//   pow(x, y) = x^n sqrt(x)^(2y odd) for y a positive multiple of 1/2 up to
//               8 (n = floor y, products from the left), else exp(y log x)
// and the same in binary32 (exp to r^7, log to s^11, cos of a fraction of a
// turn) for the perturbation draw.  Taylor coefficients are 1/k! as correctly
// rounded binary64 quotients; they live in __constant__ memory, filled once per
// device by upload_constants().
#pragma once
#include <cmath>
#include <cstdint>

#include "c2f_layout.cuh"

namespace c2f {

// coefficient tables, filled once per device by upload_constants()
__constant__ MathConstants g_mc;
// exp / log tables (lanes index them independently, so global memory through
// the read-only cache rather than __constant__), filled by k_math_tables
__device__ double g_exp_tab[64];    // 2^(j/64)
__device__ double g_log_inv[256];   // RN(1 / (1 + j/256))
__device__ double g_log_tab[256];   // -log(g_log_inv[j])

// host: compute the coefficient tables (plain IEEE binary64 arithmetic)
inline void make_math_constants(MathConstants *m) {
  double f = 1.0;
  for (int k = 0; k < 24; ++k) {
    if (k > 0) f = f * (double)k;
    m->inv_fact[k] = 1.0 / f;
  }
  for (int n = 0; n < 12; ++n) m->log_c[n] = 1.0 / (double)(2 * n + 1);
  for (int n = 0; n < 10; ++n) {
    const double sgn = (n & 1) ? -1.0 : 1.0;
    m->sin_c[n] = sgn * m->inv_fact[2 * n + 1];
    m->cos_c[n] = sgn * m->inv_fact[2 * n];
  }
  for (int k = 0; k < 12; ++k) m->inv_fact_f[k] = (float)m->inv_fact[k];
  for (int n = 0; n < 8; ++n) m->log_cf[n] = (float)m->log_c[n];
  for (int n = 0; n < 8; ++n) {
    m->sin_cf[n] = (float)m->sin_c[n];
    m->cos_cf[n] = (float)m->cos_c[n];
  }
}

constexpr double kLn2Hi = 0x1.62e42ffp-1;            // 29 significant bits
constexpr double kLn2Lo = -0x1.718432a1b0e26p-35;    // ln2 - kLn2Hi, rounded
constexpr double kInvLn2 = 0x1.71547652b82fep+0;
constexpr double kDeg2Rad = 0x1.1df46a2529d39p-6;
constexpr double kSqrt2 = 0x1.6a09e667f3bcdp+0;
constexpr float kLn2HiF = 0x1.62ep-1f;               // 13 significant bits
constexpr float kLn2LoF = 0x1.0bfbe8p-15f;
constexpr float kInvLn2F = 0x1.715476p+0f;
constexpr float kTwoPiF = 0x1.921fb6p+2f;
constexpr float kSqrt2F = 0x1.6a09e6p+0f;

// Comparisons of a double with 0 or a positive constant as integer compares of
// the bit patterns (the order of non-NaN doubles against a positive constant is
// the order of their bits read as signed 64-bit integers).  The values tested
// on the rate-of-spread path are never NaN; these keep the compares off the
// FP64 unit, which the table kernel saturates.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool pos(double x) { return dbits(x) > 0; }   // x > 0
__device__ __forceinline__ bool gt_c(double x, double c) { return dbits(x) > dbits(c); }   // x > c > 0
__device__ __forceinline__ bool lt_c(double x, double c) { return dbits(x) < dbits(c); }   // x < c, c > 0
__device__ __forceinline__ bool le_c(double x, double c) { return dbits(x) <= dbits(c); }  // x <= c, c > 0

__device__ __forceinline__ double pow2i(int k) {  // exact 2^k for -1022 <= k <= 1023
  return __longlong_as_double((long long)(k + 1023) << 52);
}

__device__ __forceinline__ double scale2(double p, int k) {
  if (k > 1023) return __dmul_rn(__dmul_rn(p, pow2i(1023)), pow2i(k - 1023));
  if (k < -1022) return __dmul_rn(__dmul_rn(p, pow2i(k + 600)), pow2i(-600));
  return __dmul_rn(p, pow2i(k));
}

__device__ inline double dexp_series(double x) {
  // |x| < 704 (integer test of the high word) skips the range checks below
  if ((__double2hiint(x) & 0x7fffffff) >= 0x40860000) {
    if (x != x) return x;
    if (x > 709.78) return __longlong_as_double(0x7ff0000000000000LL);
    if (x < -745.2) return 0.0;
  }
  const double kd = rint(__dmul_rn(x, kInvLn2));
  const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(kd, kLn2Hi)), __dmul_rn(kd, kLn2Lo));
  double p = g_mc.inv_fact[13];
#pragma unroll
  for (int i = 12; i >= 0; --i) p = __fma_rn(p, r, g_mc.inv_fact[i]);
  return scale2(p, (int)kd);
}

__device__ inline double dlog_series(double x) {
  int e = 0;
  const int hx = __double2hiint(x);
  if (hx < 0x00100000 || hx >= 0x7ff00000) {   // not a positive normal finite number
    if (x != x) return x;
    if (x < 0.0) return __longlong_as_double(0x7ff8000000000000LL);
    if (x == 0.0) return __longlong_as_double((long long)0xfff0000000000000ULL);
    if (__double_as_longlong(x) == 0x7ff0000000000000LL) return x;
    if (x < 0x1p-1022) { x = __dmul_rn(x, 0x1p54); e = -54; }
  }
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  e += (int)((b >> 52) & 0x7ff) - 1023;
  b = (b & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;
  double m = __longlong_as_double((long long)b);
  if (m > kSqrt2) { m = __dmul_rn(m, 0.5); e += 1; }
  const double f = __dsub_rn(m, 1.0);
  const double s = __ddiv_rn(f, __dadd_rn(2.0, f));
  const double z = __dmul_rn(s, s);
  double q = g_mc.log_c[10];
#pragma unroll
  for (int n = 9; n >= 1; --n) q = __fma_rn(q, z, g_mc.log_c[n]);
  const double s2 = __dadd_rn(s, s);
  const double lm = __fma_rn(__dmul_rn(s2, z), q, s2);
  const double ed = (double)e;
  return __dadd_rn(__dmul_rn(ed, kLn2Hi), __fma_rn(ed, kLn2Lo, lm));
}

__device__ inline double dexp(double x) {
  if ((__double2hiint(x) & 0x7fffffff) >= 0x40860000) {   // |x| >= 704
    if (x != x) return x;
    if (x > 709.78) return __longlong_as_double(0x7ff0000000000000LL);
    if (x < -745.2) return 0.0;
  }
  const double kd = rint(__dmul_rn(x, kInvLn2 * 64.0));
  const double r = __fma_rn(-kd, kLn2Lo / 64.0, __fma_rn(-kd, kLn2Hi / 64.0, x));
  double q = __fma_rn(__fma_rn(g_mc.inv_fact[5], r, g_mc.inv_fact[4]), r, g_mc.inv_fact[3]);
  q = __fma_rn(q, r, g_mc.inv_fact[2]);
  const double p = __fma_rn(q, __dmul_rn(r, r), r);   // exp(r) - 1 to r^5
  const long long k = (long long)kd;
  const double t = __ldg(&g_exp_tab[k & 63]);
  const double y = __fma_rn(t, p, t);                  // in [2^(-1/128), 2)
  const int m = (int)(k >> 6);
  // y 2^m is exact while it stays normal: add m to the exponent field
  if (m >= -1020 && m <= 1022) return __longlong_as_double(__double_as_longlong(y) + ((long long)m << 52));
  return scale2(y, m);
}

__device__ inline double dlog(double x) {
  int e = 0;
  const int hx = __double2hiint(x);
  if (hx < 0x00100000 || hx >= 0x7ff00000) {   // not a positive normal finite number
    if (x != x) return x;
    if (x < 0.0) return __longlong_as_double(0x7ff8000000000000LL);
    if (x == 0.0) return __longlong_as_double((long long)0xfff0000000000000ULL);
    if (__double_as_longlong(x) == 0x7ff0000000000000LL) return x;
    if (x < 0x1p-1022) { x = __dmul_rn(x, 0x1p54); e = -54; }
  }
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  e += (int)((b >> 52) & 0x7ff) - 1023;
  const int j = (int)((b >> 44) & 255);
  b = (b & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;
  const double m = __longlong_as_double((long long)b);
  const double r = __fma_rn(m, __ldg(&g_log_inv[j]), -1.0);
  // log(1 + r) = r - r^2/2 + r^3/3 - ... - r^6/6
  double q = -g_mc.inv_fact[3];             // -1/6
  q = __fma_rn(q, r, g_mc.log_c[2]);        // 1/5
  q = __fma_rn(q, r, -0.25);
  q = __fma_rn(q, r, g_mc.log_c[1]);        // 1/3
  q = __fma_rn(q, r, -0.5);
  const double lp = __fma_rn(q, __dmul_rn(r, r), r);
  const double ed = (double)e;
  const double hi = __dadd_rn(__dmul_rn(ed, kLn2Hi), __ldg(&g_log_tab[j]));
  const double lo = __fma_rn(ed, kLn2Lo, lp);
  return __dadd_rn(hi, lo);
}

__device__ inline double dpow(double x, double y) {
  if (x > 0.0) {
    const double y2 = __dadd_rn(y, y);
    if (y > 0.0 && y2 <= 16.0 && rint(y2) == y2) {   // y = n or n + 1/2, n <= 8
      const int n = (int)y;
      double r = 1.0;
      if (n > 0) {
        r = x;
        for (int i = 1; i < n; ++i) r = __dmul_rn(r, x);
      }
      if (((int)y2) & 1) r = (n > 0) ? __dmul_rn(r, __dsqrt_rn(x)) : __dsqrt_rn(x);
      return r;
    }
    return dexp(__dmul_rn(y, dlog(x)));
  }
  if (x == 0.0) return (y > 0.0) ? 0.0 : ((y == 0.0) ? 1.0 : __longlong_as_double(0x7ff0000000000000LL));
  return __longlong_as_double(0x7ff8000000000000LL);
}

// dpow with the exponent's kind decided ahead: n2 = 2y when y is a positive
// multiple of 1/2 up to 8 (the case dpow treats with products and a square
// root), else 0 -- the same results as dpow(x, y) without testing y
__device__ inline double dpow_n2(double x, double y, int n2) {
  if (pos(x)) {
    if (n2 > 0) {
      const int n = n2 >> 1;
      double r = 1.0;
      if (n > 0) {
        r = x;
        for (int i = 1; i < n; ++i) r = __dmul_rn(r, x);
      }
      if (n2 & 1) r = (n > 0) ? __dmul_rn(r, __dsqrt_rn(x)) : __dsqrt_rn(x);
      return r;
    }
    return dexp(__dmul_rn(y, dlog(x)));
  }
  if (x == 0.0) return (y > 0.0) ? 0.0 : ((y == 0.0) ? 1.0 : __longlong_as_double(0x7ff0000000000000LL));
  return __longlong_as_double(0x7ff8000000000000LL);
}

// host: n2 of dpow_n2 for a constant exponent
inline int pow_half_steps(double y) {
  const double y2 = y + y;
  return (y > 0.0 && y2 <= 16.0 && std::nearbyint(y2) == y2) ? (int)y2 : 0;
}

// fills g_exp_tab / g_log_inv / g_log_tab with the series forms (one block of 256)
__global__ void k_math_tables() {
  const int j = threadIdx.x;
  if (j < 64)
    g_exp_tab[j] = dexp_series(__dadd_rn(__dmul_rn((double)j, kLn2Hi / 64.0), __dmul_rn((double)j, kLn2Lo / 64.0)));
  if (j < 256) {
    const double v = __ddiv_rn(1.0, __dadd_rn(1.0, __ddiv_rn((double)j, 256.0)));
    g_log_inv[j] = v;
    g_log_tab[j] = -dlog_series(v);
  }
}

__device__ inline void dsincos_deg(double x, double *s_out, double *c_out) {
  const double qd = rint(__ddiv_rn(x, 90.0));
  const double r = __dsub_rn(x, __dmul_rn(qd, 90.0));
  const double t = __dmul_rn(r, kDeg2Rad);
  const double t2 = __dmul_rn(t, t);
  double ps = g_mc.sin_c[8];
#pragma unroll
  for (int n = 7; n >= 1; --n) ps = __fma_rn(ps, t2, g_mc.sin_c[n]);
  const double sn = __fma_rn(__dmul_rn(t, t2), ps, t);
  double pc = g_mc.cos_c[9];
#pragma unroll
  for (int n = 8; n >= 1; --n) pc = __fma_rn(pc, t2, g_mc.cos_c[n]);
  const double cs = __fma_rn(t2, pc, 1.0);
  const long long qi = (long long)qd;
  const int q = (int)(((qi % 4) + 4) % 4);
  double s, c;
  if (q == 0) { s = sn; c = cs; }
  else if (q == 1) { s = cs; c = -sn; }
  else if (q == 2) { s = -sn; c = -cs; }
  else { s = -cs; c = sn; }
  *s_out = s;
  *c_out = c;
}

// ---------------------------------------------------------------- binary32
__device__ __forceinline__ float pow2if(int k) {  // exact 2^k, -126 <= k <= 127
  return __int_as_float((k + 127) << 23);
}

__device__ __forceinline__ float scale2f(float p, int k) {
  if (k > 127) return __fmul_rn(__fmul_rn(p, pow2if(127)), pow2if(k - 127));
  if (k < -126) return __fmul_rn(__fmul_rn(p, pow2if(k + 64)), pow2if(-64));
  return __fmul_rn(p, pow2if(k));
}

__device__ inline float fexp(float x) {
  if (x != x) return x;
  if (x > 88.72f) return __int_as_float(0x7f800000);
  if (x < -103.9f) return 0.0f;
  const float kf = rintf(__fmul_rn(x, kInvLn2F));
  const float r = __fsub_rn(__fsub_rn(x, __fmul_rn(kf, kLn2HiF)), __fmul_rn(kf, kLn2LoF));
  float p = g_mc.inv_fact_f[7];
#pragma unroll
  for (int i = 6; i >= 0; --i) p = __fmaf_rn(p, r, g_mc.inv_fact_f[i]);
  return scale2f(p, (int)kf);
}

__device__ inline float flog(float x) {
  if (x != x) return x;
  if (x < 0.0f) return __int_as_float(0x7fc00000);
  if (x == 0.0f) return __int_as_float((int)0xff800000u);
  if (__float_as_int(x) == 0x7f800000) return x;
  int e = 0;
  if (x < 0x1p-126f) { x = __fmul_rn(x, 0x1p24f); e = -24; }
  unsigned int b = (unsigned int)__float_as_int(x);
  e += (int)((b >> 23) & 0xff) - 127;
  b = (b & 0x007fffffu) | 0x3f800000u;
  float m = __int_as_float((int)b);
  if (m > kSqrt2F) { m = __fmul_rn(m, 0.5f); e += 1; }
  const float f = __fsub_rn(m, 1.0f);
  const float s = __fdiv_rn(f, __fadd_rn(2.0f, f));
  const float z = __fmul_rn(s, s);
  float q = g_mc.log_cf[5];
#pragma unroll
  for (int n = 4; n >= 1; --n) q = __fmaf_rn(q, z, g_mc.log_cf[n]);
  const float s2 = __fadd_rn(s, s);
  const float lm = __fmaf_rn(__fmul_rn(s2, z), q, s2);
  const float ef = (float)e;
  return __fadd_rn(__fmul_rn(ef, kLn2HiF), __fmaf_rn(ef, kLn2LoF, lm));
}

// flog for u in [2^-25, 1) and fexp for |x| < 64 ln 2: the same arithmetic
// without the special-value branches (NaN, sign, zero, infinity, subnormal,
// overflow, underflow) that such arguments never take; the perturbation's
// draws always lie in these ranges
__device__ __forceinline__ float flog_unit(float x) {
  const unsigned int b0 = (unsigned int)__float_as_int(x);
  int e = (int)((b0 >> 23) & 0xff) - 127;
  float m = __int_as_float((int)((b0 & 0x007fffffu) | 0x3f800000u));
  if (m > kSqrt2F) { m = __fmul_rn(m, 0.5f); e += 1; }
  const float f = __fsub_rn(m, 1.0f);
  const float s = __fdiv_rn(f, __fadd_rn(2.0f, f));
  const float z = __fmul_rn(s, s);
  float q = g_mc.log_cf[5];
#pragma unroll
  for (int n = 4; n >= 1; --n) q = __fmaf_rn(q, z, g_mc.log_cf[n]);
  const float s2 = __fadd_rn(s, s);
  const float lm = __fmaf_rn(__fmul_rn(s2, z), q, s2);
  const float ef = (float)e;
  return __fadd_rn(__fmul_rn(ef, kLn2HiF), __fmaf_rn(ef, kLn2LoF, lm));
}

__device__ __forceinline__ float fexp_small(float x) {
  const float kf = rintf(__fmul_rn(x, kInvLn2F));
  const float r = __fsub_rn(__fsub_rn(x, __fmul_rn(kf, kLn2HiF)), __fmul_rn(kf, kLn2LoF));
  float p = g_mc.inv_fact_f[7];
#pragma unroll
  for (int i = 6; i >= 0; --i) p = __fmaf_rn(p, r, g_mc.inv_fact_f[i]);
  return __fmul_rn(p, pow2if((int)kf));
}

// cos(2 pi u)
__device__ inline float fcos_turns(float u) {
  const float qf = rintf(__fmul_rn(u, 4.0f));
  const float r = __fsub_rn(u, __fmul_rn(qf, 0.25f));
  const float t = __fmul_rn(r, kTwoPiF);
  const float t2 = __fmul_rn(t, t);
  float ps = g_mc.sin_cf[4];
#pragma unroll
  for (int n = 3; n >= 1; --n) ps = __fmaf_rn(ps, t2, g_mc.sin_cf[n]);
  const float sn = __fmaf_rn(__fmul_rn(t, t2), ps, t);
  float pc = g_mc.cos_cf[5];
#pragma unroll
  for (int n = 4; n >= 1; --n) pc = __fmaf_rn(pc, t2, g_mc.cos_cf[n]);
  const float cs = __fmaf_rn(t2, pc, 1.0f);
  const int q = ((((int)qf) % 4) + 4) % 4;
  if (q == 0) return cs;
  if (q == 1) return -sn;
  if (q == 2) return -cs;
  return sn;
}

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds, Weyl key schedule.
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

// Multiplicative ROS perturbation of (replica, cell, hour): f = exp(sigma z),
// z ~ N(0,1) by Box-Muller from the Philox block at counter
// (replica, cell, hour, 0) under the run key; binary32; sigma == 0 -> 1.
__device__ inline float noise_factor(uint64_t seed, uint32_t replica, uint32_t cell,
                                     uint32_t hour, float sigma) {
  if (sigma == 0.0f) return 1.0f;
  const U4 x = philox4x32_10(U4{replica, cell, hour, 0u}, (uint32_t)seed,
                             (uint32_t)(seed >> 32));
  const float u1 = __fmul_rn(__fadd_rn((float)(x.x >> 8), 0.5f), 0x1p-24f);
  const float u2 = __fmul_rn(__fadd_rn((float)(x.y >> 8), 0.5f), 0x1p-24f);
  // u1 >= 2^-25, so |z| <= sqrt(50 ln 2) < 6 and |sigma z| < 6 for sigma <= 1
  const float z = __fmul_rn(__fsqrt_rn(__fmul_rn(-2.0f, flog_unit(u1))), fcos_turns(u2));
  return fexp_small(__fmul_rn(sigma, z));
}

// the perturbation as a 32.32 fixed-point multiplier f 2^32: exact, since
// f >= 2^-9 has a binary32 significand whose scaled value is an integer.  Built
// from the bits (significand shifted by the exponent) rather than by a
// float-to-int64 conversion, which is slow on this GPU.
__device__ __forceinline__ uint64_t noise_fixed(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint64_t m = (uint64_t)((b & 0x7FFFFFu) | 0x800000u);
  return m << ((int)(b >> 23) - 118);   // 2^(e - 127 - 23 + 32), e >= 118 for f >= 2^-9
}

// per-period increment (base * F + 2^31) >> 32, capped at the axis length
__device__ __forceinline__ int64_t apply_noise(int64_t base, uint64_t F, int64_t dk) {
  const uint64_t b = (uint64_t)base;
  uint64_t lo = b * F;
  uint64_t hi = __umul64hi(b, F);
  const uint64_t lo2 = lo + 0x80000000ULL;
  hi += (lo2 < lo) ? 1ULL : 0ULL;
  // inc = (hi:lo2) >> 32
  if (hi >> 32) return dk;
  const uint64_t inc = (hi << 32) | (lo2 >> 32);
  return inc > (uint64_t)dk ? dk : (int64_t)inc;
}

}  // namespace c2f
