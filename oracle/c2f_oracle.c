/*
 * c2f_oracle.c -- CPU oracle for the Cell2Fire Monte-Carlo fire-growth path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * restatement of the method that the GPU library is checked against.  Only
 * the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no source with the CUDA library: its elementary
 * functions, its Philox generator, its FBP coefficient table and its step
 * loop are all written here, from the paper and the published definitions.
 *
 * Paper: Pais et al., "Cell2Fire: A Cell Based Forest Fire Growth Model"
 * (arXiv:1905.09317).  Citations below name the section / equation /
 * algorithm of that paper.
 *
 *   Sec. 3.1, 3.3   cell states (Available, Burning, Burned, Harvested,
 *                   Non-Fuel), 8 neighbours, centre-to-centre spread,
 *                   message when progress reaches the neighbour's centre,
 *                   ignition when the receiver's ROS exceeds a threshold.
 *   Sec. 3.2 (A5)   cell burn-out: no Available neighbour (ii), or ROS
 *                   below a threshold delta (i).
 *   Sec. 3.4, Alg. 1  Step 0 init, Step 1 ignition, Step 2 send/receive
 *                   repeated per fire period until TMax.
 *   Sec. 3.7, Eqs. 2-4  ellipse a = (HROS+BROS)/2, b = FROS,
 *                   FROS = (HROS+BROS)/(2 LB), eccentricity e.
 *   Sec. 2.2, Eq. 1 directional ROS a(1-e^2)/(1-e cos phi) on the forward
 *                   half, a(1-e^2) on the back half.
 *   Sec. 3.8 / App. A  send before receive within a step.
 *   Sec. 3.1 (uncertainty (1),(2))  random ignition cell, multiplicative
 *                   ROS perturbation.
 *   Sec. 3.1 (uncertainty (3))  several weather scenarios with given
 *                   probabilities; each replica runs under one of them.
 *
 * FBP rate-of-spread equations are not printed in the paper (it defers to
 * the Canadian FBP System, Forestry Canada 1992, and the 2009 update); the
 * surface-spread subset used here is the published standard form, restated.
 * Parity against that publication is unpinned (no worked example is
 * available); property pins are in the tests.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_API __attribute__((visibility("default")))

/* ======================================================================
 * 1. binary64 elementary functions (own implementation)
 *    Series forms (exp_series, log_series), used to fill the tables below:
 *    exp: Cody-Waite reduction x = k ln2 + r, |r| <= ln2/2, Taylor series
 *         of degree 13 by Horner with fused multiply-add, then scale by 2^k.
 *    log: x = 2^e m, m in [sqrt(1/2), sqrt(2)], log m = 2 atanh(s),
 *         s = (m-1)/(m+1), odd series to s^21.
 *    Table forms, the ones the method uses (Tang's table-driven method):
 *    exp: x = (64 k + j) ln2/64 + r, |r| <= ln2/128 (r by two fused steps):
 *         exp x = 2^k T_j (1 + p(r)), T_j = 2^(j/64) (exp_series), p the
 *         Taylor polynomial of exp(r) - 1 to r^5.
 *    log: x = 2^e m, m in [1, 2), j = first 8 fraction bits of m,
 *         V_j = RN(1 / (1 + j/256)), r = m V_j - 1 (one fused rounding):
 *         log x = e ln2 - log V_j + log(1 + r), log V_j by log_series,
 *         log(1 + r) by its Taylor polynomial to r^6 (|r| < 1/256).
 *    sincos in degrees: quadrant reduction by exact subtraction of a
 *         multiple of 90, Taylor series of sin (to t^17) and cos (to t^18).
 *    pow(x,y), x > 0: for y a positive multiple of 1/2 up to 8,
 *         x^n (n = floor y, n-1 products from the left) times sqrt(x) when
 *         2y is odd; otherwise exp(y log x).
 * The constants are ln 2 split into a 29-bit head and a tail, 1/ln 2 and
 * pi/180, each the double nearest to the real number; Taylor coefficients
 * are 1/k! computed as a correctly rounded division.
 * ====================================================================== */
static const double LN2_HI = 0x1.62e42ffp-1;
static const double LN2_LO = -0x1.718432a1b0e26p-35;
static const double INV_LN2 = 0x1.71547652b82fep+0;
static const double DEG2RAD = 0x1.1df46a2529d39p-6;
static const double SQRT2_D = 0x1.6a09e667f3bcdp+0;

static double g_inv_fact[24];  /* 1/k!            */
static double g_log_c[12];     /* 1/(2n+1)        */
static double g_sin_c[10];     /* (-1)^n/(2n+1)!  */
static double g_cos_c[10];     /* (-1)^n/(2n)!    */
static double g_exp_tab[64];   /* 2^(j/64)               */
static double g_log_inv[256];  /* RN(1 / (1 + j/256))    */
static double g_log_tab[256];  /* -log(g_log_inv[j])     */
static double g_log_c3, g_log_c4, g_log_c5, g_log_c6;   /* 1/n */
static float g_inv_fact_f[12];
static float g_log_cf[8];
static float g_sin_cf[8];
static float g_cos_cf[8];
static int g_init = 0;

static void fill_fn_tables(void);

static void or_init_tables(void) {
  if (g_init) return;
  double f = 1.0;  /* k! exactly (k <= 20 fits in 2^63; <= 18 is exact in binary64) */
  for (int k = 0; k < 24; ++k) {
    if (k > 0) f = f * (double)k;
    g_inv_fact[k] = 1.0 / f;
  }
  for (int n = 0; n < 12; ++n) g_log_c[n] = 1.0 / (double)(2 * n + 1);
  for (int n = 0; n < 10; ++n) {
    double s = (n % 2) ? -1.0 : 1.0;
    g_sin_c[n] = s * g_inv_fact[2 * n + 1];
    g_cos_c[n] = s * g_inv_fact[2 * n];
  }
  /* binary32 coefficients: the binary64 coefficient rounded once to
   * binary32 (the accuracy of the resulting functions is pinned in the
   * tests against high-precision references). */
  for (int k = 0; k < 12; ++k) g_inv_fact_f[k] = (float)g_inv_fact[k];
  for (int n = 0; n < 8; ++n) g_log_cf[n] = (float)g_log_c[n];
  for (int n = 0; n < 8; ++n) {
    g_sin_cf[n] = (float)g_sin_c[n];
    g_cos_cf[n] = (float)g_cos_c[n];
  }
  g_log_c3 = 1.0 / 3.0; g_log_c4 = 1.0 / 4.0; g_log_c5 = 1.0 / 5.0;
  g_log_c6 = 1.0 / 6.0;
  g_init = 1;
  fill_fn_tables();
}

static double pow2i(int k) { /* exact 2^k, -1022 <= k <= 1023 */
  uint64_t b = (uint64_t)(k + 1023) << 52;
  double d;
  memcpy(&d, &b, 8);
  return d;
}

static double scale2(double p, int k) {
  if (k > 1023) return (p * pow2i(1023)) * pow2i(k - 1023);
  if (k < -1022) return (p * pow2i(k + 600)) * pow2i(-600);
  return p * pow2i(k);
}

static double exp_series(double x) {
  if (x != x) return x;
  if (x > 709.78) return INFINITY;
  if (x < -745.2) return 0.0;
  double kd = nearbyint(x * INV_LN2);
  double r = (x - kd * LN2_HI) - kd * LN2_LO;
  double p = g_inv_fact[13];
  for (int i = 12; i >= 0; --i) p = fma(p, r, g_inv_fact[i]);
  return scale2(p, (int)kd);
}

static double log_series(double x) {
  if (x != x) return x;
  if (x < 0.0) return NAN;
  if (x == 0.0) return -INFINITY;
  if (isinf(x)) return x;
  int e = 0;
  if (x < 0x1p-1022) { x = x * 0x1p54; e = -54; }
  uint64_t b;
  memcpy(&b, &x, 8);
  e += (int)((b >> 52) & 0x7ff) - 1023;
  b = (b & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;
  double m;
  memcpy(&m, &b, 8);
  if (m > SQRT2_D) { m = m * 0.5; e += 1; }
  double f = m - 1.0;
  double s = f / (2.0 + f);
  double z = s * s;
  double q = g_log_c[10];
  for (int n = 9; n >= 1; --n) q = fma(q, z, g_log_c[n]);
  double s2 = s + s;
  double lm = fma(s2 * z, q, s2);
  double ed = (double)e;
  return ed * LN2_HI + fma(ed, LN2_LO, lm);
}

static void fill_fn_tables(void) {
  for (int j = 0; j < 64; ++j) g_exp_tab[j] = exp_series((double)j * (LN2_HI / 64.0) + (double)j * (LN2_LO / 64.0));
  for (int j = 0; j < 256; ++j) {
    g_log_inv[j] = 1.0 / (1.0 + (double)j / 256.0);
    g_log_tab[j] = -log_series(g_log_inv[j]);
  }
}

OR_API double or_exp(double x) {
  or_init_tables();
  if (x != x) return x;
  if (x > 709.78) return INFINITY;
  if (x < -745.2) return 0.0;
  double kd = nearbyint(x * (INV_LN2 * 64.0));
  double r = fma(-kd, LN2_LO / 64.0, fma(-kd, LN2_HI / 64.0, x));
  double q = fma(fma(g_inv_fact[5], r, g_inv_fact[4]), r, g_inv_fact[3]);
  q = fma(q, r, g_inv_fact[2]);
  double p = fma(q, r * r, r);          /* exp(r) - 1 to r^5 */
  long long k = (long long)kd;
  double t = g_exp_tab[k & 63];
  return scale2(fma(t, p, t), (int)(k >> 6));
}

OR_API double or_log(double x) {
  or_init_tables();
  if (x != x) return x;
  if (x < 0.0) return NAN;
  if (x == 0.0) return -INFINITY;
  if (isinf(x)) return x;
  int e = 0;
  if (x < 0x1p-1022) { x = x * 0x1p54; e = -54; }
  uint64_t b;
  memcpy(&b, &x, 8);
  e += (int)((b >> 52) & 0x7ff) - 1023;
  int j = (int)((b >> 44) & 255);
  b = (b & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;
  double m;
  memcpy(&m, &b, 8);
  double r = fma(m, g_log_inv[j], -1.0);
  /* log(1 + r) = r - r^2/2 + r^3/3 - ... - r^6/6 */
  double q = -g_log_c6;
  q = fma(q, r, g_log_c5);
  q = fma(q, r, -g_log_c4);
  q = fma(q, r, g_log_c3);
  q = fma(q, r, -0.5);
  double lp = fma(q, r * r, r);
  double ed = (double)e;
  double hi = ed * LN2_HI + g_log_tab[j];
  double lo = fma(ed, LN2_LO, lp);
  return hi + lo;
}

OR_API double or_pow(double x, double y) {
  if (x > 0.0) {
    double y2 = y + y;
    if (y > 0.0 && y2 <= 16.0 && nearbyint(y2) == y2) {   /* y = n or n + 1/2, n <= 8 */
      int n = (int)y;
      double r = 1.0;
      if (n > 0) {
        r = x;
        for (int i = 1; i < n; ++i) r = r * x;
      }
      if (((int)y2) & 1) r = (n > 0) ? r * sqrt(x) : sqrt(x);
      return r;
    }
    return or_exp(y * or_log(x));
  }
  if (x == 0.0) return (y > 0.0) ? 0.0 : ((y == 0.0) ? 1.0 : INFINITY);
  return NAN;
}

OR_API void or_sincos_deg(double x, double *s_out, double *c_out) {
  or_init_tables();
  double qd = nearbyint(x / 90.0);
  double r = x - qd * 90.0;
  double t = r * DEG2RAD;
  double t2 = t * t;
  double ps = g_sin_c[8];
  for (int n = 7; n >= 1; --n) ps = fma(ps, t2, g_sin_c[n]);
  double sn = fma(t * t2, ps, t);
  double pc = g_cos_c[9];
  for (int n = 8; n >= 1; --n) pc = fma(pc, t2, g_cos_c[n]);
  double cs = fma(t2, pc, 1.0);
  long long qi = (long long)qd;
  int q = (int)(((qi % 4) + 4) % 4);
  double s, c;
  switch (q) {
    case 0: s = sn; c = cs; break;
    case 1: s = cs; c = -sn; break;
    case 2: s = -sn; c = -cs; break;
    default: s = -cs; c = sn; break;
  }
  *s_out = s;
  *c_out = c;
}

/* ======================================================================
 * 2. binary32 functions for the ROS perturbation draw
 *    same constructions in single precision: exp (degree 7), log (odd
 *    series to s^11) and cos(2 pi u) of a fraction of a turn.
 * ====================================================================== */
static const float LN2_HI_F = 0x1.62ep-1f;
static const float LN2_LO_F = 0x1.0bfbe8p-15f;
static const float INV_LN2_F = 0x1.715476p+0f;
static const float TWO_PI_F = 0x1.921fb6p+2f;
static const float SQRT2_F = 0x1.6a09e6p+0f;

static float pow2if(int k) { /* exact 2^k, -126 <= k <= 127 */
  uint32_t b = (uint32_t)(k + 127) << 23;
  float f;
  memcpy(&f, &b, 4);
  return f;
}

static float scale2f(float p, int k) {
  if (k > 127) return (p * pow2if(127)) * pow2if(k - 127);
  if (k < -126) return (p * pow2if(k + 64)) * pow2if(-64);
  return p * pow2if(k);
}

OR_API float or_expf(float x) {
  or_init_tables();
  if (x != x) return x;
  if (x > 88.72f) return INFINITY;
  if (x < -103.9f) return 0.0f;
  float kf = nearbyintf(x * INV_LN2_F);
  float r = (x - kf * LN2_HI_F) - kf * LN2_LO_F;
  float p = g_inv_fact_f[7];
  for (int i = 6; i >= 0; --i) p = fmaf(p, r, g_inv_fact_f[i]);
  return scale2f(p, (int)kf);
}

OR_API float or_logf(float x) {
  or_init_tables();
  if (x != x) return x;
  if (x < 0.0f) return NAN;
  if (x == 0.0f) return -INFINITY;
  if (isinf(x)) return x;
  int e = 0;
  if (x < 0x1p-126f) { x = x * 0x1p24f; e = -24; }
  uint32_t b;
  memcpy(&b, &x, 4);
  e += (int)((b >> 23) & 0xff) - 127;
  b = (b & 0x007fffffu) | 0x3f800000u;
  float m;
  memcpy(&m, &b, 4);
  if (m > SQRT2_F) { m = m * 0.5f; e += 1; }
  float f = m - 1.0f;
  float s = f / (2.0f + f);
  float z = s * s;
  float q = g_log_cf[5];
  for (int n = 4; n >= 1; --n) q = fmaf(q, z, g_log_cf[n]);
  float s2 = s + s;
  float lm = fmaf(s2 * z, q, s2);
  float ef = (float)e;
  return ef * LN2_HI_F + fmaf(ef, LN2_LO_F, lm);
}

/* cos(2 pi u) */
OR_API float or_cos_turnsf(float u) {
  or_init_tables();
  float qf = nearbyintf(u * 4.0f);
  float r = u - qf * 0.25f;
  float t = r * TWO_PI_F;
  float t2 = t * t;
  float ps = g_sin_cf[4];
  for (int n = 3; n >= 1; --n) ps = fmaf(ps, t2, g_sin_cf[n]);
  float sn = fmaf(t * t2, ps, t);
  float pc = g_cos_cf[5];
  for (int n = 4; n >= 1; --n) pc = fmaf(pc, t2, g_cos_cf[n]);
  float cs = fmaf(t2, pc, 1.0f);
  int q = (((int)qf % 4) + 4) % 4;
  switch (q) {
    case 0: return cs;
    case 1: return -sn;
    case 2: return -cs;
    default: return sn;
  }
}

/* ======================================================================
 * 3. Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
 *    32x32->64 multiplies with the Weyl key schedule.
 * ====================================================================== */
OR_API void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                             uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Multiplicative ROS perturbation f = exp(sigma z), z standard normal by
 * Box-Muller from one Philox block keyed by the run seed at counter
 * (replica, cell, hour, 0) -- uncertainty source (2) of Sec. 3.1.  The
 * draw is made in binary32; sigma == 0 gives f = 1 with no draw. */
OR_API float or_noise_factor(uint64_t seed, uint32_t replica, uint32_t cell,
                             uint32_t hour, float sigma) {
  if (sigma == 0.0f) return 1.0f;
  uint32_t ctr[4] = {replica, cell, hour, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  or_philox4x32_10(ctr, key, x);
  float u1 = ((float)(x[0] >> 8) + 0.5f) * 0x1p-24f;
  float u2 = ((float)(x[1] >> 8) + 0.5f) * 0x1p-24f;
  float z = sqrtf(-2.0f * or_logf(u1)) * or_cos_turnsf(u2);
  return or_expf(sigma * z);
}

/* ======================================================================
 * 4. FBP surface rate of spread (Canadian FBP System, surface spread
 *    only) and the ellipse projection of Eqs. (1)-(4).
 * ====================================================================== */
enum { F_NONE = 0, F_C1, F_C2, F_C3, F_C4, F_C5, F_C6, F_C7, F_D1, F_M1, F_M2,
       F_O1A, F_O1B, F_S1, F_S2, F_S3, F_NCODES };

typedef struct { double a, b, c, q, bui0; } fbp_coef;

/* grid code -> (a, b, c, q, BUI0); code 1 = C-1, 2 = C-2, 3 = C-3 as in
 * Table 1 of the paper, continuing through the FBP fuel types. */
static const fbp_coef FBP_COEF[F_NCODES] = {
    {0, 0, 0, 1, 1},                 /* 0 non-fuel */
    {90.0, 0.0649, 4.5, 0.90, 72.0}, /* C1 */
    {110.0, 0.0282, 1.5, 0.70, 64.0},/* C2 */
    {110.0, 0.0444, 3.0, 0.75, 62.0},/* C3 */
    {110.0, 0.0293, 1.5, 0.80, 66.0},/* C4 */
    {30.0, 0.0697, 4.0, 0.80, 56.0}, /* C5 */
    {30.0, 0.0800, 3.0, 0.80, 62.0}, /* C6 */
    {45.0, 0.0305, 2.0, 0.85, 106.0},/* C7 */
    {30.0, 0.0232, 1.6, 0.90, 32.0}, /* D1 */
    {0, 0, 0, 0.80, 50.0},           /* M1: C2/D1 mixture */
    {0, 0, 0, 0.80, 50.0},           /* M2: C2/D1 mixture */
    {190.0, 0.0310, 1.4, 1.0, 1.0},  /* O1a */
    {250.0, 0.0350, 1.7, 1.0, 1.0},  /* O1b */
    {75.0, 0.0297, 1.3, 0.75, 38.0}, /* S1 */
    {40.0, 0.0438, 1.7, 0.75, 63.0}, /* S2 */
    {55.0, 0.0829, 3.2, 0.75, 31.0}, /* S3 */
};

static double rsi_abc(const fbp_coef *k, double isi) {
  double x = 1.0 - or_exp(-k->b * isi);
  return k->a * or_pow(x, k->c);
}

static double curing_factor(double c) {
  if (c < 58.8) return 0.005 * (or_exp(0.061 * c) - 1.0);
  return 0.176 + 0.02 * (c - 58.8);
}

/* initial spread index -> RSI for a fuel code */
static double rsi_fuel(int fuel, double isi, double pcf, double cf) {
  switch (fuel) {
    case F_M1:
      return pcf * rsi_abc(&FBP_COEF[F_C2], isi) + (1.0 - pcf) * rsi_abc(&FBP_COEF[F_D1], isi);
    case F_M2:
      return pcf * rsi_abc(&FBP_COEF[F_C2], isi) +
             0.2 * ((1.0 - pcf) * rsi_abc(&FBP_COEF[F_D1], isi));
    case F_O1A:
    case F_O1B:
      return rsi_abc(&FBP_COEF[fuel], isi) * cf;
    default:
      return rsi_abc(&FBP_COEF[fuel], isi);
  }
}

/* inverse of RSI for one (a,b,c) curve scaled by mult: the ISI that gives rsf.
 * The divisions by a*mult and by -b are multiplications by the rounded
 * reciprocals (divisors fixed per fuel and hour). */
static double isf_abc(const fbp_coef *k, double mult, double rsf) {
  if (!(rsf > 0.0)) return 0.0;
  double x = 1.0 - or_pow(rsf * (1.0 / (k->a * mult)), 1.0 / k->c);
  if (x < 0.01) x = 0.01;
  return or_log(x) * (-1.0 / k->b);
}

/* slope-equivalent ISI (ISF) at slope factor sf */
static double isf_fuel(int fuel, double isz, double sf, double pcf, double cf) {
  switch (fuel) {
    case F_M1: {
      double rsf_c2 = rsi_abc(&FBP_COEF[F_C2], isz) * sf;
      double rsf_d1 = rsi_abc(&FBP_COEF[F_D1], isz) * sf;
      return pcf * isf_abc(&FBP_COEF[F_C2], 1.0, rsf_c2) +
             (1.0 - pcf) * isf_abc(&FBP_COEF[F_D1], 1.0, rsf_d1);
    }
    case F_M2: {
      double rsf_c2 = rsi_abc(&FBP_COEF[F_C2], isz) * sf;
      double rsf_d1 = (0.2 * rsi_abc(&FBP_COEF[F_D1], isz)) * sf;
      return pcf * isf_abc(&FBP_COEF[F_C2], 1.0, rsf_c2) +
             (1.0 - pcf) * isf_abc(&FBP_COEF[F_D1], 0.2, rsf_d1);
    }
    case F_O1A:
    case F_O1B: {
      double rsf = rsi_fuel(fuel, isz, pcf, cf) * sf;
      return isf_abc(&FBP_COEF[fuel], cf, rsf);
    }
    default: {
      double rsf = rsi_abc(&FBP_COEF[fuel], isz) * sf;
      return isf_abc(&FBP_COEF[fuel], 1.0, rsf);
    }
  }
}

static double wind_fn(double w) { /* f(W) of the ISI, 2009 high-wind branch above 40 km/h */
  if (w <= 40.0) return or_exp(0.05039 * w);
  return 12.0 * (1.0 - or_exp(-0.0818 * (w - 28.0)));
}

static double ffmc_fn(double ffmc) { /* f(F) of the ISI */
  double m = 147.2 * (101.0 - ffmc) / (59.5 + ffmc);
  return 91.9 * or_exp(-0.1386 * m) * (1.0 + or_pow(m, 5.31) / 4.93e7);
}

static double buildup_effect(int fuel, double bui) {
  if (fuel == F_O1A || fuel == F_O1B) return 1.0;
  const fbp_coef *k = &FBP_COEF[fuel];
  double t = 50.0 * or_log(k->q);
  double u = 1.0 / bui - 1.0 / k->bui0;
  return or_exp(t * u);
}

/* direction cosines of the 8 axes, theta_k = 45 k degrees, 0 = East,
 * counter-clockwise (Sec. 3.4 (i)); (east, north) components */
static void axis_dirs(double ct[8], double st[8]) {
  double h = sqrt(0.5);
  const double cx[8] = {1.0, h, 0.0, -h, -1.0, -h, 0.0, h};
  const double sy[8] = {0.0, h, 1.0, h, 0.0, -h, -1.0, -h};
  for (int k = 0; k < 8; ++k) { ct[k] = cx[k]; st[k] = sy[k]; }
}

/* Output row layout of or_fbp_cell (and of ellipse_axes' part of it):
 *  0 HROS  1 BROS  2 LB  3 FROS  4 a  5 e  6 ux  7 uy  8 WSV  9 WSE
 *  10..17 ros_k for k = 0..7                                                    */
#define ROW_LEN 18

/* Sec. 3.7, Eqs. (2)-(4): the ellipse of a cell from HROS, BROS and LB, and
 * its rate along each of the 8 axes for a head direction (ux, uy) (unit
 * vector, x east, y north): Eq. (1) (mode 0) or the ray from the ignition
 * point (mode 1).  Fills out[2..7] and out[10..17]. */
static void ellipse_axes(double hros, double bros, double lb, double ux, double uy,
                         int ellipse_mode, double out[ROW_LEN]) {
  double ilb = 1.0 / lb;   /* one reciprocal for FROS and e */
  double fros = ((hros + bros) * ilb) * 0.5;
  double a = (hros + bros) * 0.5;
  double e = sqrt(1.0 - ilb * ilb);
  out[2] = lb; out[3] = fros; out[4] = a; out[5] = e; out[6] = ux; out[7] = uy;
  double ct[8], st[8];
  axis_dirs(ct, st);
  if (ellipse_mode == 0) {
    /* Eq. (1): forward half (cos phi > 0) a(1-e^2)/(1-e cos phi), back half a(1-e^2) */
    double A = a * (1.0 - e * e);
    for (int k = 0; k < 8; ++k) {
      double cphi = ct[k] * ux + st[k] * uy;
      out[10 + k] = (cphi > 0.0) ? A / (1.0 - e * cphi) : A;
    }
  } else {
    /* Centre-offset ellipse (Sec. 3.7, figure CellularHuygens): the ray from
     * the ignition point, c = (HROS-BROS)/2 behind the centre, to the ellipse
     * with semi-axes a (along the head) and b = FROS:
     *   r = (b^2 c cos + a b sqrt(Q)) / (b^2 cos^2 + a^2 sin^2),
     *   Q = b^2 cos^2 + (a^2 - c^2) sin^2,  a^2 - c^2 = HROS BROS.
     * On the back half (cos < 0) the numerator is a difference of nearly
     * equal terms when HROS >> BROS; multiplied out by its conjugate the
     * same ray is r = b^2 HROS BROS / (a b sqrt(Q) - b^2 c cos), a sum of
     * non-negative terms.  a^2 - c^2 is taken as the product HROS BROS. */
    double b = fros;
    double c = (hros - bros) * 0.5;
    double hb = hros * bros;
    for (int k = 0; k < 8; ++k) {
      double cphi = ct[k] * ux + st[k] * uy;
      double sphi2 = 1.0 - cphi * cphi;
      if (sphi2 < 0.0) sphi2 = 0.0;
      double bc = b * b * cphi * cphi;
      double den = bc + a * a * sphi2;
      double root = sqrt(bc + hb * sphi2);
      double r = 0.0;
      if (cphi >= 0.0) {
        if (den > 0.0) r = (b * b * c * cphi + a * b * root) / den;
      } else {
        double q = a * b * root - b * b * c * cphi;
        if (q > 0.0) r = (b * b * hb) / q;
      }
      out[10 + k] = r;
    }
  }
}


OR_API void or_fbp_cell(int fuel, double gs, double aspect_deg, double ws, double wd_from,
                        double ffmc, double bui, double m1_pc, double o1_curing,
                        int ellipse_mode, double out[ROW_LEN]) {
  or_init_tables();
  for (int i = 0; i < ROW_LEN; ++i) out[i] = 0.0;
  if (fuel <= F_NONE || fuel >= F_NCODES) return;
  double pcf = m1_pc / 100.0;
  double cf = curing_factor(o1_curing);
  /* weather-only terms (hour) */
  double ff = ffmc_fn(ffmc);
  double isz = 0.208 * ff;
  double sin_w, cos_w;
  or_sincos_deg(wd_from + 180.0, &sin_w, &cos_w);
  double be = buildup_effect(fuel, bui);
  /* topography (cell) */
  double sin_s, cos_s;
  or_sincos_deg(aspect_deg + 180.0, &sin_s, &cos_s);
  double wse = 0.0;
  if (gs > 0.0) {
    double g = (gs < 60.0 ? gs : 60.0) / 100.0;
    double sf = or_exp(3.533 * or_pow(g, 1.2));
    double isf = isf_fuel(fuel, isz, sf, pcf, cf);
    if (isf > 0.0) {
      wse = or_log(isf * (1.0 / isz)) * (1.0 / 0.05039);
      if (wse > 40.0) {
        if (isf < 0.999 * 2.496 * ff)
          wse = 28.0 - or_log(1.0 - isf / (2.496 * ff)) / 0.0818;
        else
          wse = 112.45;
      }
    }
  }
  /* net effective wind vector, compass components (x east, y north) */
  double wsx = ws * sin_w + wse * sin_s;
  double wsy = ws * cos_w + wse * cos_s;
  double wsv = sqrt(wsx * wsx + wsy * wsy);
  double ux = 1.0, uy = 0.0;
  if (wsv > 0.0) {
    double iw = 1.0 / wsv;
    ux = wsx * iw;
    uy = wsy * iw;
  }
  double isi = isz * wind_fn(wsv);
  double hros = rsi_fuel(fuel, isi, pcf, cf) * be;
  double bisi = isz * or_exp(-0.05039 * wsv);
  double bros = rsi_fuel(fuel, bisi, pcf, cf) * be;
  double lb;
  if (fuel == F_O1A || fuel == F_O1B)
    lb = (wsv >= 1.0) ? 1.1 * or_pow(wsv, 0.464) : 1.0;
  else
    lb = 1.0 + 8.729 * or_pow(1.0 - or_exp(-0.030 * wsv), 2.155);
  out[0] = hros; out[1] = bros; out[8] = wsv; out[9] = wse;
  ellipse_axes(hros, bros, lb, ux, uy, ellipse_mode, out);
}

/* ======================================================================
 * 5. Fixed-point progress (2^32 units per metre) and the simulation.
 * ====================================================================== */
#define FP_ONE 4294967296.0
#define FIX_CAP 4611686018427387904LL /* 2^62 */

static int64_t fixed_of(double x) {
  if (!(x > 0.0)) return 0;
  if (x >= 4611686018427387904.0) return FIX_CAP;
  return (int64_t)llrint(x);
}

/* noise factor f as a 32.32 fixed-point multiplier */
static uint64_t noise_fixed(float f) { return (uint64_t)((double)f * FP_ONE); }

static int64_t apply_noise(int64_t base, uint64_t F, int64_t dk) {
  unsigned __int128 p = (unsigned __int128)(uint64_t)base * F + ((unsigned __int128)1 << 31);
  unsigned __int128 inc = p >> 32;
  if (inc > (unsigned __int128)dk) return dk;
  return (int64_t)inc;
}

typedef struct {
  uint64_t seed;
  int32_t hours;
  int32_t minutes_per_step;
  int32_t ignition_mode;  /* 0 fixed cell, 1 uniform over burnable cells */
  int32_t ignition_cell;
  double ros_sigma;
  double ros_threshold;
  double burnout_delta;
  int32_t ellipse_mode;
  double o1_curing_pct;
  double m1_pc;
  double const_ros;       /* > 0: every burnable cell spreads at this rate on all axes */
  int32_t burn_hours_min; /* burning hours per day drawn per replica from       */
  int32_t burn_hours_max; /* {min..max}; 0, 0: no limit (A5 general cond. (1))  */
  double const_bros;      /* with const_ros > 0: BROS (0 = const_ros) and LB (<= 1:  */
  double const_lb;        /* a circle); the head follows the hour's wind direction */
} or_params;

typedef struct {
  int32_t rows, cols, n;
  double cell_size;
  uint8_t *fuel;
  float *slope, *aspect;
  uint8_t *burnable;
  int32_t n_hours;
  double *weather; /* n_hours x 4 : ws_kmh, wd_from_deg, ffmc, bui */
  or_params p;
  int32_t n_burnable;
  int32_t *burnable_list;
  /* lazily filled table rows, per (hour, cell) */
  uint8_t *have;
  int64_t *base; /* (hour, cell, 8) */
  double *hros;  /* (hour, cell)    */
  int64_t D[8];
  int32_t sph, S;
} or_ctx;

OR_API or_ctx *or_create(int32_t rows, int32_t cols, double cell_size, const uint8_t *fuel,
                         const float *slope, const float *aspect, const uint8_t *unburnable,
                         int32_t n_hours, const double *weather, const or_params *p) {
  or_init_tables();
  or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
  c->rows = rows; c->cols = cols; c->n = rows * cols; c->cell_size = cell_size;
  size_t n = (size_t)c->n;
  c->fuel = (uint8_t *)malloc(n);
  c->slope = (float *)malloc(n * 4);
  c->aspect = (float *)malloc(n * 4);
  c->burnable = (uint8_t *)malloc(n);
  memcpy(c->fuel, fuel, n);
  for (size_t i = 0; i < n; ++i) {
    c->slope[i] = slope ? slope[i] : 0.0f;
    c->aspect[i] = aspect ? aspect[i] : 0.0f;
    c->burnable[i] = (fuel[i] != 0 && !(unburnable && unburnable[i])) ? 1 : 0;
  }
  c->n_hours = n_hours;
  c->weather = (double *)malloc((size_t)n_hours * 4 * 8);
  memcpy(c->weather, weather, (size_t)n_hours * 4 * 8);
  c->p = *p;
  c->burnable_list = (int32_t *)malloc(n * 4);
  c->n_burnable = 0;
  for (size_t i = 0; i < n; ++i)
    if (c->burnable[i]) c->burnable_list[c->n_burnable++] = (int32_t)i;
  size_t nh = (size_t)p->hours;
  c->have = (uint8_t *)calloc(nh * n, 1);
  c->base = (int64_t *)malloc(nh * n * 8 * 8);
  c->hros = (double *)malloc(nh * n * 8);
  int64_t dorth = (int64_t)llrint(cell_size * FP_ONE);
  int64_t ddiag = (int64_t)llrint((cell_size * sqrt(2.0)) * FP_ONE);
  for (int k = 0; k < 8; ++k) c->D[k] = (k % 2 == 0) ? dorth : ddiag;
  c->sph = 60 / p->minutes_per_step;
  c->S = p->hours * c->sph;
  return c;
}

OR_API void or_destroy(or_ctx *c) {
  if (!c) return;
  free(c->fuel); free(c->slope); free(c->aspect); free(c->burnable); free(c->weather);
  free(c->burnable_list); free(c->have); free(c->base); free(c->hros);
  free(c);
}

OR_API void or_distances(const or_ctx *c, int64_t out[8]) {
  for (int k = 0; k < 8; ++k) out[k] = c->D[k];
}

/* full FBP / Eq. (1) row of one cell at one weather hour */
OR_API void or_cell_row(const or_ctx *c, int32_t cell, int32_t hour, double out[ROW_LEN]) {
  const double *w = c->weather + (size_t)hour * 4;
  if (!c->burnable[cell]) {
    for (int i = 0; i < ROW_LEN; ++i) out[i] = 0.0;
    return;
  }
  if (c->p.const_ros > 0.0) {
    for (int i = 0; i < ROW_LEN; ++i) out[i] = 0.0;
    if (c->p.const_bros > 0.0 || c->p.const_lb > 1.0) {
      /* test hook: the ellipse of Sec. 3.7 from given HROS, BROS and LB, its
       * head along the hour's wind (toward WD + 180), rates by Eq. (1) or the
       * ray of ellipse_mode 1 */
      double hros = c->p.const_ros;
      double bros = c->p.const_bros > 0.0 ? c->p.const_bros : hros;
      double lb = c->p.const_lb > 1.0 ? c->p.const_lb : 1.0;
      double sw, cw;
      or_sincos_deg(w[1] + 180.0, &sw, &cw);
      out[0] = hros; out[1] = bros;
      ellipse_axes(hros, bros, lb, sw, cw, c->p.ellipse_mode, out);
      return;
    }
    out[0] = c->p.const_ros; out[1] = c->p.const_ros; out[2] = 1.0; out[3] = c->p.const_ros;
    out[4] = c->p.const_ros; out[6] = 1.0;
    for (int k = 0; k < 8; ++k) out[10 + k] = c->p.const_ros;
    return;
  }
  or_fbp_cell(c->fuel[cell], (double)c->slope[cell], (double)c->aspect[cell], w[0], w[1], w[2],
              w[3], c->p.m1_pc, c->p.o1_curing_pct, c->p.ellipse_mode, out);
}

static void ensure_row(or_ctx *c, int32_t cell, int32_t hour) {
  size_t idx = (size_t)hour * c->n + cell;
  if (c->have[idx]) return;
  double row[ROW_LEN];
  or_cell_row(c, cell, hour, row);
  double dt2p32 = (double)c->p.minutes_per_step * FP_ONE;
  for (int k = 0; k < 8; ++k) c->base[idx * 8 + k] = fixed_of(row[10 + k] * dt2p32);
  c->hros[idx] = row[0];
  c->have[idx] = 1;
}

/* test hook: the table row of (cell, hour) from given rates -- the 8 axis rates
 * (m/min) and HROS -- instead of the oracle's own FBP evaluation; the
 * fixed-point increments follow from them as for computed rows ([R2]) */
OR_API void or_set_row(or_ctx *c, int32_t cell, int32_t hour, const double ros8[8], double hros) {
  size_t idx = (size_t)hour * c->n + cell;
  double dt2p32 = (double)c->p.minutes_per_step * FP_ONE;
  for (int k = 0; k < 8; ++k) c->base[idx * 8 + k] = fixed_of(ros8[k] * dt2p32);
  c->hros[idx] = hros;
  c->have[idx] = 1;
}

/* base fixed-point increments B_k = fixed(ros_k * dt * 2^32) of (cell, hour) */
OR_API void or_base_inc(or_ctx *c, int32_t cell, int32_t hour, int64_t out[8], double *hros) {
  ensure_row(c, cell, hour);
  size_t idx = (size_t)hour * c->n + cell;
  for (int k = 0; k < 8; ++k) out[k] = c->base[idx * 8 + k];
  if (hros) *hros = c->hros[idx];
}

static int nbr_of(const or_ctx *c, int32_t cell, int k) {
  static const int DR[8] = {0, -1, -1, -1, 0, 1, 1, 1};
  static const int DC[8] = {1, 1, 0, -1, -1, -1, 0, 1};
  int r = cell / c->cols, q = cell % c->cols;
  int rr = r + DR[k], qq = q + DC[k];
  if (rr < 0 || rr >= c->rows || qq < 0 || qq >= c->cols) return -1;
  return rr * c->cols + qq;
}

/* Step 1 of Alg. 1: ignition cell of a replica (uncertainty source (1)) */
OR_API int32_t or_ignition_cell(const or_ctx *c, int32_t replica) {
  if (c->p.ignition_mode == 0) return c->p.ignition_cell;
  uint32_t ctr[4] = {(uint32_t)replica, 0u, 0u, 1u};
  uint32_t key[2] = {(uint32_t)c->p.seed, (uint32_t)(c->p.seed >> 32)};
  uint32_t x[4];
  or_philox4x32_10(ctr, key, x);
  uint64_t idx = ((uint64_t)x[0] * (uint64_t)(uint32_t)c->n_burnable) >> 32;
  return c->burnable_list[idx];
}

/* A5, general fire dynamics (1): a replica's fire burns for at most B hours of
 * each day.  B is drawn per replica uniformly from {min..max} with one Philox
 * block at counter (replica, 0, 0, 3): B = min + (x0 (max - min + 1)) >> 32
 * (min = max: a constant).  Weather hour h is a burning hour iff h mod 24 < B;
 * in the other hours the fire is dormant: no spread, no messages, no
 * ignitions, no burn-out, no work counted, progress kept.  Returns 24 when
 * there is no limit. */
OR_API int32_t or_burn_hours(const or_ctx *c, int32_t replica) {
  if (c->p.burn_hours_max <= 0) return 24;
  uint32_t ctr[4] = {(uint32_t)replica, 0u, 0u, 3u};
  uint32_t key[2] = {(uint32_t)c->p.seed, (uint32_t)(c->p.seed >> 32)};
  uint32_t x[4];
  or_philox4x32_10(ctr, key, x);
  uint64_t span = (uint64_t)(c->p.burn_hours_max - c->p.burn_hours_min + 1);
  return c->p.burn_hours_min + (int32_t)(((uint64_t)x[0] * span) >> 32);
}

static float noise_of(const or_ctx *c, int32_t replica, int32_t cell, int32_t hour) {
  return or_noise_factor(c->p.seed, (uint32_t)replica, (uint32_t)cell, (uint32_t)hour,
                         (float)c->p.ros_sigma);
}

/* per-replica memo of noise factors, one per (cell) for the current hour */
typedef struct { int32_t *hour; float *val; } noise_memo;

static float memo_noise(const or_ctx *c, noise_memo *m, int32_t r, int32_t cell, int32_t h) {
  if (m->hour[cell] != h) { m->val[cell] = noise_of(c, r, cell, h); m->hour[cell] = h; }
  return m->val[cell];
}

enum { ST_AVAIL = 0, ST_BURNING = 1, ST_BURNED = 2, ST_UNBURNABLE = 3 };

/* ----------------------------------------------------------------------
 * O1: Algorithm 1 stepped one fire period at a time, exactly as stated:
 *   per step s: count the burning set; send (every burning cell advances
 *   each open axis whose neighbour is Available at the start of the step,
 *   and messages the neighbour when progress reaches its centre); receive
 *   (a messaged Available cell ignites if its ROS exceeds the threshold);
 *   burn-out (A5 (ii), and (i) when delta > 0); stop when nothing burns.
 * Outputs: scar (1 = ever ignited), ignition step (-1 = never), the work
 * count W = sum over steps of the burning-set size, and ignited cells.
 * ---------------------------------------------------------------------- */
OR_API int or_run_replica(or_ctx *c, int32_t replica, uint8_t *scar, int32_t *ign_out,
                          int64_t *work_out, int32_t *n_ign_out, int32_t *ic_out) {
  int32_t n = c->n;
  uint8_t *state = (uint8_t *)malloc((size_t)n);
  int32_t *ign = (int32_t *)malloc((size_t)n * 4);
  noise_memo nm;
  nm.hour = (int32_t *)malloc((size_t)n * 4);
  nm.val = (float *)malloc((size_t)n * 4);
  for (int32_t i = 0; i < n; ++i) {
    state[i] = c->burnable[i] ? ST_AVAIL : ST_UNBURNABLE;
    ign[i] = -1;
    nm.hour[i] = -1;
  }
  /* burning list */
  int32_t cap = 1024, len = 0;
  int32_t *lcell = (int32_t *)malloc((size_t)cap * 4);
  int64_t *lP = (int64_t *)malloc((size_t)cap * 64);
  uint8_t *lopen = (uint8_t *)malloc((size_t)cap);
  int32_t *msg = (int32_t *)malloc((size_t)n * 4);

  int32_t ic = or_ignition_cell(c, replica);
  state[ic] = ST_BURNING;
  ign[ic] = 0;
  lcell[0] = ic; memset(lP, 0, 64); lopen[0] = 0xFF; len = 1;

  int64_t W = 0;
  int32_t dt = c->p.minutes_per_step;
  int32_t B = or_burn_hours(c, replica);
  for (int32_t s = 1; s <= c->S; ++s) {
    int32_t h = ((s - 1) * dt) / 60;
    if (len == 0) break;
    if (h % 24 >= B) continue;   /* dormant hour of the day */
    W += len;
    /* send: the state array is not modified until the receive stage */
    int32_t nmsg = 0;
    for (int32_t e = 0; e < len; ++e) {
      int32_t i = lcell[e];
      int64_t base[8];
      uint64_t F = 0;
      int have_inc = 0;
      for (int k = 0; k < 8; ++k) {
        if (!(lopen[e] & (1u << k))) continue;
        int j = nbr_of(c, i, k);
        if (j < 0 || state[j] != ST_AVAIL) continue;
        if (!have_inc) {
          or_base_inc(c, i, h, base, NULL);
          F = noise_fixed(memo_noise(c, &nm, replica, i, h));
          have_inc = 1;
        }
        lP[(size_t)e * 8 + k] += apply_noise(base[k], F, c->D[k]);
        if (lP[(size_t)e * 8 + k] >= c->D[k]) {
          msg[nmsg++] = j;
          lopen[e] &= (uint8_t)~(1u << k);
        }
      }
    }
    /* receive */
    for (int32_t m = 0; m < nmsg; ++m) {
      int32_t j = msg[m];
      if (state[j] != ST_AVAIL) continue;
      double hr;
      int64_t bj[8];
      or_base_inc(c, j, h, bj, &hr);
      float fj = memo_noise(c, &nm, replica, j, h);
      if (!(hr * (double)fj > c->p.ros_threshold)) continue;
      state[j] = ST_BURNING;
      ign[j] = s;
      if (len == cap) {
        cap *= 2;
        lcell = (int32_t *)realloc(lcell, (size_t)cap * 4);
        lP = (int64_t *)realloc(lP, (size_t)cap * 64);
        lopen = (uint8_t *)realloc(lopen, (size_t)cap);
      }
      lcell[len] = j; memset(lP + (size_t)len * 8, 0, 64); lopen[len] = 0xFF; ++len;
    }
    /* burn-out (A5): (ii) no Available neighbour; (i) ROS below delta */
    int32_t out = 0;
    for (int32_t e = 0; e < len; ++e) {
      int32_t i = lcell[e];
      int dead = 1;
      for (int k = 0; k < 8 && dead; ++k) {
        int j = nbr_of(c, i, k);
        if (j >= 0 && state[j] == ST_AVAIL) dead = 0;
      }
      if (!dead && c->p.burnout_delta > 0.0) {
        double hr;
        int64_t bi[8];
        or_base_inc(c, i, h, bi, &hr);
        float fi = memo_noise(c, &nm, replica, i, h);
        if (hr * (double)fi < c->p.burnout_delta) dead = 1;
      }
      if (dead) {
        state[i] = ST_BURNED;
      } else {
        lcell[out] = lcell[e];
        memmove(lP + (size_t)out * 8, lP + (size_t)e * 8, 64);
        lopen[out] = lopen[e];
        ++out;
      }
    }
    len = out;
  }
  int32_t nig = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (scar) scar[i] = (ign[i] >= 0) ? 1 : 0;
    if (ign_out) ign_out[i] = ign[i];
    if (ign[i] >= 0) ++nig;
  }
  if (work_out) *work_out = W;
  if (n_ign_out) *n_ign_out = nig;
  if (ic_out) *ic_out = ic;
  free(state); free(ign); free(nm.hour); free(nm.val);
  free(lcell); free(lP); free(lopen); free(msg);
  return 0;
}

/* ----------------------------------------------------------------------
 * O2: the same model as a label-setting (Dijkstra) search over integer
 * ignition steps.  Progress along an axis is piecewise linear in the step
 * count (constant increment within a weather hour), so the step at which
 * sender i's axis reaches the neighbour's centre follows from i's ignition
 * step alone; the neighbour's ignition step is the earliest such crossing
 * whose receive test passes.  The work count follows from the ignition
 * steps: cell i is burning at the start of steps t_i+1 .. min(death_i, S).
 * With a burning-hours limit the dormant hours add no progress, burn
 * nothing out and count no work.
 * ---------------------------------------------------------------------- */
typedef struct { int32_t t, cell; } heap_item;

static void heap_push(heap_item *h, int32_t *len, heap_item it) {
  int32_t i = (*len)++;
  h[i] = it;
  while (i > 0) {
    int32_t p = (i - 1) / 2;
    if (h[p].t <= h[i].t) break;
    heap_item tmp = h[p]; h[p] = h[i]; h[i] = tmp;
    i = p;
  }
}

static heap_item heap_pop(heap_item *h, int32_t *len) {
  heap_item top = h[0];
  h[0] = h[--(*len)];
  int32_t i = 0;
  for (;;) {
    int32_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < *len && h[l].t < h[m].t) m = l;
    if (r < *len && h[r].t < h[m].t) m = r;
    if (m == i) break;
    heap_item tmp = h[m]; h[m] = h[i]; h[i] = tmp;
    i = m;
  }
  return top;
}

static double ros_times_noise(or_ctx *c, int32_t r, int32_t cell, int32_t hour) {
  double hr;
  int64_t b[8];
  or_base_inc(c, cell, hour, b, &hr);
  return hr * (double)noise_of(c, r, cell, hour);
}

/* first step s >= from at which the delta burn-out fires, or INT32_MAX */
/* the step at whose end A5 (i) burns the cell out, tested from step `from` on
 * in the burning hours only (B = burning hours per day; dormant hours burn
 * nothing out) */
static int32_t delta_death(or_ctx *c, int32_t r, int32_t cell, int32_t from, int32_t B) {
  if (!(c->p.burnout_delta > 0.0)) return INT32_MAX;
  int32_t dt = c->p.minutes_per_step;
  for (int32_t s = from; s <= c->S;) {
    int32_t h = ((s - 1) * dt) / 60;
    if (h % 24 < B && ros_times_noise(c, r, cell, h) < c->p.burnout_delta) return s;
    s = (h + 1) * c->sph + 1;
  }
  return INT32_MAX;
}

/* steps a+1 .. b that fall in burning hours (the others count no work) */
static int64_t burning_steps(const or_ctx *c, int32_t a, int32_t b, int32_t B) {
  if (B >= 24) return b > a ? (int64_t)(b - a) : 0;
  int64_t w = 0;
  for (int32_t s = a + 1; s <= b;) {
    int32_t h = ((s - 1) * c->p.minutes_per_step) / 60;
    int32_t L = (h + 1) * c->sph;
    if (L > b) L = b;
    if (h % 24 < B) w += (int64_t)(L - s + 1);
    s = L + 1;
  }
  return w;
}

OR_API int or_run_replica_event(or_ctx *c, int32_t replica, uint8_t *scar, int32_t *ign_out,
                                int64_t *work_out, int32_t *n_ign_out, int32_t *ic_out) {
  int32_t n = c->n;
  const int32_t B = or_burn_hours(c, replica);   /* 24: no dormant hours */
  const int32_t INF = INT32_MAX;
  int32_t *t = (int32_t *)malloc((size_t)n * 4);
  uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
  int32_t *death = (int32_t *)malloc((size_t)n * 4);
  heap_item *heap = (heap_item *)malloc(((size_t)n * 8 + 8) * sizeof(heap_item));
  int32_t hl = 0;
  for (int32_t i = 0; i < n; ++i) t[i] = INF;
  int32_t ic = or_ignition_cell(c, replica);
  t[ic] = 0;
  heap_push(heap, &hl, (heap_item){0, ic});
  int32_t dt = c->p.minutes_per_step;
  while (hl > 0) {
    heap_item it = heap_pop(heap, &hl);
    int32_t i = it.cell;
    if (done[i] || it.t != t[i]) continue;
    done[i] = 1;
    int32_t ti = t[i];
    int32_t first = ti > 1 ? ti : 1;
    death[i] = delta_death(c, replica, i, first, B);
    int32_t limit = death[i] < c->S ? death[i] : c->S;
    for (int k = 0; k < 8; ++k) {
      int32_t j = nbr_of(c, i, k);
      if (j < 0 || !c->burnable[j] || done[j]) continue;
      /* crossing step of axis k of i, accumulating from step ti+1 */
      int64_t P = 0;
      int32_t cross = INF;
      for (int32_t s = ti + 1; s <= limit;) {
        int32_t h = ((s - 1) * dt) / 60;
        int32_t L = (h + 1) * c->sph;
        if (L > limit) L = limit;
        if (h % 24 >= B) { s = L + 1; continue; }   /* dormant hour: no progress */
        int64_t b[8];
        or_base_inc(c, i, h, b, NULL);
        int64_t inc = apply_noise(b[k], noise_fixed(noise_of(c, replica, i, h)), c->D[k]);
        int64_t nsteps = (int64_t)(L - s + 1);
        if (inc > 0 && P + nsteps * inc >= c->D[k]) {
          int64_t need = (c->D[k] - P + inc - 1) / inc;
          cross = s + (int32_t)need - 1;
          break;
        }
        P += nsteps * inc;
        s = L + 1;
      }
      if (cross == INF || cross >= t[j]) continue;
      int32_t hc = ((cross - 1) * dt) / 60;
      if (!(ros_times_noise(c, replica, j, hc) > c->p.ros_threshold)) continue;
      t[j] = cross;
      heap_push(heap, &hl, (heap_item){cross, j});
    }
  }
  int64_t W = 0;
  int32_t nig = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (t[i] == INF) continue;
    ++nig;
    int32_t b = t[i] > 1 ? t[i] : 1;
    for (int k = 0; k < 8; ++k) {
      int32_t j = nbr_of(c, i, k);
      if (j < 0 || !c->burnable[j]) continue;
      if (t[j] == INF) { b = INF; break; }
      if (t[j] > b) b = t[j];
    }
    int32_t d = death[i] < b ? death[i] : b;
    if (d > c->S) d = c->S;
    W += burning_steps(c, t[i], d, B);
  }
  for (int32_t i = 0; i < n; ++i) {
    if (scar) scar[i] = (t[i] != INF) ? 1 : 0;
    if (ign_out) ign_out[i] = (t[i] != INF) ? t[i] : -1;
  }
  if (work_out) *work_out = W;
  if (n_ign_out) *n_ign_out = nig;
  if (ic_out) *ic_out = ic;
  free(t); free(done); free(death); free(heap);
  return 0;
}

/* ======================================================================
 * 6. Weather scenarios (Sec. 3.1, uncertainty source (3)): a request may
 *    carry several weather streams, scenario s occurring with probability
 *    p_s.  Every replica runs under one scenario, drawn with those
 *    probabilities from its own Philox block at counter (replica, 0, 0, 2):
 *    with x0 the block's first word, the replica takes the first s with
 *    x0 < T_s, where T_s = floor(2^32 (p_0 + ... + p_s) / (p_0 + ... +
 *    p_{S-1})) (sums left to right in binary64) and T_{S-1} = 2^32.  So
 *    P(s) = (T_s - T_{s-1}) / 2^32, within 2^-32 of p_s / sum p, and a
 *    scenario with p_s = 0 is never taken.
 * ====================================================================== */
OR_API int or_scenario_thresholds(int32_t n, const double *prob, uint64_t *thr) {
  if (n < 1) return -1;
  double total = 0.0;
  for (int32_t s = 0; s < n; ++s) {
    if (!(prob[s] >= 0.0) || !isfinite(prob[s])) return -1;
    total += prob[s];
  }
  if (!(total > 0.0) || !isfinite(total)) return -1;
  double cum = 0.0;
  for (int32_t s = 0; s < n; ++s) {
    cum += prob[s];
    if (s == n - 1) thr[s] = (uint64_t)1 << 32;
    else thr[s] = (uint64_t)((cum / total) * FP_ONE);   /* cum <= total: at most 2^32 */
  }
  return 0;
}

OR_API int32_t or_scenario(uint64_t seed, int32_t replica, int32_t n, const uint64_t *thr) {
  if (n <= 1) return 0;
  uint32_t ctr[4] = {(uint32_t)replica, 0u, 0u, 2u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  or_philox4x32_10(ctr, key, x);
  for (int32_t s = 0; s < n - 1; ++s)
    if ((uint64_t)x[0] < thr[s]) return s;
  return n - 1;
}
