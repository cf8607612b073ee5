// c2f_fbp.cuh -- FBP surface rate of spread and the ellipse projection.
//
// Cell2Fire takes HROS, BROS and the length-to-breadth ratio LB of each cell
// from the Canadian FBP System (Sec. 2.3, 3.1, assumption A2) and projects
// them onto an ellipse (Sec. 3.7, Eqs. 2-4) to get the rate of spread along
// the 8 centre-to-centre axes by Eq. (1).  The FBP equations are not printed
// in the paper; this file restates the standard surface-spread form (RSI
// curve a(1-exp(-b ISI))^c, build-up effect, slope factor and slope-equivalent
// wind, net wind vector, LB; M1/M2 mixtures; O1 curing), surface fire only.
//
// Work is split three ways so the expensive binary64 transcendentals run once
// where they can:
//   HourPrep  per weather hour  (FFMC function, zero-wind ISI, wind vector,
//             build-up effect and zero-wind RSI per fuel code)
//   CellPrep  per cell          (slope factor, upslope direction)
//   fbp_row   per (cell, hour)  (slope-equivalent wind, net wind, HROS, BROS,
//             LB, ellipse, the 8 axis rates)
#pragma once
#include "c2f_math.cuh"

namespace c2f {

// FBP fuel-type coefficients (a, b, c of the RSI curve; q and BUI0 of the
// build-up effect).  Table 1 of the paper maps grid code 1 -> C-1, 2 -> C-2,
// 3 -> C-3; the remaining codes continue through the FBP fuel types.
__constant__ FuelCoef g_fuel[F_NCODES];

inline void make_fuel_table(FuelCoef t[F_NCODES]) {
  const FuelCoef v[F_NCODES] = {
      {0, 0, 0, 1, 1},
      {90.0, 0.0649, 4.5, 0.90, 72.0},    // C1 spruce-lichen woodland
      {110.0, 0.0282, 1.5, 0.70, 64.0},   // C2 boreal spruce
      {110.0, 0.0444, 3.0, 0.75, 62.0},   // C3 mature jack / lodgepole pine
      {110.0, 0.0293, 1.5, 0.80, 66.0},   // C4 immature jack / lodgepole pine
      {30.0, 0.0697, 4.0, 0.80, 56.0},    // C5 red and white pine
      {30.0, 0.0800, 3.0, 0.80, 62.0},    // C6 conifer plantation
      {45.0, 0.0305, 2.0, 0.85, 106.0},   // C7 ponderosa pine / Douglas-fir
      {30.0, 0.0232, 1.6, 0.90, 32.0},    // D1 leafless aspen
      {0, 0, 0, 0.80, 50.0},              // M1 boreal mixedwood, leafless
      {0, 0, 0, 0.80, 50.0},              // M2 boreal mixedwood, green
      {190.0, 0.0310, 1.4, 1.0, 1.0},     // O1a matted grass
      {250.0, 0.0350, 1.7, 1.0, 1.0},     // O1b standing grass
      {75.0, 0.0297, 1.3, 0.75, 38.0},    // S1 jack / lodgepole pine slash
      {40.0, 0.0438, 1.7, 0.75, 63.0},    // S2 white spruce / balsam slash
      {55.0, 0.0829, 3.2, 0.75, 31.0},    // S3 coastal cedar / hemlock slash
  };
  for (int i = 0; i < F_NCODES; ++i) {
    t[i] = v[i];
    t[i].inv_c = v[i].c != 0.0 ? 1.0 / v[i].c : 0.0;          // divisors of isf_curve,
    t[i].neg_inv_b = v[i].b != 0.0 ? -1.0 / v[i].b : 0.0;     // fixed per fuel
    t[i].c2 = pow_half_steps(v[i].c);
    t[i].inv_c2 = pow_half_steps(t[i].inv_c);
  }
}

__device__ __forceinline__ bool is_o1(int f) { return f == F_O1A || f == F_O1B; }

__device__ __forceinline__ double rsi_curve(const FuelCoef &k, double isi) {
  const double x = __dsub_rn(1.0, dexp(__dmul_rn(-k.b, isi)));
  return __dmul_rn(k.a, dpow_n2(x, k.c, k.c2));
}

__device__ inline double curing_factor(double c) {
  if (c < 58.8) return __dmul_rn(0.005, __dsub_rn(dexp(__dmul_rn(0.061, c)), 1.0));
  return __dadd_rn(0.176, __dmul_rn(0.02, __dsub_rn(c, 58.8)));
}

__device__ inline double rsi_of(int fuel, double isi, double pcf, double cf) {
  if (fuel == F_M1)
    return __dadd_rn(__dmul_rn(pcf, rsi_curve(g_fuel[F_C2], isi)),
                     __dmul_rn(__dsub_rn(1.0, pcf), rsi_curve(g_fuel[F_D1], isi)));
  if (fuel == F_M2)
    return __dadd_rn(__dmul_rn(pcf, rsi_curve(g_fuel[F_C2], isi)),
                     __dmul_rn(0.2, __dmul_rn(__dsub_rn(1.0, pcf), rsi_curve(g_fuel[F_D1], isi))));
  if (is_o1(fuel)) return __dmul_rn(rsi_curve(g_fuel[fuel], isi), cf);
  return rsi_curve(g_fuel[fuel], isi);
}

// ISI at which the (a*mult, b, c) curve gives rsf; the 1 - (rsf/a)^(1/c) term is
// held at >= 0.01.  inv_am = RN(1 / (a mult)); the divisions by a mult and by
// -b are multiplications by rounded reciprocals.
__device__ inline double isf_curve(const FuelCoef &k, double inv_am, double rsf) {
  if (!pos(rsf)) return 0.0;
  double x = __dsub_rn(1.0, dpow_n2(__dmul_rn(rsf, inv_am), k.inv_c, k.inv_c2));
  if (lt_c(x, 0.01)) x = 0.01;
  return __dmul_rn(dlog(x), k.neg_inv_b);
}

__device__ inline double isf_of(int fuel, const HourPrep &hp, double sf, double pcf) {
  if (fuel == F_M1) {
    const double rsf_c2 = __dmul_rn(hp.rszf[F_C2], sf);
    const double rsf_d1 = __dmul_rn(hp.rszf[F_D1], sf);
    return __dadd_rn(__dmul_rn(pcf, isf_curve(g_fuel[F_C2], hp.inv_a[F_C2], rsf_c2)),
                     __dmul_rn(__dsub_rn(1.0, pcf), isf_curve(g_fuel[F_D1], hp.inv_a[F_D1], rsf_d1)));
  }
  if (fuel == F_M2) {
    const double rsf_c2 = __dmul_rn(hp.rszf[F_C2], sf);
    const double rsf_d1 = __dmul_rn(__dmul_rn(0.2, hp.rszf[F_D1]), sf);
    return __dadd_rn(__dmul_rn(pcf, isf_curve(g_fuel[F_C2], hp.inv_a[F_C2], rsf_c2)),
                     __dmul_rn(__dsub_rn(1.0, pcf), isf_curve(g_fuel[F_D1], hp.inv_a_d1m2, rsf_d1)));
  }
  const double rsf = __dmul_rn(hp.rszf[fuel], sf);
  return isf_curve(g_fuel[fuel], hp.inv_a[fuel], rsf);
}

// wind function of the ISI; above 40 km/h the saturating branch of the 2009 update
__device__ __forceinline__ double wind_fn(double w) {
  if (le_c(w, 40.0)) return dexp(__dmul_rn(0.05039, w));
  return __dmul_rn(12.0, __dsub_rn(1.0, dexp(__dmul_rn(-0.0818, __dsub_rn(w, 28.0)))));
}

// per weather hour: (ws, wd_from, ffmc, bui) -> HourPrep
__device__ inline void hour_prep(double ws, double wd_from, double ffmc, double bui, double cf,
                                 HourPrep *hp) {
  const double m = __ddiv_rn(__dmul_rn(147.2, __dsub_rn(101.0, ffmc)), __dadd_rn(59.5, ffmc));
  const double ff = __dmul_rn(__dmul_rn(91.9, dexp(__dmul_rn(-0.1386, m))),
                              __dadd_rn(1.0, __ddiv_rn(dpow(m, 5.31), 4.93e7)));
  hp->ws = ws;
  hp->ff = ff;
  hp->cf = cf;
  hp->isz = __dmul_rn(0.208, ff);
  dsincos_deg(__dadd_rn(wd_from, 180.0), &hp->sin_w, &hp->cos_w);
  for (int f = 0; f < F_NCODES; ++f) {
    double be = 1.0;
    if (f != F_NONE && !is_o1(f)) {
      const double t = __dmul_rn(50.0, dlog(g_fuel[f].q));
      const double u = __dsub_rn(__ddiv_rn(1.0, bui), __ddiv_rn(1.0, g_fuel[f].bui0));
      be = dexp(__dmul_rn(t, u));
    }
    hp->be[f] = be;
    double rz = 0.0;
    if (f != F_NONE && f != F_M1 && f != F_M2) {
      rz = rsi_curve(g_fuel[f], hp->isz);
      if (is_o1(f)) rz = __dmul_rn(rz, cf);
    }
    hp->rszf[f] = rz;
    const double mult = is_o1(f) ? cf : 1.0;
    hp->inv_a[f] = g_fuel[f].a != 0.0 ? __ddiv_rn(1.0, __dmul_rn(g_fuel[f].a, mult)) : 0.0;
  }
  hp->inv_a_d1m2 = __ddiv_rn(1.0, __dmul_rn(g_fuel[F_D1].a, 0.2));
  hp->inv_isz = __ddiv_rn(1.0, hp->isz);
  hp->wsx_w = __dmul_rn(hp->ws, hp->sin_w);
  hp->wsy_w = __dmul_rn(hp->ws, hp->cos_w);
  // A lower bound on every fuel's HROS this hour: the RSI curve grows with the
  // ISI and the ISI with the wind (wind_fn >= 1 for w >= 0), so RSI >= RSI at
  // zero wind (rszf); a C2/D1 mixture is at least 0.2 x its smaller part.
  int32_t pos = 1;
  for (int f = 1; f < F_NCODES; ++f) {
    double lo = hp->rszf[f];
    if (f == F_M1 || f == F_M2) {
      const double c2 = hp->rszf[F_C2], d1 = hp->rszf[F_D1];
      lo = __dmul_rn(0.2, c2 < d1 ? c2 : d1);
    }
    if (!(__dmul_rn(lo, hp->be[f]) > 1e-150)) pos = 0;
  }
  hp->pos = pos;
}

// per cell: slope factor and the upslope direction (aspect is the downslope azimuth)
__device__ inline void cell_prep(double gs, double aspect_deg, CellPrep *cp) {
  double sf = 1.0;
  if (gs > 0.0) {
    const double g = __ddiv_rn(gs < 60.0 ? gs : 60.0, 100.0);
    sf = dexp(__dmul_rn(3.533, dpow(g, 1.2)));
  }
  cp->sf = sf;
  dsincos_deg(__dadd_rn(aspect_deg, 180.0), &cp->sin_s, &cp->cos_s);
}

struct FbpOut { double hros, bros, lb, fros, a, e, ux, uy, wsv, wse; double ros[8]; };

// Sec. 3.7, Eqs. (2)-(4): the ellipse of a cell from HROS, BROS and LB, and
// its rate along each of the 8 axes for the head direction (ux, uy) (unit
// vector, x east, y north) by Eq. (1) (ellipse_mode 0) or by the ray from the
// ignition point (mode 1).  Sets o->lb, fros, a, e, ux, uy and ros[].
__device__ __forceinline__ void ellipse_axes(double hros, double bros, double lb, double ux, double uy,
                                             int ellipse_mode, FbpOut *o) {
  const double hb = __dadd_rn(hros, bros);
  const double ilb = __ddiv_rn(1.0, lb);   // one reciprocal for FROS and e
  const double fros = __dmul_rn(__dmul_rn(hb, ilb), 0.5);
  const double a = __dmul_rn(hb, 0.5);
  const double e = __dsqrt_rn(__dsub_rn(1.0, __dmul_rn(ilb, ilb)));
  o->lb = lb; o->fros = fros; o->a = a; o->e = e; o->ux = ux; o->uy = uy;
  // cos(phi_k) = (cos theta_k) ux + (sin theta_k) uy for the 8 axes, whose
  // cosines and sines are 0, +-1 and +-h (h = RN(sqrt(1/2))): products by 0 and
  // +-1 are exact, so the sums are ux, uy, their negatives and +-(h ux) +- (h uy)
  // -- the same values (up to the sign of a zero, which no test below sees)
  const double h = 0x1.6a09e667f3bcdp-1;
  const double hx = __dmul_rn(h, ux), hy = __dmul_rn(h, uy);
  const double dpp = __dadd_rn(hx, hy), dmp = __dsub_rn(hy, hx);
  const double cphk[8] = {ux, dpp, uy, dmp, -ux, -dpp, -uy, -dmp};
  if (ellipse_mode == 0) {
    const double A = __dmul_rn(a, __dsub_rn(1.0, __dmul_rn(e, e)));
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double cphi = cphk[k];
      // cphi > 0 as a sign test on the bits (cphi is never NaN)
      o->ros[k] = (__double_as_longlong(cphi) > 0) ? __ddiv_rn(A, __dsub_rn(1.0, __dmul_rn(e, cphi))) : A;
    }
  } else {
    // the ray from the ignition point, c = (HROS - BROS)/2 behind the centre,
    // to the ellipse with semi-axes a and b = FROS:
    //   r = (b^2 c cos + a b sqrt(Q)) / (b^2 cos^2 + a^2 sin^2),
    //   Q = b^2 cos^2 + (a^2 - c^2) sin^2, a^2 - c^2 = HROS BROS;
    // on the back half (cos < 0), the same ray multiplied out by the conjugate
    // of its numerator, r = b^2 HROS BROS / (a b sqrt(Q) - b^2 c cos), so that
    // no nearly equal terms are subtracted when HROS >> BROS
    const double b = fros;
    const double c = __dmul_rn(__dsub_rn(hros, bros), 0.5);
    const double hbp = __dmul_rn(hros, bros);
    const double bb = __dmul_rn(b, b), aa = __dmul_rn(a, a), ab = __dmul_rn(a, b);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double cphi = cphk[k];
      double sphi2 = __dsub_rn(1.0, __dmul_rn(cphi, cphi));
      if (sphi2 < 0.0) sphi2 = 0.0;
      const double bc = __dmul_rn(__dmul_rn(bb, cphi), cphi);
      const double den = __dadd_rn(bc, __dmul_rn(aa, sphi2));
      const double root = __dsqrt_rn(__dadd_rn(bc, __dmul_rn(hbp, sphi2)));
      double r = 0.0;
      if (cphi >= 0.0) {
        if (den > 0.0) r = __ddiv_rn(__dadd_rn(__dmul_rn(__dmul_rn(bb, c), cphi), __dmul_rn(ab, root)), den);
      } else {
        const double q = __dsub_rn(__dmul_rn(ab, root), __dmul_rn(__dmul_rn(bb, c), cphi));
        if (q > 0.0) r = __ddiv_rn(__dmul_rn(bb, hbp), q);
      }
      o->ros[k] = r;
    }
  }
}

// per (cell, hour): FBP surface spread, Eqs. (2)-(4), then the 8 axis rates
// by Eq. (1) (ellipse_mode 0) or by the centre-offset ellipse ray (mode 1).
__device__ inline void fbp_row(int fuel, double gs, const CellPrep &cp, const HourPrep &hp,
                               double pcf, int ellipse_mode, FbpOut *o) {
  const double cf = hp.cf;
  double wse = 0.0;
  if (pos(gs)) {
    const double isf = isf_of(fuel, hp, cp.sf, pcf);
    if (pos(isf)) {
      wse = __dmul_rn(dlog(__dmul_rn(isf, hp.inv_isz)), 1.0 / 0.05039);
      if (gt_c(wse, 40.0)) {
        if (isf < __dmul_rn(__dmul_rn(0.999, 2.496), hp.ff))
          wse = __dsub_rn(28.0, __ddiv_rn(dlog(__dsub_rn(1.0, __ddiv_rn(isf, __dmul_rn(2.496, hp.ff)))),
                                          0.0818));
        else
          wse = 112.45;
      }
    }
  }
  const double wsx = __dadd_rn(hp.wsx_w, __dmul_rn(wse, cp.sin_s));
  const double wsy = __dadd_rn(hp.wsy_w, __dmul_rn(wse, cp.cos_s));
  const double wsv = __dsqrt_rn(__dadd_rn(__dmul_rn(wsx, wsx), __dmul_rn(wsy, wsy)));
  double ux = 1.0, uy = 0.0;
  if (pos(wsv)) {
    const double iw = __ddiv_rn(1.0, wsv);
    ux = __dmul_rn(wsx, iw);
    uy = __dmul_rn(wsy, iw);
  }
  const double isi = __dmul_rn(hp.isz, wind_fn(wsv));
  const double be = hp.be[fuel];
  const double hros = __dmul_rn(rsi_of(fuel, isi, pcf, cf), be);
  const double bisi = __dmul_rn(hp.isz, dexp(__dmul_rn(-0.05039, wsv)));
  const double bros = __dmul_rn(rsi_of(fuel, bisi, pcf, cf), be);
  double lb;
  if (is_o1(fuel))
    lb = !lt_c(wsv, 1.0) ? __dmul_rn(1.1, dpow_n2(wsv, 0.464, 0)) : 1.0;
  else
    lb = __dadd_rn(1.0, __dmul_rn(8.729, dpow_n2(__dsub_rn(1.0, dexp(__dmul_rn(-0.030, wsv))), 2.155, 0)));
  o->hros = hros; o->bros = bros; o->wsv = wsv; o->wse = wse;
  ellipse_axes(hros, bros, lb, ux, uy, ellipse_mode, o);
}

// 2^32 fixed point of a non-negative real: 0 for non-positive / NaN, capped at
// 2^62.  The conversion saturates (and gives INT64_MIN for NaN), so clamping
// the integer gives the same result as testing x first, without FP64 compares.
__device__ __forceinline__ int64_t fixed_of(double x) {
  const long long v = __double2ll_rn(x);
  return v <= 0 ? 0 : (v >= 4611686018427387904LL ? 4611686018427387904LL : (int64_t)v);
}

}  // namespace c2f
