"""Plain evaluation of one rate-of-spread table row (test helper, no oracle code).

The FBP surface-spread chain the fire model takes its rates from (Sec. 2.3,
3.1 assumption A2; the FBP equations themselves are not printed in the paper)
followed by the ellipse of Sec. 3.7 (Eqs. 2-4) and the directional rates of
Eq. (1), written the straightforward way: true divisions, ``x ** y`` powers
and the backend's own exp / log / sqrt / sin / cos.  Nothing here uses the
rounded reciprocals, table-driven exp / log or half-integer power shortcuts
that the oracle and the GPU library use to save work, so comparing them with
this evaluation bounds what those choices cost (1e-12 relative, the table
tolerance) and checks their branch structure.

The backend is either ``mpmath`` (``MP``, 120-bit working precision) or the
C library through Python floats (``LIBM``).  This module imports nothing from
``oracle/`` or from the GPU package.
"""
from __future__ import annotations

import math

# grid code -> (a, b, c, q, BUI0) of the RSI curve and the build-up effect;
# Table 1 of the paper maps code 1 -> C-1, 2 -> C-2, 3 -> C-3 and the codes
# continue through the FBP fuel types; M1 / M2 mix the C2 and D1 curves.
COEF = {
    1: (90.0, 0.0649, 4.5, 0.90, 72.0),     # C1
    2: (110.0, 0.0282, 1.5, 0.70, 64.0),    # C2
    3: (110.0, 0.0444, 3.0, 0.75, 62.0),    # C3
    4: (110.0, 0.0293, 1.5, 0.80, 66.0),    # C4
    5: (30.0, 0.0697, 4.0, 0.80, 56.0),     # C5
    6: (30.0, 0.0800, 3.0, 0.80, 62.0),     # C6
    7: (45.0, 0.0305, 2.0, 0.85, 106.0),    # C7
    8: (30.0, 0.0232, 1.6, 0.90, 32.0),     # D1
    9: (None, None, None, 0.80, 50.0),      # M1
    10: (None, None, None, 0.80, 50.0),     # M2
    11: (190.0, 0.0310, 1.4, 1.0, 1.0),     # O1a
    12: (250.0, 0.0350, 1.7, 1.0, 1.0),     # O1b
    13: (75.0, 0.0297, 1.3, 0.75, 38.0),    # S1
    14: (40.0, 0.0438, 1.7, 0.75, 63.0),    # S2
    15: (55.0, 0.0829, 3.2, 0.75, 31.0),    # S3
}
C2, D1, M1, M2, O1A, O1B = 2, 8, 9, 10, 11, 12


class _Libm:
    name = "libm"

    @staticmethod
    def num(x):
        return float(x)

    exp = staticmethod(math.exp)
    log = staticmethod(math.log)
    sqrt = staticmethod(math.sqrt)

    @staticmethod
    def sincos_deg(d):
        r = math.radians(d % 360.0)
        return math.sin(r), math.cos(r)


class _Mp:
    name = "mpmath"

    def __init__(self):
        import mpmath
        self.m = mpmath.mp.clone()
        self.m.prec = 120

    def num(self, x):
        return self.m.mpf(x)

    def exp(self, x):
        return self.m.exp(x)

    def log(self, x):
        return self.m.log(x)

    def sqrt(self, x):
        return self.m.sqrt(x)

    def sincos_deg(self, d):
        r = self.m.mpf(d) % 360
        # exact at the quadrant points, where the binary64 implementations are exact too
        q = {0: (0, 1), 90: (1, 0), 180: (0, -1), 270: (-1, 0)}
        if r in q:
            s, c = q[int(r)]
            return self.m.mpf(s), self.m.mpf(c)
        t = r * self.m.pi / 180
        return self.m.sin(t), self.m.cos(t)


LIBM = _Libm()


def mp_backend():
    return _Mp()


def fbp_row(B, fuel, gs, aspect, ws, wd_from, ffmc, bui, pc=50.0, curing=60.0, ellipse_mode=0,
            conjugate_back=False):
    """HROS, BROS, LB, FROS, a, e, head direction, WSV, WSE and the 8 axis rates
    (axis k at 45 k degrees counter-clockwise from east) of one cell and hour,
    plus the branches taken (for coverage checks).

    ellipse_mode 1 is the ray from the ignition point to the ellipse, written
    as r = (b^2 c cos + a b sqrt(Q)) / (b^2 cos^2 + a^2 sin^2) with
    Q = b^2 cos^2 + (a^2 - c^2) sin^2.  With ``conjugate_back`` the back half
    (cos < 0) uses the same ray multiplied out by the conjugate of its
    numerator, r = b^2 (a^2 - c^2) / (a b sqrt(Q) - b^2 c cos), and
    a^2 - c^2 = HROS BROS: in binary64 the written form loses about
    log2(HROS / BROS) bits there, so the libm evaluation needs it; at 120 bits
    the two agree (checked)."""
    n = B.num
    one = n(1)
    gs, aspect, ws, wd_from, ffmc, bui = map(n, (gs, aspect, ws, wd_from, ffmc, bui))
    pcf = n(pc) / 100
    branch = {}

    def curve(code, isi):            # RSI = a (1 - e^{-b ISI})^c
        a, b, c = (n(v) for v in COEF[code][:3])
        return a * (one - B.exp(-b * isi)) ** c

    # O1 curing factor
    C = n(curing)
    branch["curing_low"] = bool(C < n(58.8))
    cf = n(0.005) * (B.exp(n(0.061) * C) - 1) if C < n(58.8) else n(0.176) + n(0.02) * (C - n(58.8))

    def rsi(isi):
        if fuel == M1:
            return pcf * curve(C2, isi) + (1 - pcf) * curve(D1, isi)
        if fuel == M2:
            return pcf * curve(C2, isi) + n(0.2) * (1 - pcf) * curve(D1, isi)
        if fuel in (O1A, O1B):
            return curve(fuel, isi) * cf
        return curve(fuel, isi)

    # FFMC moisture, f(F), zero-wind ISI
    m = n(147.2) * (n(101) - ffmc) / (n(59.5) + ffmc)
    ff = n(91.9) * B.exp(n(-0.1386) * m) * (one + m ** n(5.31) / n(4.93e7))
    isz = n(0.208) * ff

    def fw(w):                        # f(W), with the saturating branch above 40 km/h
        if w <= n(40):
            return B.exp(n(0.05039) * w)
        return n(12) * (one - B.exp(n(-0.0818) * (w - n(28))))

    # build-up effect
    if fuel in (O1A, O1B):
        be = one
    else:
        q, bui0 = n(COEF[fuel][3]), n(COEF[fuel][4])
        be = B.exp(n(50) * B.log(q) * (one / bui - one / bui0))

    # slope: slope factor, ISF by inverting the RSI curve(s), slope-equivalent wind
    def isf_curve(code, mult, rsf):
        if not rsf > 0:
            return n(0)
        a, b, c = (n(v) for v in COEF[code][:3])
        x = one - (rsf / (a * mult)) ** (one / c)
        if x < n(0.01):
            branch["isf_guard"] = True
            x = n(0.01)
        return B.log(x) / (-b)

    wse = n(0)
    branch["sloped"] = bool(gs > 0)
    if gs > 0:
        g = (gs if gs < n(60) else n(60)) / 100
        sf = B.exp(n(3.533) * g ** n(1.2))
        if fuel == M1:
            isf = (pcf * isf_curve(C2, one, curve(C2, isz) * sf)
                   + (1 - pcf) * isf_curve(D1, one, curve(D1, isz) * sf))
        elif fuel == M2:
            isf = (pcf * isf_curve(C2, one, curve(C2, isz) * sf)
                   + (1 - pcf) * isf_curve(D1, n(0.2), n(0.2) * curve(D1, isz) * sf))
        elif fuel in (O1A, O1B):
            isf = isf_curve(fuel, cf, curve(fuel, isz) * cf * sf)
        else:
            isf = isf_curve(fuel, one, curve(fuel, isz) * sf)
        if isf > 0:
            wse = B.log(isf / isz) / n(0.05039)
            if wse > n(40):
                if isf < n(0.999) * n(2.496) * ff:
                    branch["wse_high"] = "formula"
                    wse = n(28) - B.log(one - isf / (n(2.496) * ff)) / n(0.0818)
                else:
                    branch["wse_high"] = "cap"
                    wse = n(112.45)

    # net wind vector: wind toward WD + 180, upslope toward aspect + 180
    sw, cw = B.sincos_deg(wd_from + 180)
    ss, cs = B.sincos_deg(aspect + 180)
    wsx = ws * sw + wse * ss
    wsy = ws * cw + wse * cs
    wsv = B.sqrt(wsx * wsx + wsy * wsy)
    ux, uy = (wsx / wsv, wsy / wsv) if wsv > 0 else (one, n(0))
    branch["wind_high"] = bool(wsv > n(40))

    hros = rsi(isz * fw(wsv)) * be
    bros = rsi(isz * B.exp(n(-0.05039) * wsv)) * be
    if fuel in (O1A, O1B):
        branch["o1_wsv_ge_1"] = bool(wsv >= 1)
        lb = n(1.1) * wsv ** n(0.464) if wsv >= 1 else one
    else:
        lb = one + n(8.729) * (one - B.exp(n(-0.030) * wsv)) ** n(2.155)

    # Eqs. (2)-(4)
    fros = (hros + bros) / (2 * lb)
    a = (hros + bros) / 2
    e = B.sqrt(one - one / (lb * lb))
    h = B.sqrt(n(0.5))
    ct = [one, h, n(0), -h, -one, -h, n(0), h]
    st = [n(0), h, one, h, n(0), -h, -one, -h]
    ros = []
    for k in range(8):
        cphi = ct[k] * ux + st[k] * uy
        if ellipse_mode == 0:       # Eq. (1)
            ros.append(a * (1 - e * e) / (1 - e * cphi) if cphi > 0 else a * (1 - e * e))
        else:                       # ray from the ignition point, c behind the centre
            b = fros
            c = (hros - bros) / 2
            s2 = 1 - cphi * cphi
            if s2 < 0:
                s2 = n(0)
            den = b * b * cphi * cphi + a * a * s2
            if conjugate_back:
                q = B.sqrt(b * b * cphi * cphi + hros * bros * s2)
                if cphi >= 0:
                    ros.append((b * b * c * cphi + a * b * q) / den if den > 0 else n(0))
                else:
                    d = a * b * q - b * b * c * cphi
                    ros.append(b * b * hros * bros / d if d > 0 else n(0))
            else:
                ros.append((b * b * c * cphi + a * b * B.sqrt(b * b * cphi * cphi + (a * a - c * c) * s2))
                           / den if den > 0 else n(0))
    return dict(hros=hros, bros=bros, lb=lb, fros=fros, a=a, e=e, ux=ux, uy=uy, wsv=wsv, wse=wse,
                ros8=ros, branch=branch)
