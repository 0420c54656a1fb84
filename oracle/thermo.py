"""Peng-Robinson thermodynamics for the checks: EOS, critical point and the
Maxwell equal-area construction of the coexistence densities (Sec. 3.1,
Eqs. (PREoS) and (Maxwell_equal_area)).

TEST INFRASTRUCTURE ONLY (part of the oracle).  Plain float64 numpy/scipy.

Maxwell construction, written in specific volume v = 1/rho: the coexistence
pair (v_l, v_v) at saturation pressure P_sat satisfies P(v_l) = P(v_v) = P_sat
and P_sat (v_v - v_l) = int_{v_l}^{v_v} P dv, which is the paper's
int_{rho_v}^{rho_l} (P_sat - P)/rho^2 drho = 0 after the change of variable
drho/rho^2 = -dv.  Peng-Robinson integrates in closed form:

  int P dv = R T ln(v - b) - a alpha/(2 sqrt(2) b) ln((v + b - sqrt(2) b)/(v + b + sqrt(2) b)).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def alpha_of(T_over_Tc: float, acentric: float) -> float:
    m = 0.37464 + 1.54226 * acentric - 0.26992 * acentric ** 2
    return (1.0 + m * (1.0 - math.sqrt(T_over_Tc))) ** 2


def critical_temperature(a: float, b: float, R: float) -> float:
    """From a = 0.45724 R^2 Tc^2 / Pc and b = 0.0778 R Tc / Pc."""
    return 0.0778 * a / (0.45724 * b * R)


def critical_pressure(a: float, b: float, R: float) -> float:
    return 0.0778 * R * critical_temperature(a, b, R) / b


def pressure(rho, a, b, R, T_over_Tc, acentric):
    rho = np.asarray(rho, dtype=np.float64)
    T = T_over_Tc * critical_temperature(a, b, R)
    al = alpha_of(T_over_Tc, acentric)
    return rho * R * T / (1.0 - b * rho) - a * al * rho ** 2 / (1.0 + 2.0 * rho * b - b ** 2 * rho ** 2)


def _p_of_v(v, a, b, R, T, al):
    return R * T / (v - b) - a * al / (v * v + 2.0 * b * v - b * b)


def _int_p_dv(v, a, b, R, T, al):
    s2 = math.sqrt(2.0)
    return R * T * math.log(v - b) - a * al / (2.0 * s2 * b) * math.log((v + b - s2 * b) / (v + b + s2 * b))


def _volume_roots(P, a, b, R, T, al):
    """Real roots v > b of P(v) = P (a cubic in v)."""
    # (P)(v - b)(v^2 + 2bv - b^2) = R T (v^2 + 2bv - b^2) - a al (v - b)
    c3 = P
    c2 = P * (2 * b - b) - R * T
    c1 = P * (-b * b - 2 * b * b) - 2 * b * R * T + a * al
    c0 = P * (b ** 3) + R * T * b * b - a * al * b
    r = np.roots([c3, c2, c1, c0])
    r = np.sort(r[np.abs(r.imag) < 1e-9 * np.abs(r.real)].real)
    return r[r > b]


def maxwell(T_over_Tc: float, a: float = 2.0 / 49.0, b: float = 2.0 / 21.0, R: float = 1.0,
            acentric: float = 0.344):
    """Coexistence densities (rho_v, rho_l) and P_sat by the equal-area rule."""
    T = T_over_Tc * critical_temperature(a, b, R)
    al = alpha_of(T_over_Tc, acentric)
    # spinodal pressures bound the search: local extrema of P(v)
    vs = np.geomspace(b * 1.0001, b * 1e6, 200001)
    Pv = _p_of_v(vs, a, b, R, T, al)
    dP = np.diff(Pv)
    idx = np.where(np.sign(dP[1:]) != np.sign(dP[:-1]))[0] + 1
    if len(idx) < 2:
        raise ValueError("no two-phase region at this temperature")
    p_lo = max(Pv[idx[0]], 1e-300)  # local minimum (liquid spinodal)
    p_hi = Pv[idx[1]]  # local maximum (vapour spinodal)

    def area(P):
        r = _volume_roots(P, a, b, R, T, al)
        vl, vv = r[0], r[-1]
        return P * (vv - vl) - (_int_p_dv(vv, a, b, R, T, al) - _int_p_dv(vl, a, b, R, T, al))

    eps = 1e-12 * (p_hi - p_lo)
    Psat = brentq(area, p_lo + eps, p_hi - eps, xtol=1e-300, rtol=1e-15, maxiter=500)
    r = _volume_roots(Psat, a, b, R, T, al)
    return 1.0 / r[-1], 1.0 / r[0], Psat
