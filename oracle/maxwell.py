"""Sec. 3.1: Maxwell construction of the liquid-vapour coexistence curve of the van der Waals
fluid P^w = 3 rho T / (3 - rho) - 9 rho^2 / 8 (critical point rho_c = T_c = 1, P_c = 3/8).

Written as the equal-area rule on the isotherm in the specific volume v = 1/rho:
the saturation pressure P_s is the pressure at which the outer roots v_l < v_v of
P(v) = P_s satisfy  integral_{v_l}^{v_v} (P(v) - P_s) dv = 0.
"""
import numpy as np
from scipy.integrate import quad
from scipy.optimize import brentq, minimize_scalar

from .model import pressure_vdw


def _outer_roots(P, T):
    # P(rho) = P  <=>  9/8 rho^3 - 27/8 rho^2 + (3T + P) rho - 3P = 0, rho in (0, 3)
    r = np.roots([9.0 / 8.0, -27.0 / 8.0, 3.0 * T + P, -3.0 * P])
    r = np.sort(r[(np.abs(r.imag) < 1e-9) & (r.real > 0) & (r.real < 3)].real)
    return r[0], r[-1]


def coexistence(T):
    """Coexisting (rho_liquid, rho_vapour) at temperature T < 1."""
    if not (0.0 < T < 1.0):
        raise ValueError("coexistence needs 0 < T < T_c = 1")
    # spinodal pressures: local min (liquid side) and local max (vapour side) of P(rho)
    pmax = -minimize_scalar(lambda r: -pressure_vdw(r, T), bounds=(1e-6, 1.0), method="bounded").fun
    pmin = minimize_scalar(lambda r: pressure_vdw(r, T), bounds=(1.0, 2.999), method="bounded").fun
    lo, hi = max(pmin, 1e-12), pmax

    def area(Ps):
        rv, rl = _outer_roots(Ps, T)
        val, _ = quad(lambda v: pressure_vdw(1.0 / v, T) - Ps, 1.0 / rl, 1.0 / rv,
                      epsabs=1e-14, epsrel=1e-13, limit=200)
        return val

    eps = 1e-9 * (hi - lo)
    Ps = brentq(area, lo + eps, hi - eps, xtol=1e-15, rtol=1e-14, maxiter=200)
    rv, rl = _outer_roots(Ps, T)
    return rl, rv
