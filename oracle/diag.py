"""Global diagnostics of a state: total mass, momentum, total energy and maximum speed.

Total energy density (Sec. 2.2, after the recovered equations):
    e_T = rho T - 9 rho^2 / 8 + K |grad rho|^2 / 2 + rho u^2 / 2,
with grad rho taken by the spectral scheme of Eq. (3). Totals are sums over nodes
times the cell area dx dy.
"""
import numpy as np

from .dvm import moments
from .wfft import spectral_deriv


def diagnostics(dvm, f, p):
    rho, ux, uy, T = moments(dvm, f, p.b)
    rx = spectral_deriv(rho, 1, 0, p.dx, p.dy, p.win_alpha, p.win_p)
    ry = spectral_deriv(rho, 0, 1, p.dx, p.dy, p.win_alpha, p.win_p)
    u2 = ux * ux + uy * uy
    eT = rho * T - 9.0 / 8.0 * rho * rho + 0.5 * p.K * (rx * rx + ry * ry) + 0.5 * rho * u2
    cell = p.dx * p.dy
    return dict(mass=rho.sum() * cell, px=(rho * ux).sum() * cell, py=(rho * uy).sum() * cell,
                energy=eT.sum() * cell, umax=float(np.sqrt(u2.max())))
