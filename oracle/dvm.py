"""Sec. 2.1: the D2V16 discrete-velocity model of Kataoka and Tsutahara, its moments and
its discrete equilibrium f_i^eq.

Readings (the paper cites the DVM but does not print it):
* Velocities (not printed): the four speeds of Kataoka and Tsutahara's D2V16 set, 1, 6, sqrt2
  and 3/sqrt2, the first two along the axes and the last two along the diagonals: i = 1..4 are
  (+-1, 0) and (0, +-1); i = 5..8 are (+-6, 0) and (0, +-6); i = 9..12 are (+-1, +-1) (speed
  sqrt2); i = 13..16 are (+-1.5, +-1.5) (speed 3/sqrt2). Within each group the four vectors go
  counter-clockwise starting from the +x axis (groups 1-2) or from the first quadrant
  (groups 3-4). (Reading the diagonal speeds as component values instead, i.e. speeds 2 and 3,
  also gives an invertible moment system, but the droplet runs of Sec. 3.3 then diverge within
  a few hundred steps, while the paper runs them for long times; with these speeds they stay
  bounded.)
* eta_i = eta0 = 2.5 on i = 1..4 and 0 on i = 5..16 (Sec. 2.1).
* The moment definition of the energy in Sec. 2.1 lacks the factor rho; it is read as
  rho (b T + u^2) = sum f_i (v_i^2 + eta_i^2).
* f^eq is "a polynomial of u up to fourth order" (Sec. 2.1) that satisfies the seven
  kinetic moment relations (Sec. 2.2, Chapman-Enskog remark). These relations have 16
  independent components, so f^eq is the unique solution of the 16x16 linear system
  M f^eq = m^eq(rho, u, T) built here. Any closed form that meets the same moments
  equals it.
"""
import numpy as np


class D2V16:
    """Velocity set and extra-degree-of-freedom parameters (Sec. 2.1)."""

    def __init__(self, eta0=2.5):
        v = []
        for c in (1.0, 6.0):
            v += [(c, 0.0), (0.0, c), (-c, 0.0), (0.0, -c)]
        for c in (1.0, 1.5):  # diagonal speeds sqrt2 and 3/sqrt2
            v += [(c, c), (-c, c), (-c, -c), (c, -c)]
        self.v = np.array(v, dtype=np.float64)          # (16, 2)
        self.vx = self.v[:, 0].copy()
        self.vy = self.v[:, 1].copy()
        self.eta = np.zeros(16)
        self.eta[:4] = eta0                              # Sec. 2.1: eta_i = 2.5 for i = 1..4
        self.psi = self.vx ** 2 + self.vy ** 2 + self.eta ** 2


def moment_matrix(dvm):
    """Rows: the 16 moment functionals of the seven kinetic moment relations, in the order
    1; v_x, v_y; psi; v_x v_x, v_x v_y, v_y v_y; psi v_x, psi v_y;
    v_x^3, v_x^2 v_y, v_x v_y^2, v_y^3; psi v_x^2, psi v_x v_y, psi v_y^2,
    with psi = v^2 + eta^2."""
    vx, vy, psi = dvm.vx, dvm.vy, dvm.psi
    rows = [np.ones(16), vx, vy, psi,
            vx * vx, vx * vy, vy * vy,
            psi * vx, psi * vy,
            vx ** 3, vx * vx * vy, vx * vy * vy, vy ** 3,
            psi * vx * vx, psi * vx * vy, psi * vy * vy]
    return np.array(rows)


def equilibrium_moments(rho, ux, uy, T, b):
    """The values the moment functionals take on the equilibrium (moments of a local
    Maxwellian with b degrees of freedom), same order as moment_matrix rows.
    Arguments broadcast; the result has a leading axis of 16."""
    u2 = ux * ux + uy * uy
    e = (b + 2.0) * T + u2          # energy-flux factor
    g = (b + 4.0) * T + u2
    m = [np.ones_like(u2),
         ux, uy,
         b * T + u2,
         T + ux * ux, ux * uy, T + uy * uy,
         ux * e, uy * e,
         3.0 * T * ux + ux ** 3, T * uy + ux * ux * uy, T * ux + ux * uy * uy, 3.0 * T * uy + uy ** 3,
         T * e + g * ux * ux, g * ux * uy, T * e + g * uy * uy]
    return rho * np.array(np.broadcast_arrays(*m))


def feq(dvm, rho, ux, uy, T, b, Minv=None):
    """f_i^eq = M^{-1} m^eq(rho, u, T) at every node. Shape (16,) + rho.shape."""
    if Minv is None:
        Minv = np.linalg.inv(moment_matrix(dvm))
    m = equilibrium_moments(rho, ux, uy, T, b)
    return np.tensordot(Minv, m, axes=(1, 0))


def moments(dvm, f, b):
    """Sec. 2.1: rho = sum f_i, rho u = sum f_i v_i, rho (b T + u^2) = sum f_i (v_i^2 + eta_i^2).
    f has shape (16, ny, nx). Returns rho, u_x, u_y, T."""
    rho = f.sum(axis=0)
    jx = np.tensordot(dvm.vx, f, axes=(0, 0))
    jy = np.tensordot(dvm.vy, f, axes=(0, 0))
    E = np.tensordot(dvm.psi, f, axes=(0, 0))
    ux = jx / rho
    uy = jy / rho
    T = (E / rho - (ux * ux + uy * uy)) / b
    return rho, ux, uy, T
