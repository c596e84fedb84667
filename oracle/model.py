"""Sec. 2.2 and Sec. 2.3: the kinetic equation with the Gonnella-Lamura-Sofonea forcing term,
and its two-stage Runge-Kutta time step.

Eq. (1):  d f_i/dt + v_i . grad f_i = -(f_i - f_i^eq)/tau + I_i
Eq. (2):  I_i = -[A + B . (v_i - u) + (C + C_q) |v_i - u|^2] f_i^eq
with A = -2 (C + C_q) T, B, C and C_q as printed after Eq. (2), the van der Waals EOS
P^w = 3 rho T / (3 - rho) - 9 rho^2 / 8 and the stress
Lambda = M grad rho grad rho - M (rho lap rho + |grad rho|^2 / 2) I - [rho T grad rho . grad(M/T)] I,
M = K + H T (Sec. 2.2, the text after the recovered Navier-Stokes equations).

Readings:
* B is (1/(rho T)) div S with S = (P^w - rho T - zeta div u) I + Lambda, and C_q is
  (1/(rho T^2)) div Q with Q = q rho T grad T: both divergences are taken spectrally from
  the flux fields, since the paper computes all spatial derivatives by the FFT scheme.
* grad(M/T) = -K grad T / T^2 (chain rule on M/T = K/T + H), so only grad T is needed.
* In C the term printed "-zeta (div u)" is read as -zeta (div u)^2 (bulk dissipation);
  every run here has zeta = 0.
* grad rho . grad u . grad rho = sum_{a,b} d_a rho (d_a u_b) d_b rho.
* The printed Runge-Kutta stages (Sec. 2.3) carry a sign inconsistent with Eq. (1). The
  stages follow Eq. (1): with R(f) = -v . grad f - (f - f^eq)/tau + I,
  f^{n+1/2} = f^n + (dt/2) R(f^n) and f^{n+1} = f^n + dt R(f^{n+1/2}), where f^eq and I
  of each stage are built from the moments of that stage's f.

Numerical variants (Sec. 3.2 runs the D2V33 comparison model with the 8th-order modified
wavenumber and the forward Euler scheme): `keff_terms` keeps the first terms of the series
of Eq. (3) (8 = 16th order, 4 = 8th order) and `scheme = "euler"` advances
f^{n+1} = f^n + dt R(f^n). Isothermal mode (the fixed temperature of the droplet runs of
Sec. 3.3): with T_iso > 0, f^eq and I_i of every stage use T = T_iso at every node instead of
the temperature moment of f (the energy equation is replaced by a thermostat; mass and
momentum stay conserved).

Solution filter (filter_alpha > 0; a second reading of the "windowed" FFT scheme): after each
step every f_i is replaced by the inverse transform of W(m_x) W(m_y) times its spectrum, with
the window W of wfft.window. The paper prints no filter, so against the paper this is
"parity unpinned"; tests pin it to this definition on single Fourier modes.
"""
from dataclasses import dataclass

import numpy as np

from .dvm import D2V16, moment_matrix, feq, moments
from .wfft import spectral_deriv, window

_MINV = {}


def _minv(dvm):
    key = float(dvm.eta[0])
    if key not in _MINV:
        _MINV[key] = np.linalg.inv(moment_matrix(dvm))
    return _MINV[key]


@dataclass
class Params:
    """Model and discretisation parameters (Sec. 2.2, Sec. 3). The defaults are the
    phase-separation set of Sec. 3.2 (tau = dt = 1e-4, dx = dy = 1/256, K = 5e-6) with
    q = -0.004 and b = 2 from Sec. 3.1. `force`, `collide` and `advect` switch the
    three terms of Eq. (1) on or off (test hooks). `deriv` selects how the derivative
    operator of Eq. (3) is applied: "fft" (numpy's FFT of the field) or "dft" (explicit DFT
    sums along each axis, the same operator with O(N) work per value). `filter_alpha` > 0 ends
    every step with the solution filter of window exponent (filter_alpha, filter_p)."""
    tau: float = 1e-4
    dt: float = 1e-4
    dx: float = 1.0 / 256.0
    dy: float = 1.0 / 256.0
    K: float = 5e-6
    H: float = 0.0
    q: float = -0.004
    zeta: float = 0.0
    b: float = 2.0
    eta0: float = 2.5
    win_alpha: float = 0.0
    win_p: float = 36.0
    force: bool = True
    collide: bool = True
    advect: bool = True
    keff_terms: int = 8
    scheme: str = "rk2"
    T_iso: float = 0.0
    deriv: str = "fft"
    filter_alpha: float = 0.0
    filter_p: float = 36.0

    @staticmethod
    def phase_separation():
        """Sec. 3.2 (D2V16 column); q from Sec. 3.1."""
        return Params()

    @staticmethod
    def droplet():
        """Sec. 3.3: dx = dy = 0.01, tau = 5 dt = 5e-4, K = 1e-5, q = -0.05."""
        return Params(tau=5e-4, dt=1e-4, dx=0.01, dy=0.01, K=1e-5, q=-0.05)

    @staticmethod
    def coexistence():
        """Sec. 3.1: tau = 1e-4, dt = 5e-5, dx = dy = 0.02, K = 1e-5, H = 0, zeta = 0, q = -0.004, b = 2."""
        return Params(tau=1e-4, dt=5e-5, dx=0.02, dy=0.02, K=1e-5, q=-0.004)


def pressure_vdw(rho, T):
    """Sec. 2.2: van der Waals EOS P^w = 3 rho T / (3 - rho) - 9 rho^2 / 8."""
    return 3.0 * rho * T / (3.0 - rho) - 9.0 / 8.0 * rho * rho


def forcing_terms(dvm, rho, ux, uy, T, fe, p):
    """Eq. (2) and the coefficient definitions after it. Returns I (16, ny, nx) and a dict
    of the intermediate fields (A, B_x, B_y, C, C_q, ...)."""
    def D(h, ox, oy):
        return spectral_deriv(h, ox, oy, p.dx, p.dy, p.win_alpha, p.win_p, p.keff_terms, p.deriv)

    # spatial derivatives of the macroscopic fields
    rx, ry = D(rho, 1, 0), D(rho, 0, 1)
    lap = D(rho, 2, 0) + D(rho, 0, 2)
    dux_dx, dux_dy = D(ux, 1, 0), D(ux, 0, 1)
    duy_dx, duy_dy = D(uy, 1, 0), D(uy, 0, 1)
    divu = dux_dx + duy_dy
    ddivu_x = D(ux, 2, 0) + D(uy, 1, 1)
    ddivu_y = D(ux, 1, 1) + D(uy, 0, 2)
    Tx, Ty = D(T, 1, 0), D(T, 0, 1)

    # local thermodynamics: EOS, M = K + H T, grad(M/T) = -K grad T / T^2, stress Lambda
    Pw = pressure_vdw(rho, T)
    M = p.K + p.H * T
    gx, gy = -p.K * Tx / (T * T), -p.K * Ty / (T * T)
    grr = rx * rx + ry * ry
    iso = M * (rho * lap + 0.5 * grr) + rho * T * (rx * gx + ry * gy)
    Lxx = M * rx * rx - iso
    Lxy = M * rx * ry
    Lyy = M * ry * ry - iso

    # fluxes whose divergences give B and C_q
    Pn = Pw - rho * T - p.zeta * divu
    Sxx, Sxy, Syy = Pn + Lxx, Lxy, Pn + Lyy
    Qx, Qy = p.q * rho * T * Tx, p.q * rho * T * Ty
    divS_x = D(Sxx, 1, 0) + D(Sxy, 0, 1)
    divS_y = D(Sxy, 1, 0) + D(Syy, 0, 1)
    divQ = D(Qx, 1, 0) + D(Qy, 0, 1)

    rT = rho * T
    Bx, By = divS_x / rT, divS_y / rT
    L_gradu = Lxx * dux_dx + Lxy * (duy_dx + dux_dy) + Lyy * duy_dy
    r_gradu_r = rx * (dux_dx * rx + duy_dx * ry) + ry * (dux_dy * rx + duy_dy * ry)
    C = ((Pw - rT) * divu + L_gradu - p.zeta * divu * divu + 9.0 / 8.0 * rho * rho * divu
         + p.K * (-0.5 * grr * divu - rho * (rx * ddivu_x + ry * ddivu_y) - r_gradu_r)) / (2.0 * rT * T)
    Cq = divQ / (rT * T)
    A = -2.0 * (C + Cq) * T

    cx = dvm.vx[:, None, None] - ux[None]
    cy = dvm.vy[:, None, None] - uy[None]
    I = -(A[None] + Bx[None] * cx + By[None] * cy + (C + Cq)[None] * (cx * cx + cy * cy)) * fe
    extra = dict(A=A, Bx=Bx, By=By, C=C, Cq=Cq, Pw=Pw, rx=rx, ry=ry, lap=lap, divu=divu,
                 Sxx=Sxx, Sxy=Sxy, Syy=Syy, Qx=Qx, Qy=Qy, divS_x=divS_x, divS_y=divS_y, divQ=divQ)
    return I, extra


def advection(dvm, f, p):
    """v_i . grad f_i for all 16 fields (Eq. (1) left side), by the FFT scheme of Eq. (3)."""
    out = np.empty_like(f)
    for i in range(16):
        out[i] = dvm.vx[i] * spectral_deriv(f[i], 1, 0, p.dx, p.dy, p.win_alpha, p.win_p, p.keff_terms, p.deriv) \
            + dvm.vy[i] * spectral_deriv(f[i], 0, 1, p.dx, p.dy, p.win_alpha, p.win_p, p.keff_terms, p.deriv)
    return out


def rhs(dvm, f, p):
    """R(f) = -v . grad f - (f - f^eq)/tau + I, with f^eq and I from the moments of f."""
    rho, ux, uy, T = moments(dvm, f, p.b)
    if p.T_iso > 0.0:
        T = np.full_like(rho, p.T_iso)
    fe = feq(dvm, rho, ux, uy, T, p.b, _minv(dvm))
    R = np.zeros_like(f)
    if p.advect:
        R -= advection(dvm, f, p)
    if p.collide:
        R -= (f - fe) / p.tau
    if p.force:
        I, _ = forcing_terms(dvm, rho, ux, uy, T, fe, p)
        R += I
    return R


def solution_filter(f, p):
    """The window applied to the solution (a reading of the "windowed" FFT scheme, abstract and
    Sec. 2.3): each f_i becomes the inverse transform of W(m_x) W(m_y) times its spectrum, with
    the exponential window W of wfft.window (the Nyquist index included)."""
    ny, nx = f.shape[1:]
    W = window(ny, p.filter_alpha, p.filter_p)[:, None] * window(nx, p.filter_alpha, p.filter_p)[None, :]
    return np.fft.ifft2(W[None] * np.fft.fft2(f, axes=(1, 2)), axes=(1, 2)).real


def rk2_step(dvm, f, p):
    """Sec. 2.3: two-stage (midpoint) Runge-Kutta step of Eq. (1); the forward Euler step
    f + dt R(f) when p.scheme == "euler". With p.filter_alpha > 0 the step ends with the
    solution filter."""
    if p.scheme == "euler":
        out = f + p.dt * rhs(dvm, f, p)
    else:
        fh = f + 0.5 * p.dt * rhs(dvm, f, p)
        out = f + p.dt * rhs(dvm, fh, p)
    return solution_filter(out, p) if p.filter_alpha > 0 else out


def init_feq(dvm, rho, ux, uy, T, p):
    """f_i := f_i^eq(rho, u, T) (the initial state of every run; T = T_iso in isothermal mode)."""
    if p.T_iso > 0.0:
        T = np.full_like(rho, p.T_iso)
    return feq(dvm, rho, ux, uy, T, p.b, _minv(dvm))


def run(f, p, steps, dvm=None):
    """Advance f (16, ny, nx) by `steps` Runge-Kutta steps."""
    dvm = dvm or D2V16(p.eta0)
    for _ in range(steps):
        f = rk2_step(dvm, f, p)
    return f
