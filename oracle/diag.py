"""Global diagnostics of a state: total mass, momentum, total energy and maximum speed, and
the circularly averaged structure factor of the density.

Total energy density (Sec. 2.2, after the recovered equations):
    e_T = rho T - 9 rho^2 / 8 + K |grad rho|^2 / 2 + rho u^2 / 2,
with grad rho taken by the spectral scheme of Eq. (3) (the run's k_eff series and window). Totals are sums over nodes
times the cell area dx dy.
"""
import numpy as np

from .dvm import moments
from .wfft import spectral_deriv


def shell_index(nx, ny):
    """Shell b of each 2D DFT index (my, mx): b = round(|q|), q = (mx N/nx, my N/ny), N = max(nx, ny),
    with mx, my the signed DFT indices in [-n/2, n/2) (|q| in units of 2 pi / L of the longer axis)."""
    N = max(nx, ny)
    mx = np.fft.fftfreq(nx) * nx * (N / nx)
    my = np.fft.fftfreq(ny) * ny * (N / ny)
    return np.rint(np.sqrt(mx[None, :] ** 2 + my[:, None] ** 2)).astype(np.int64)


def structure_factor(rho, nbins):
    """Circularly averaged structure factor of the density (the domain-growth measure of the
    phase-separation runs, Sec. 3.2): S(b) = mean over shell b of |rho_hat(m)|^2 / (nx ny),
    rho_hat the unnormalised 2D DFT of rho - mean(rho). Returns (S, count) for b < nbins."""
    ny, nx = rho.shape
    P = np.abs(np.fft.fft2(rho - rho.mean())) ** 2 / (nx * ny)
    b = shell_index(nx, ny).ravel()
    keep = b < nbins
    tot = np.bincount(b[keep], weights=P.ravel()[keep], minlength=nbins)[:nbins]
    cnt = np.bincount(b[keep], minlength=nbins)[:nbins].astype(np.float64)
    S = np.divide(tot, cnt, out=np.zeros(nbins), where=cnt > 0)
    return S, cnt


def diagnostics(dvm, f, p):
    rho, ux, uy, T = moments(dvm, f, p.b)
    rx = spectral_deriv(rho, 1, 0, p.dx, p.dy, p.win_alpha, p.win_p, p.keff_terms, p.deriv)
    ry = spectral_deriv(rho, 0, 1, p.dx, p.dy, p.win_alpha, p.win_p, p.keff_terms, p.deriv)
    u2 = ux * ux + uy * uy
    eT = rho * T - 9.0 / 8.0 * rho * rho + 0.5 * p.K * (rx * rx + ry * ry) + 0.5 * rho * u2
    cell = p.dx * p.dy
    return dict(mass=rho.sum() * cell, px=(rho * ux).sum() * cell, py=(rho * uy).sum() * cell,
                energy=eT.sum() * cell, umax=float(np.sqrt(u2.max())))
