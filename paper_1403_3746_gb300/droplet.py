"""Large deformation of a rectangular droplet (Sec. 3.3), through the library.

A rectangular droplet of length 118 and height 14 (lattice units) sits at the centre of a
periodic box, liquid 1.462 inside and vapour 0.579 outside, with the temperature held at 0.95
(read as the isothermal mode, LBM_FLAG_ISOTHERMAL with T_iso = 0.95) and the parameters
dx = dy = 0.01, tau = 5 dt = 5e-4, K = 1e-5, q = -0.05. Under surface tension it turns into
a dumbbell, then an oscillating ellipse, and relaxes to a circle; the maximum spurious
velocity settles once the droplet is at rest.

Readings: the box size is not stated (default 256 x 256, which holds the droplet and its
relaxed circle of radius sqrt(118 * 14 / pi) ~ 23 cells with wide margins); the edges of the
rectangle are tanh profiles of width `width` cells (the sharp-edged start is not specified).

The shape is measured by the second moments of the liquid region (rho above the mean of the
two densities): aspect = sqrt(lambda_max / lambda_min) of its coordinate covariance
(118 / 14 = 8.43 at the start, 1 for a circle). The run is on the GPU; this module only drives
it and reduces the moments it returns.
"""
import numpy as np

from . import LBM_FLAG_ISOTHERMAL, LBM_MIXED, Simulation, default_params

SEC33 = dict(tau=5e-4, dt=1e-4, dx=0.01, dy=0.01, K=1e-5, q=-0.05, b=2.0)
RHO_L, RHO_V, T_FIXED = 1.462, 0.579, 0.95


def rectangle(n=256, length=118, height=14, rho_l=RHO_L, rho_v=RHO_V, T=T_FIXED, width=1.0):
    """Initial fields: the rectangle centred in an n x n box, tanh edges."""
    c = n / 2.0
    x = np.arange(n)[None, :] - c + 0.5
    y = np.arange(n)[:, None] - c + 0.5
    sx = 0.5 * (1.0 + np.tanh((length / 2.0 - np.abs(x)) / width))
    sy = 0.5 * (1.0 + np.tanh((height / 2.0 - np.abs(y)) / width))
    rho = rho_v + (rho_l - rho_v) * sx * sy
    z = np.zeros((n, n))
    return rho, z, z.copy(), np.full((n, n), float(T))


def aspect_ratio(rho, rho_l=RHO_L, rho_v=RHO_V):
    """sqrt of the eigenvalue ratio of the coordinate covariance of the liquid region."""
    ny, nx = rho.shape
    w = (rho > 0.5 * (rho_l + rho_v)).astype(np.float64)
    Y, X = np.mgrid[0:ny, 0:nx]
    m = w.sum()
    cx, cy = (w * X).sum() / m, (w * Y).sum() / m
    cov = np.array([[(w * (X - cx) ** 2).sum(), (w * (X - cx) * (Y - cy)).sum()],
                    [(w * (X - cx) * (Y - cy)).sum(), (w * (Y - cy) ** 2).sum()]]) / m
    ev = np.linalg.eigvalsh(cov)
    return float(np.sqrt(ev[1] / ev[0]))


def deform(steps, sample_every, n=256, precision=LBM_MIXED, params=None, width=1.0):
    """Runs the rectangle for `steps` steps; returns samples (t, aspect, max |u|, mass) every
    `sample_every` steps, including t = 0."""
    kw = dict(SEC33, **(params or {}))
    p = default_params(precision=precision, flags=LBM_FLAG_ISOTHERMAL, T_iso=T_FIXED, **kw)
    out = []
    with Simulation(n, n, p) as sim:
        sim.init(*rectangle(n, width=width))
        done = 0
        while True:
            rho = sim.moments()[0]
            if not np.isfinite(rho).all():
                out.append(dict(t=done * kw["dt"], aspect=float("nan"), umax=float("nan"), mass=float("nan"),
                                finite=False))
                break
            d = sim.diagnostics()
            out.append(dict(t=done * kw["dt"], aspect=aspect_ratio(rho), umax=d["umax"], mass=d["mass"],
                            finite=True))
            if done >= steps:
                break
            k = min(sample_every, steps - done)
            sim.step(k)
            done += k
    return out
