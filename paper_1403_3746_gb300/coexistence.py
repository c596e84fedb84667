"""Liquid-vapour coexistence curve by the protocol of Sec. 3.1, through the library.

A quasi-one-dimensional periodic box (512 x 2) starts as vapour | liquid | vapour
(rho_v = 0.955 for x <= N/4, rho_l = 1.045 for N/4 < x <= 3N/4, rho_v beyond) at T0 = 0.9975,
u = 0, with the parameters of Sec. 3.1 (tau = 1e-4, dt = 5e-5, dx = dy = 0.02, K = 1e-5, H = 0,
zeta = 0, q = -0.004, b = 2). Once the state is at equilibrium the temperature is lowered by
a small amount and the run continues from the current density profile: f is reset to
f^eq(rho, u, T_new) (lbm_init with the current rho and u and a uniform T_new). At each
temperature the coexisting densities are the bulk means of the liquid (centre) and vapour
(edges) regions; they are compared with the Maxwell construction (lbm_maxwell).

Equilibrium: after at least `min_steps` steps, the bulk densities change by less than `tol`
(absolute) between two checks `check_every` steps apart. Near the critical point the
relaxation is very slow (the start state of Sec. 3.1 lies inside the spinodal at T0 = 0.9975
but the densities move by ~1e-4 in 2e5 steps), so a short window can mistake slow
coarsening for equilibrium; `coexistence_parallel` instead starts every temperature from its
Maxwell densities in the same layout and runs all of them as one batch. The runs are on the
GPU; this module only drives them and reduces the moments they return.
"""
import numpy as np

from . import LBM_FLAG_ISOTHERMAL, LBM_MIXED, Batch, Simulation, default_params, maxwell

SEC31 = dict(tau=1e-4, dt=5e-5, dx=0.02, dy=0.02, K=1e-5, H=0.0, zeta=0.0, q=-0.004, b=2.0)
RHO_V0, RHO_L0, T_START = 0.955, 1.045, 0.9975


def initial_profile(nx=512, ny=2, rho_v=RHO_V0, rho_l=RHO_L0, T=T_START):
    """Sec. 3.1: vapour for x <= nx/4, liquid for nx/4 < x <= 3 nx/4, vapour beyond (x = 1..nx)."""
    x = np.arange(1, nx + 1)
    rho = np.where((x > nx // 4) & (x <= 3 * nx // 4), rho_l, rho_v)[None, :] * np.ones((ny, 1))
    z = np.zeros((ny, nx))
    return rho, z, z.copy(), np.full((ny, nx), float(T))


def bulk_densities(rho):
    """Mean density over the central eighth (liquid) and the outer eighth (vapour) of x."""
    r = rho.mean(axis=0)
    nx = r.size
    w = max(nx // 16, 1)
    return float(r[nx // 2 - w: nx // 2 + w].mean()), float(np.concatenate([r[:w], r[nx - w:]]).mean())


def _settle(sim, check_every, tol, min_steps, max_steps):
    rl, rv = bulk_densities(sim.moments()[0])
    steps = 0
    while steps < max_steps:
        sim.step(check_every)
        steps += check_every
        nl, nv = bulk_densities(sim.moments()[0])
        if not (np.isfinite(nl) and np.isfinite(nv)):
            return nl, nv, steps, False
        if steps >= min_steps and abs(nl - rl) < tol and abs(nv - rv) < tol:
            return nl, nv, steps, True
        rl, rv = nl, nv
    return rl, rv, steps, False


def coexistence_curve(temps, nx=512, ny=2, precision=LBM_MIXED, params=None, check_every=5000, tol=1e-6,
                      min_steps=100000, max_steps=400000, isothermal=False, start=None):
    """The stepwise protocol of Sec. 3.1 over the decreasing temperatures `temps` (the first
    is the start temperature). Returns one dict per temperature: T, rho_l, rho_v (bulk), the
    Maxwell pair, steps taken, and whether equilibrium was reached within max_steps."""
    kw = dict(SEC31, **(params or {}))
    out = []
    fields = start if start is not None else initial_profile(nx, ny, T=temps[0])
    for T in temps:
        flags = LBM_FLAG_ISOTHERMAL if isothermal else 0
        p = default_params(precision=precision, flags=flags, T_iso=float(T) if isothermal else 0.0, **kw)
        with Simulation(nx, ny, p) as sim:
            sim.init(fields[0], fields[1], fields[2], np.full((ny, nx), float(T)))
            rl, rv, steps, ok = _settle(sim, check_every, tol, min_steps, max_steps)
            rho, ux, uy, _ = sim.moments()
        finite = bool(np.isfinite(rho).all())
        ml, mv = maxwell(T)
        out.append(dict(T=float(T), rho_l=rl, rho_v=rv, maxwell_rho_l=ml, maxwell_rho_v=mv, steps=steps,
                        equilibrium=ok, finite=finite))
        if not finite:
            break
        fields = (rho, ux, uy)
    return out


def coexistence_parallel(temps, nx=512, ny=2, precision=LBM_MIXED, params=None, steps=100000):
    """All temperatures at once as one batch (each instance starts from the Maxwell densities
    at its own temperature in the Sec. 3.1 layout) for `steps` steps. Returns per temperature
    the bulk densities, the Maxwell pair and the relative deviations."""
    kw = dict(SEC31, **(params or {}))
    out = []
    with Batch([(nx, ny)] * len(temps), default_params(precision=precision, **kw)) as b:
        for k, T in enumerate(temps):
            ml, mv = maxwell(T)
            b.init(k, *initial_profile(nx, ny, rho_v=mv, rho_l=ml, T=T))
        b.step(steps)
        for k, T in enumerate(temps):
            rl, rv = bulk_densities(b.moments(k)[0])
            ml, mv = maxwell(T)
            out.append(dict(T=float(T), rho_l=rl, rho_v=rv, maxwell_rho_l=ml, maxwell_rho_v=mv,
                            rel_l=abs(rl / ml - 1), rel_v=abs(rv / mv - 1)))
    return out
