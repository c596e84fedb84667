"""Error of the mixed-precision path (LBM_MIXED) against the plain float64 path (LBM_FP64),
stated per physical result of Sec. 3 on the same seeded inputs:

* coexistence densities of a flat liquid slab (Sec. 3.1), measured in the bulk of each phase;
* relative mass drift over the run;
* pressure jump P_in - P_out of the van der Waals pressure across a static circular droplet
  (the relaxed state of the droplet runs of Sec. 3.3; Laplace law);
* spurious (parasitic) velocity max |u| around that droplet;
and, separately (`laplace_check`), the Laplace law in 2D, P_in - P_out = sigma / R, with the
surface tension of the flat interface sigma = K * integral of (d rho / dn)^2 across it (the
gradient energy of the Korteweg stress of Sec. 2.2), taken from a slab at the droplets'
temperature, and R the droplet's equimolar radius.

Both paths run through the library (each instance set advanced as one batch); the float64
path agrees with the oracle to round-off on short runs, so it stands in for it on runs of
thousands of steps, which the oracle cannot finish quickly. Host-side numpy only reduces the
moments the library returns.
"""
import numpy as np

import synthetic

from . import Batch, LBM_FP64, LBM_MIXED, LBM_MIXED_RHO64, Simulation, default_params, maxwell

PHASE = dict(tau=1e-4, dt=1e-4, dx=1 / 256, dy=1 / 256, K=5e-6, q=-0.004, b=2.0)


def vdw_pressure(rho, T):
    """Van der Waals pressure with a = 9/8, b = 1/3 (Sec. 2.2): P = 3 rho T/(3 - rho) - 9 rho^2/8."""
    return 3.0 * rho * T / (3.0 - rho) - 1.125 * rho * rho


def surface_tension(profile, dx, K):
    """sigma = K * integral (d rho/dx)^2 dx per interface, for a periodic profile rho(x) with
    two interfaces (the slab); the derivative is spectral (exact for the band-limited profile)."""
    n = profile.size
    k = 2.0 * np.pi * np.fft.fftfreq(n, d=dx)
    k[n // 2] = 0.0  # no first derivative at the Nyquist frequency
    d = np.real(np.fft.ifft(1j * k * np.fft.fft(profile)))
    return 0.5 * K * float(np.sum(d * d) * dx)


def equimolar_radius(rho, rho_in, rho_out):
    """Radius (cells) of the disc holding the droplet's excess mass at the inner density."""
    area = float(np.sum((rho - rho_out) / (rho_in - rho_out)))
    return float(np.sqrt(area / np.pi))


def slab_runs(temps, precision, nx=256, ny=2, steps=20000, params=None):
    """Flat slabs (liquid in the middle half of x) at each temperature, advanced `steps` steps.
    Returns per temperature (rho_l, rho_v, mass drift, sigma): bulk means over the central nx/8
    of the liquid and the outer nx/8 of the vapour, and the surface tension of the final
    profile."""
    kw = dict(params or PHASE)
    p = default_params(precision=precision, **kw)
    out = []
    with Batch([(nx, ny)] * len(temps), p) as b:
        mass0 = []
        for k, T in enumerate(temps):
            rl, rv = maxwell(T)
            fields = synthetic.slab(nx, ny, rl, rv, T, center=nx / 2, half_width=nx / 4, width=2.0)
            b.init(k, *fields)
            mass0.append(b.diagnostics(k)["mass"])
        b.step(steps)
        w = nx // 16
        for k in range(len(temps)):
            rho = b.moments(k)[0].mean(axis=0)
            rho_l = float(rho[nx // 2 - w: nx // 2 + w].mean())
            rho_v = float(np.concatenate([rho[:w], rho[nx - w:]]).mean())
            drift = (b.diagnostics(k)["mass"] - mass0[k]) / mass0[k]
            out.append((rho_l, rho_v, drift, surface_tension(rho, kw["dx"], kw["K"])))
    return out


def droplet_runs(radii, precision, n=128, T=0.9, steps=10000, params=None):
    """Static droplets of radius R (cells) centred in an n x n box at temperature T.
    Returns per radius (P_in - P_out, max |u|, mass drift, equimolar radius in cells); P_in and
    rho_in at the centre node, P_out and rho_out averaged over the four corner nodes."""
    p = default_params(precision=precision, **(params or PHASE))
    rl, rv = maxwell(T)
    out = []
    with Batch([(n, n)] * len(radii), p) as b:
        mass0 = []
        for k, R in enumerate(radii):
            b.init(k, *synthetic.droplet(n, n, R, rl, rv, T, width=2.0))
            mass0.append(b.diagnostics(k)["mass"])
        b.step(steps)
        for k in range(len(radii)):
            rho, ux, uy, Tf = b.moments(k)
            P = vdw_pressure(rho, Tf)
            corners = ((0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1))
            p_in = float(P[n // 2, n // 2])
            p_out = float(np.mean([P[c] for c in corners]))
            r_eq = equimolar_radius(rho, float(rho[n // 2, n // 2]), float(np.mean([rho[c] for c in corners])))
            umax = float(np.sqrt(ux * ux + uy * uy).max())
            drift = (b.diagnostics(k)["mass"] - mass0[k]) / mass0[k]
            out.append((p_in - p_out, umax, drift, r_eq))
    return out


def error_table(temps=(0.85, 0.9, 0.95), radii=(8, 12, 16, 24, 32), slab_steps=20000, drop_steps=10000,
                rho64=False):
    """Runs both precisions and returns the per-result comparison (plain dicts, JSON-ready).
    rho64: also LBM_MIXED_RHO64 (the density chain in float64), its errors against float64 in
    the same rows under the suffix _rho64."""
    s64 = slab_runs(temps, LBM_FP64, steps=slab_steps)
    s32 = slab_runs(temps, LBM_MIXED, steps=slab_steps)
    d64 = droplet_runs(radii, LBM_FP64, steps=drop_steps)
    d32 = droplet_runs(radii, LBM_MIXED, steps=drop_steps)
    sr = slab_runs(temps, LBM_MIXED_RHO64, steps=slab_steps) if rho64 else [None] * len(temps)
    dr = droplet_runs(radii, LBM_MIXED_RHO64, steps=drop_steps) if rho64 else [None] * len(radii)
    coex = []
    for T, a, m, r in zip(temps, s64, s32, sr):
        rl, rv = maxwell(T)
        row = {"T": T, "rho_l_fp64": a[0], "rho_l_mixed": m[0], "rho_v_fp64": a[1], "rho_v_mixed": m[1],
               "rel_err_rho_l": abs(m[0] - a[0]) / abs(a[0]), "rel_err_rho_v": abs(m[1] - a[1]) / abs(a[1]),
               "maxwell_rho_l": rl, "maxwell_rho_v": rv,
               "mass_drift_fp64": a[2], "mass_drift_mixed": m[2]}
        if r is not None:
            row.update({"rel_err_rho_l_rho64": abs(r[0] - a[0]) / abs(a[0]),
                        "rel_err_rho_v_rho64": abs(r[1] - a[1]) / abs(a[1]), "mass_drift_rho64": r[2]})
        coex.append(row)
    drops = []
    for R, a, m, r in zip(radii, d64, d32, dr):
        row = {"R": R, "dp_fp64": a[0], "dp_mixed": m[0], "rel_err_dp": abs(m[0] - a[0]) / abs(a[0]),
               "umax_fp64": a[1], "umax_mixed": m[1], "rel_err_umax": abs(m[1] - a[1]) / abs(a[1]),
               "mass_drift_fp64": a[2], "mass_drift_mixed": m[2], "R_eq_fp64": a[3], "R_eq_mixed": m[3],
               "surface_tension_fp64": s64[list(temps).index(0.9)][3] if 0.9 in temps else None}
        if r is not None:
            row.update({"rel_err_dp_rho64": abs(r[0] - a[0]) / abs(a[0]),
                        "rel_err_umax_rho64": abs(r[1] - a[1]) / abs(a[1]), "mass_drift_rho64": r[2]})
        drops.append(row)
    return {"slab": {"nx": 256, "ny": 2, "steps": slab_steps, "rows": coex},
            "droplet": {"n": 128, "T": 0.9, "steps": drop_steps, "rows": drops}}


def laplace_check(radii=(12, 16, 24, 32), n=128, T=0.9, steps=100000, slab_steps=20000, precision=LBM_MIXED,
                  params=None):
    """Laplace law of static droplets against the flat-interface surface tension.

    sigma from a flat slab at the same temperature and parameters (`surface_tension` of its
    final profile); droplets of radius R (cells) relaxed for `steps` steps (the thermal and
    acoustic transients of the start decay slowly at tau = 1e-4); pressures as bulk means of the
    van der Waals pressure, inside over r < R/3 and outside over r > R + 16 cells; R the
    equimolar radius. Returns sigma and per radius (R_eq, P_in - P_out, (P_in - P_out) R / sigma)."""
    kw = dict(params or PHASE)
    sigma = slab_runs([T], precision, steps=slab_steps, params=kw)[0][3]
    p = default_params(precision=precision, **kw)
    rl, rv = maxwell(T)
    Y, X = np.mgrid[0:n, 0:n]
    r = np.hypot(X - n / 2 + 0.5, Y - n / 2 + 0.5)
    rows = []
    with Batch([(n, n)] * len(radii), p) as b:
        for k, R in enumerate(radii):
            b.init(k, *synthetic.droplet(n, n, R, rl, rv, T, width=2.0))
        b.step(steps)
        for k, R in enumerate(radii):
            rho, _, _, Tf = b.moments(k)
            P = vdw_pressure(rho, Tf)
            inner, outer = r < R / 3.0, r > R + 16.0
            dp = float(P[inner].mean() - P[outer].mean())
            r_eq = equimolar_radius(rho, float(rho[inner].mean()), float(rho[outer].mean()))
            rows.append({"R": R, "R_eq": r_eq, "dp": dp, "dp_R_over_sigma": dp * r_eq * kw["dx"] / sigma})
    return {"sigma": sigma, "T": T, "steps": steps, "rows": rows}


def structure_factor_growth(n=4096, checkpoints=(500, 1000, 2000), nbins=None, seed=5, T=0.9):
    """Growth of the structure factor S(k) of the density after a quench (Sec. 3.2's measure of
    domain growth), LBM_MIXED against LBM_FP64 on the same seeded n x n spinodal field
    (rho = 1 +/- 1%, u = 0, T), phase-separation set. Returns per checkpoint the FP64 peak
    shell and height, the mixed peak height, and the relative L2 difference of the two S(k).
    nbins: shells of |q| (default: every shell of the box, up to the corner of the spectrum)."""
    nbins = nbins or int(np.ceil(np.sqrt(2) * n / 2)) + 2
    fields = synthetic.spinodal(n, n, 1.0, 0.01, T, seed=seed)
    S = {}
    for prec in (LBM_FP64, LBM_MIXED):
        with Simulation(n, n, default_params(precision=prec, **PHASE)) as s:
            s.init(*fields)
            done = 0
            for c in checkpoints:
                s.step(c - done)
                done = c
                S[(prec, c)] = s.structure_factor(nbins)[0]
    rows = []
    for c in checkpoints:
        a, m = S[(LBM_FP64, c)], S[(LBM_MIXED, c)]
        k = int(np.argmax(a[1:])) + 1
        rows.append({"steps": c, "peak_shell": k, "peak_fp64": float(a[k]), "peak_mixed": float(m[k]),
                     "rel_l2": float(np.linalg.norm(m - a) / np.linalg.norm(a))})
    return {"n": n, "T": T, "seed": seed, "nbins": nbins, "rows": rows}
