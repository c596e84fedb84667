"""GPU parity of the numerical variants and the isothermal mode against the FP64 oracle:
forward Euler (LBM_FLAG_EULER), the 8th-order modified wavenumber (keff_terms = 4) - the
numerics of the D2V33 runs of Sec. 3.2 - and the thermostat T = T_iso (LBM_FLAG_ISOTHERMAL).
Same per-field metric and 1e-10 bound as tests/test_gpu_parity.py."""
import numpy as np
import pytest

import oracle
import synthetic
from oracle.dvm import D2V16
from oracle.model import init_feq, rk2_step

import paper_1403_3746_gb300 as lbm
from paper_1403_3746_gb300 import build as lbm_build

pytestmark = pytest.mark.gpu
TOL64 = 1e-10
PHASE = dict(tau=1e-4, dt=1e-4, dx=1 / 256, dy=1 / 256, K=5e-6, q=-0.004, b=2.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    lbm_build.build()


def oracle_params(flags=0, T_iso=0.0, keff_terms=8, **kw):
    return oracle.Params(scheme="euler" if flags & lbm.LBM_FLAG_EULER else "rk2",
                         T_iso=T_iso if flags & lbm.LBM_FLAG_ISOTHERMAL else 0.0,
                         keff_terms=keff_terms, **kw)


def run_both(fields, steps, precision=lbm.LBM_FP64, **kw):
    p = oracle_params(**kw)
    d = D2V16(p.eta0)
    f = init_feq(d, *fields, p)
    for _ in range(steps):
        f = rk2_step(d, f, p)
    ny, nx = fields[0].shape
    with lbm.Simulation(nx, ny, lbm.default_params(precision=precision, **kw)) as s:
        s.init(*fields)
        s.step(steps)
        fg, mg = s.get_f(), s.moments()
    return fg, mg, f, oracle.moments(d, f, p.b)


def errors(fg, mg, fo, mo):
    floor = 1e-2 * np.max(np.abs(fo))
    ef = max(float(np.max(np.abs(fg[i] - fo[i])) / max(np.max(np.abs(fo[i])), floor)) for i in range(16))
    em = [float(np.max(np.abs(mg[k] - mo[k])) / max(np.max(np.abs(mo[k])), 1e-3 if k in (1, 2) else 0.0))
          for k in range(4)]
    return ef, em


def slab(nx=64, ny=64, T=0.9, seed=1):
    rl, rv = oracle.coexistence(T)
    return synthetic.slab(nx, ny, rl, rv, T, center=nx / 2, half_width=nx / 4, width=2.0, noise=1e-4, seed=seed)


@pytest.mark.parametrize("flags,terms,steps", [(lbm.LBM_FLAG_EULER, 8, 40), (0, 4, 40),
                                               (lbm.LBM_FLAG_EULER, 4, 40)])
def test_numerical_variants_fp64(flags, terms, steps):
    kw = dict(PHASE, flags=flags, keff_terms=terms)
    if flags & lbm.LBM_FLAG_EULER:
        kw["dt"] = 1e-5  # the Euler runs of Sec. 3.2 take dt = 1e-5
    fg, mg, fo, mo = run_both(slab(), steps, **kw)
    ef, em = errors(fg, mg, fo, mo)
    print(f"flags={flags} terms={terms}: f {ef:.2e}, moments {em}")
    assert ef <= TOL64 and max(em) <= TOL64


def test_isothermal_fp64_slab_and_relaxation():
    # a slab at T = 0.9 held by the thermostat, and a spinodal state at T = 0.95 relaxing to 0.9
    for fields in (slab(), synthetic.spinodal(64, 32, 1.0, 0.02, 0.95, seed=11)):
        fg, mg, fo, mo = run_both(fields, 30, flags=lbm.LBM_FLAG_ISOTHERMAL, T_iso=0.9, **PHASE)
        ef, em = errors(fg, mg, fo, mo)
        print(f"isothermal: f {ef:.2e}, moments {em}")
        assert ef <= TOL64 and max(em[:3]) <= TOL64
        assert np.all(mg[3] == 0.9)  # the stored temperature field is the thermostat's


def test_isothermal_mixed_tracks_fp64():
    fields = synthetic.spinodal(128, 64, 1.0, 0.02, 0.95, seed=12)
    out = {}
    for prec in (lbm.LBM_FP64, lbm.LBM_MIXED):
        with lbm.Simulation(128, 64, lbm.default_params(precision=prec, flags=lbm.LBM_FLAG_ISOTHERMAL,
                                                        T_iso=0.9, **PHASE)) as s:
            s.init(*fields)
            d0 = s.diagnostics()
            s.step(200)
            out[prec] = (s.get_f(), s.moments(), d0, s.diagnostics())
    f64, m64, _, _ = out[lbm.LBM_FP64]
    f32, m32, d0, d1 = out[lbm.LBM_MIXED]
    rel = float(np.linalg.norm(f32 - f64) / np.linalg.norm(f64))
    drho = float(np.max(np.abs(m32[0] - m64[0])) / np.max(np.abs(m64[0])))
    print(f"isothermal mixed vs FP64: f {rel:.2e}, rho {drho:.2e}, mass drift {(d1['mass'] - d0['mass']) / d0['mass']:.2e}")
    assert rel <= 2e-6 and drho <= 2e-6
    assert abs(d1["mass"] - d0["mass"]) <= 1e-6 * d0["mass"]


def test_rectangular_droplet_protocol_against_oracle():
    # Sec. 3.3's protocol scaled to a 64 x 64 box: a 30 x 6 rectangle, liquid 1.462 inside,
    # vapour 0.579 outside, T held at 0.95 (isothermal), dx = dy = 0.01, tau = 5 dt = 5e-4,
    # K = 1e-5, q = -0.05. FP64 against the oracle at the 1e-10 bound. The mixed path's bound is
    # wider than the 2e-6 of the smooth phase-separation cases: the rectangle's edges are one
    # cell wide and its corners sharp, so the float32 rounding of f (6e-8) is amplified by the
    # spectral derivatives' gain at the highest wavenumbers and, with tau = 5 dt, is damped
    # five times more slowly by the collision; measured f 1.7e-5, u 5e-5 after 40 steps.
    from paper_1403_3746_gb300 import droplet as dr
    fields = dr.rectangle(64, length=30, height=6)
    kw = dict(dr.SEC33, flags=lbm.LBM_FLAG_ISOTHERMAL, T_iso=dr.T_FIXED)
    fg, mg, fo, mo = run_both(fields, 40, **kw)
    ef, em = errors(fg, mg, fo, mo)
    print(f"droplet protocol FP64: f {ef:.2e}, moments {em}")
    assert ef <= TOL64 and max(em[:3]) <= TOL64
    fg, mg, fo, mo = run_both(fields, 40, precision=lbm.LBM_MIXED, **kw)
    ef, em = errors(fg, mg, fo, mo)
    print(f"droplet protocol mixed: f {ef:.2e}, moments {em}")
    assert ef <= 1e-4 and max(em[:3]) <= 1e-4


@pytest.mark.parametrize("precision", [lbm.LBM_FP64, lbm.LBM_MIXED])
def test_solution_filter_against_oracle(precision):
    # the window applied to the solution after every step (filter_alpha = 36, filter_p = 36),
    # on a slab (phase-separation set) and a droplet (droplet set of Sec. 3.3, T = 0.9).
    # FP64: the 1e-10 bound. Mixed: in this per-field max metric the float32 path's own error
    # (the same run without the filter) is already ~2.5e-5 on the four eta-carrying fields
    # (f ~ f^eq through the float32 moment-space collision, cond(M) ~ 2e3 times 2^-24 per step
    # at tau = dt), so the filter is held to adding at most half of that again, within the
    # 1e-4 bound of the mixed droplet-protocol test; rho and T to 2e-6, u to 1e-3 of its floor.
    rl, rv = oracle.coexistence(0.9)
    cases = [(slab(), dict(PHASE)),
             (synthetic.droplet(64, 64, 16, rl, rv, 0.9, width=2.0),
              dict(tau=5e-4, dt=1e-4, dx=0.01, dy=0.01, K=1e-5, q=-0.05, b=2.0))]
    for fields, kw in cases:
        fg, mg, fo, mo = run_both(fields, 30, precision=precision, filter_alpha=36.0, filter_p=36.0, **kw)
        ef, em = errors(fg, mg, fo, mo)
        print(f"filter precision={precision}: f {ef:.2e}, moments {em}")
        if precision == lbm.LBM_FP64:
            assert ef <= TOL64 and max(em) <= TOL64
            continue
        ef0, _ = errors(*run_both(fields, 30, precision=precision, **kw))
        print(f"  without the filter: f {ef0:.2e}")
        assert ef <= min(1.5 * ef0 + 2e-6, 1e-4)
        assert max(em[0], em[3]) <= 2e-6 and max(em[1], em[2]) <= 1e-3


def test_solution_filter_keeps_the_droplet_set_bounded():
    # the droplet parameter set of Sec. 3.3 in the thermal mode (T = 0.9, R = 32 on 128^2)
    # with the solution filter: bounded and mass-conserving through 3000 steps in both paths
    rl, rv = oracle.coexistence(0.9)
    fields = synthetic.droplet(128, 128, 32, rl, rv, 0.9, width=2.0)
    kw = dict(tau=5e-4, dt=1e-4, dx=0.01, dy=0.01, K=1e-5, q=-0.05, b=2.0, filter_alpha=36.0, filter_p=36.0)
    for precision in (lbm.LBM_FP64, lbm.LBM_MIXED):
        with lbm.Simulation(128, 128, lbm.default_params(precision=precision, **kw)) as s:
            s.init(*fields)
            d0 = s.diagnostics()
            s.step(3000)
            d1 = s.diagnostics()
            rho = s.moments()[0]
        print(f"precision {precision}: umax {d1['umax']:.3e}, rho {rho.min():.4f}..{rho.max():.4f}")
        assert d1["umax"] < 0.1 and abs(d1["mass"] / d0["mass"] - 1) < 1e-6
        assert rv * 0.9 < rho.min() and rho.max() < rl * 1.1
