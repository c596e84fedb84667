"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on the same
seeded inputs, element by element.

Error metric (per field, as the distributions f_1..f_4 vanish at rest when b = 2):
    err = max |x_gpu - x_oracle| / max |x_oracle|
Bound for the FP64 path: 1e-10 after the run's steps (spectral derivatives, the moment
inversion and the Runge-Kutta stages are evaluated in a different order than the
oracle's, so results agree to rounding, amplified at most mildly over the steps).
"""
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    lbm_build.build()


def oracle_params(**kw):
    flags = kw.pop("flags", 0)
    kw.pop("precision", None)
    return oracle.Params(advect=not flags & lbm.LBM_FLAG_NO_ADVECTION,
                         collide=not flags & lbm.LBM_FLAG_NO_COLLISION,
                         force=not flags & lbm.LBM_FLAG_NO_FORCE, **kw)


def lib_params(**kw):
    return lbm.default_params(**kw)


def run_oracle(fields, steps, **kw):
    p = oracle_params(**kw)
    d = D2V16(p.eta0)
    f = init_feq(d, *fields, p)
    for _ in range(steps):
        f = rk2_step(d, f, p)
    return f, oracle.moments(d, f, p.b)


def run_gpu(fields, steps, **kw):
    ny, nx = fields[0].shape
    with lbm.Simulation(nx, ny, lib_params(**kw)) as s:
        s.init(*fields)
        s.step(steps)
        return s.get_f(), s.moments()


def field_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def assert_parity(fg, mg, fo, mo, tol, what=""):
    errs = [field_err(fg[i], fo[i]) for i in range(16)]
    merrs = [field_err(mg[k], mo[k]) for k in range(4)]
    assert max(errs) <= tol, f"{what}: f errors {errs}"
    assert max(merrs) <= tol, f"{what}: moment errors {merrs}"


def slab_fields(nx, ny, T=0.9, noise=1e-4, seed=1):
    rl, rv = oracle.coexistence(T)
    return synthetic.slab(nx, ny, rl, rv, T, center=nx / 2, half_width=nx / 4, width=2.0, noise=noise, seed=seed)


def moving_fields(nx, ny, seed=9):
    # non-trivial velocity and temperature fields so every term of I_i is exercised
    rho = synthetic.spinodal(nx, ny, 1.0, 0.02, 0.92, seed=seed)[0]
    x = np.arange(nx)[None, :] / nx
    y = np.arange(ny)[:, None] / ny
    ux = 0.03 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    uy = -0.02 * np.cos(4 * np.pi * x) * np.sin(2 * np.pi * y)
    T = 0.92 + 0.01 * np.cos(2 * np.pi * (x + y))
    return rho, ux, uy, T


def test_init_is_equilibrium_of_the_given_moments():
    fields = moving_fields(32, 16)
    with lbm.Simulation(32, 16, lib_params()) as s:
        s.init(*fields)
        f = s.get_f()
        m = s.moments()
    d = D2V16(2.5)
    fo = init_feq(d, *fields, oracle.Params())
    assert max(field_err(f[i], fo[i]) for i in range(16)) <= 1e-13
    for a, b in zip(m, fields):
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b)) + 1e-15


@pytest.mark.parametrize("flags", [
    lbm.LBM_FLAG_NO_COLLISION | lbm.LBM_FLAG_NO_FORCE,   # advection only
    lbm.LBM_FLAG_NO_ADVECTION | lbm.LBM_FLAG_NO_FORCE,   # BGK only
    lbm.LBM_FLAG_NO_ADVECTION | lbm.LBM_FLAG_NO_COLLISION,  # forcing only
    0,
])
@pytest.mark.parametrize("nx,ny", [(64, 32), (16, 128)])
def test_each_term_of_eq1(flags, nx, ny):
    fields = moving_fields(nx, ny)
    kw = dict(flags=flags, q=-0.02, zeta=1e-3, H=1e-6)
    fo, mo = run_oracle(fields, 3, **kw)
    fg, mg = run_gpu(fields, 3, **kw)
    assert_parity(fg, mg, fo, mo, 1e-11, f"flags={flags} {nx}x{ny}")


def test_slab_64_200_steps():
    # 64 x 64 planar slab at T = 0.9 with seeded noise 1e-4, 200 Runge-Kutta steps
    fields = slab_fields(64, 64)
    fo, mo = run_oracle(fields, 200)
    fg, mg = run_gpu(fields, 200)
    assert_parity(fg, mg, fo, mo, TOL64, "slab 64^2 x 200")


@pytest.mark.parametrize("nx,ny", [(128, 32), (32, 128), (512, 2), (2, 64), (2, 2), (4, 8)])
def test_grid_shapes(nx, ny):
    fields = slab_fields(nx, ny) if nx >= 8 else moving_fields(nx, ny)
    fo, mo = run_oracle(fields, 5)
    fg, mg = run_gpu(fields, 5)
    assert_parity(fg, mg, fo, mo, TOL64, f"{nx}x{ny}")


def test_spinodal_256_20_steps():
    fields = synthetic.spinodal(256, 256, 1.0, 0.01, 0.9, seed=2)
    fo, mo = run_oracle(fields, 20)
    fg, mg = run_gpu(fields, 20)
    assert_parity(fg, mg, fo, mo, TOL64, "spinodal 256^2 x 20")


def test_droplet_1024_one_step():
    # the 1024^2 droplet workload (droplet parameter set, T = 0.85, R = 128), one full step
    T = 0.85
    rl, rv = oracle.coexistence(T)
    fields = synthetic.droplet(1024, 1024, 128, rl, rv, T, width=2.0)
    kw = dict(tau=5e-4, dt=1e-4, dx=0.01, dy=0.01, K=1e-5, q=-0.05)
    fo, mo = run_oracle(fields, 1, **kw)
    fg, mg = run_gpu(fields, 1, **kw)
    assert_parity(fg, mg, fo, mo, TOL64, "droplet 1024^2 x 1")


def test_conservation_and_diagnostics():
    fields = synthetic.spinodal(128, 128, 1.0, 0.01, 0.9, seed=2)
    p = oracle.Params()
    d = D2V16(p.eta0)
    with lbm.Simulation(128, 128, lib_params()) as s:
        s.init(*fields)
        d0 = s.diagnostics()
        o0 = oracle.diagnostics(d, init_feq(d, *fields, p), p)
        for k in ("mass", "px", "py", "energy", "umax"):
            assert d0[k] == pytest.approx(o0[k], rel=1e-12, abs=1e-15)
        s.step(300)
        d1 = s.diagnostics()
    assert d1["steps"] == 300
    assert abs(d1["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert abs(d1["px"]) <= 1e-13 * d0["mass"] and abs(d1["py"]) <= 1e-13 * d0["mass"]


def test_set_get_roundtrip_and_errors():
    fields = slab_fields(32, 32)
    d = D2V16(2.5)
    f = init_feq(d, *fields, oracle.Params()) * (1 + 1e-3 * np.sin(np.arange(16))[:, None, None])
    with lbm.Simulation(32, 32, lib_params()) as s:
        with pytest.raises(lbm.LbmError, match="out of order"):
            s.step(1)
        s.set_f(f)
        assert np.array_equal(s.get_f(), f)
        m = s.moments()
        mo = oracle.moments(d, f, 2.0)
        for a, b in zip(m, mo):
            assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b)) + 1e-16
        bad = f.copy()
        bad[3, 4, 5] = np.nan
        with pytest.raises(lbm.LbmError, match="not finite"):
            s.set_f(bad)


def test_unsupported_row_length_in_fp64():
    with pytest.raises(lbm.LbmError, match="unsupported"):
        lbm.Simulation(4096, 8, lib_params())
