"""The structure-factor diagnostic (lbm_structure_factor) against the oracle's definition on
the same density field, a single-mode closed form, and the growth of S(k) after a quench
(mixed path against the FP64 path on the same seed)."""
import numpy as np
import pytest

import oracle
import synthetic
from oracle.diag import structure_factor

import paper_1403_3746_gb300 as lbm
from paper_1403_3746_gb300 import build as lbm_build

pytestmark = pytest.mark.gpu
PHASE = dict(tau=1e-4, dt=1e-4, dx=1 / 256, dy=1 / 256, K=5e-6, q=-0.004, b=2.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    lbm_build.build()


@pytest.mark.parametrize("precision,nx,ny,steps", [(lbm.LBM_FP64, 64, 32, 20), (lbm.LBM_MIXED, 128, 128, 20),
                                                   (lbm.LBM_MIXED, 1024, 1024, 2), (lbm.LBM_FP64, 2, 4, 0),
                                                   (lbm.LBM_MIXED, 8, 256, 3)])
def test_matches_oracle_on_the_same_density(precision, nx, ny, steps):
    nbins = int(np.ceil(np.sqrt(2) * max(nx, ny) / 2)) + 2
    with lbm.Simulation(nx, ny, lbm.default_params(precision=precision, **PHASE)) as s:
        s.init(*synthetic.spinodal(nx, ny, 1.0, 0.01, 0.9, seed=21))
        s.step(steps)
        S, cnt = s.structure_factor(nbins)
        rho = s.moments()[0]
    So, co = structure_factor(rho, nbins)
    So[0] = 0.0
    assert np.array_equal(cnt, co)
    err = float(np.max(np.abs(S - So)) / max(np.max(So), 1e-300))
    print(f"{nx}x{ny}: max rel err {err:.2e}")
    assert err <= 1e-10


def test_single_mode_closed_form():
    N, a = 64, 0.02
    x = np.arange(N)[None, :]
    y = np.arange(N)[:, None]
    rho = 1.0 + a * np.cos(2 * np.pi * (3 * x + 4 * y) / N)
    z = np.zeros((N, N))
    with lbm.Simulation(N, N, lbm.default_params(**PHASE)) as s:
        s.init(rho, z, z.copy(), np.full((N, N), 0.95))
        S, cnt = s.structure_factor(50)
    ref = 2 * (a * N * N / 2) ** 2 / (N * N) / cnt[5]
    assert S[5] == pytest.approx(ref, rel=1e-12)
    assert np.max(np.abs(np.delete(S, 5))) < 1e-20 * ref + 1e-24


def test_batch_instance_and_growth_mixed_vs_fp64():
    # quench: S(k) grows at the unstable wavenumbers; the mixed path follows the FP64 path
    n, steps, nbins = 256, 1000, 182
    fields = synthetic.spinodal(n, n, 1.0, 0.01, 0.9, seed=5)
    curves = {}
    for prec in (lbm.LBM_FP64, lbm.LBM_MIXED):
        with lbm.Batch([(n, n), (64, 64)], lbm.default_params(precision=prec, **PHASE)) as b:
            b.init(0, *fields)
            b.init(1, *synthetic.spinodal(64, 64, 1.0, 0.01, 0.9, seed=6))
            S0, _ = b.structure_factor(0, nbins)
            b.step(steps)
            S1, _ = b.structure_factor(0, nbins)
            Sb, _ = b.structure_factor(1, 48)
            rho_b = b.moments(1)[0]
        So, _ = structure_factor(rho_b, 48)
        So[0] = 0
        assert np.max(np.abs(Sb - So)) <= 1e-10 * np.max(So)
        curves[prec] = (S0, S1)
    S0, S1 = curves[lbm.LBM_FP64]
    kmax = int(np.argmax(S1[1:])) + 1
    print(f"peak shell {kmax}: growth {S1[kmax] / S0[kmax]:.3g}")
    assert S1[kmax] > 2 * S0[kmax]  # spinodal growth
    rel = float(np.linalg.norm(curves[lbm.LBM_MIXED][1] - S1) / np.linalg.norm(S1))
    print(f"S(k) mixed vs FP64 after {steps} steps: {rel:.2e}")
    assert rel <= 1e-4
