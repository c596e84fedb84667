"""Flat-interface coexistence of the oracle's dynamics against the Maxwell construction
(Sec. 3.1, Fig. 1(a): the simulated coexistence curve follows the Maxwell construction of the
van der Waals fluid).

A flat liquid slab between vapour layers, at rest and at uniform temperature, is a steady state
of Eqs. (1)-(2) when the momentum source of the discrete kinetic equation vanishes at every node.
The profile with that property is found here by Newton's method, using the oracle's own
right-hand side R(f) (the function its Runge-Kutta step advances) as a black box: the residual
is the momentum moment sum_i v_ix R_i at f = f^eq(rho, 0, T). Its bulk densities must be the
coexisting pair of the Maxwell construction (oracle.coexistence, pinned separately against the
densities the paper prints at T = 0.95). That holds only if the pressure tensor built from the
EOS and the stress Lambda of Sec. 2.2 is of the Korteweg form that obeys the Gibbs-Duhem
relation, so a wrong sign or factor in Lambda, or an EOS inconsistent with the Maxwell solver,
moves the bulk densities (the planted-mistake test below shows the size of such a shift).

Parameters: Sec. 3.1's set (dx = 0.02, dt = 5e-5, tau = 1e-4, q = -0.004, b = 2) with the
surface-tension coefficient raised from 1e-5 to 4e-4, so that the interface spans about two
cells (at K = 1e-5 it is a third of a cell, which the spectral scheme cannot represent as a
smooth steady profile). The bulk densities of a flat-interface equilibrium do not depend on K
(they follow from the EOS alone), so the comparison with Maxwell is unchanged by it.
"""
import numpy as np
import pytest

import oracle
import synthetic
from oracle.dvm import D2V16, moments
from oracle.model import Params, init_feq, rhs, rk2_step

NX, NY = 128, 2
K_RESOLVED = 4e-4


def _params():
    p = Params.coexistence()
    p.K = K_RESOLVED
    return p


def _fields(rho1d, T0):
    rho = np.broadcast_to(rho1d, (NY, rho1d.size)).copy()
    z = np.zeros_like(rho)
    return rho, z, z.copy(), np.full_like(rho, T0)


def _momentum_source(d, p, rho1d, T0):
    f = init_feq(d, *_fields(rho1d, T0), p)
    R = rhs(d, f, p)
    return np.tensordot(d.vx, R, axes=(0, 0)).mean(axis=0)


def _steady_slab(d, p, T0, rl0, rv0, iters=8):
    """Newton iteration on the even (about x = nx/2) density profile at fixed total mass, with
    the grid-scale alternating mode (invisible to the spectral derivatives, whose Nyquist
    multiplier is zero) kept out of every update. Returns the profile and the last residual."""
    h = NX // 2
    E = np.zeros((NX, h + 1))
    E[np.arange(NX), np.abs(np.arange(NX) - h)] = 1.0
    alt = (-1.0) ** np.arange(NX)
    B = (np.eye(NX) - np.outer(alt, alt) / NX) @ E
    rho = synthetic.slab(NX, 1, rl0, rv0, T0, width=3.0)[0][0]
    mass = rho.sum()
    eps = 1e-7
    for _ in range(iters):
        r = _momentum_source(d, p, rho, T0)
        if np.max(np.abs(r)) < 1e-10:
            break
        J = np.empty((NX, h + 1))
        for j in range(h + 1):
            J[:, j] = (_momentum_source(d, p, rho + eps * B[:, j], T0) - r) / eps
        A = np.vstack([J, B.sum(axis=0)[None]])
        da = np.linalg.lstsq(A, np.concatenate([-r, [mass - rho.sum()]]), rcond=1e-13)[0]
        rho = rho + B @ da
    return rho, np.max(np.abs(_momentum_source(d, p, rho, T0)))


@pytest.mark.slow
@pytest.mark.parametrize("T0", [0.95, 0.9])
def test_steady_flat_interface_has_maxwell_densities(dvm, T0):
    p = _params()
    rl, rv = oracle.coexistence(T0)
    # start 1% / 2% off the coexisting pair; mass fixes how much of each phase there is
    rho, res = _steady_slab(dvm, p, T0, 1.01 * rl, 0.98 * rv)
    assert res < 1e-10, res
    # bulk values: the slab centre (liquid) and the box edge (vapour), 32 cells from the interfaces
    assert rho[NX // 2] / rl - 1 == pytest.approx(0.0, abs=2e-6)
    assert rho[0] / rv - 1 == pytest.approx(0.0, abs=2e-6)
    # and the two phases are flat there
    assert np.ptp(rho[NX // 2 - 4: NX // 2 + 5]) < 1e-5 and np.ptp(rho[:5]) < 1e-5


@pytest.mark.slow
def test_planted_eos_mistake_moves_the_bulk_densities(dvm, monkeypatch):
    # The same solve with the attraction constant of the EOS off by 1% inside the forcing
    # term (a planted mistake; the Maxwell solver keeps the printed EOS). The steady bulk
    # densities then miss the Maxwell pair by far more than the tolerance above.
    import oracle.model as om
    monkeypatch.setattr(om, "pressure_vdw", lambda rho, T: 3.0 * rho * T / (3.0 - rho) - 1.01 * 9.0 / 8.0 * rho ** 2)
    T0 = 0.9
    rl, rv = oracle.coexistence(T0)
    rho, res = _steady_slab(dvm, _params(), T0, 1.01 * rl, 0.98 * rv)
    assert res < 1e-10
    assert abs(rho[NX // 2] / rl - 1) > 1e-3 and abs(rho[0] / rv - 1) > 1e-3


@pytest.mark.slow
def test_runge_kutta_run_keeps_the_coexisting_slab(dvm):
    # 400 Runge-Kutta steps (Sec. 2.3) from the steady profile with f = f^eq: the kinetic
    # scheme itself (not only its momentum source at f = f^eq) keeps the slab at the Maxwell
    # densities, with mass conserved and only small residual currents.
    T0 = 0.9
    p = _params()
    rl, rv = oracle.coexistence(T0)
    rho, _ = _steady_slab(dvm, p, T0, 1.01 * rl, 0.98 * rv)
    f = init_feq(dvm, *_fields(rho, T0), p)
    m0 = f.sum()
    for _ in range(400):
        f = rk2_step(dvm, f, p)
    r, ux, uy, T = moments(dvm, f, p.b)
    assert abs(f.sum() / m0 - 1) < 1e-13
    assert r[0, NX // 2] / rl - 1 == pytest.approx(0.0, abs=1e-5)
    assert r[0, 0] / rv - 1 == pytest.approx(0.0, abs=1e-5)
    assert np.max(np.abs(ux)) < 1e-3 and np.max(np.abs(uy)) < 1e-12
