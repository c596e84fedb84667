"""Pins of the oracle's discrete-velocity model and equilibrium (Sec. 2.1, Sec. 2.2's
Chapman-Enskog remark): the equilibrium moments must be those of a continuous Maxwellian
with b degrees of freedom, computed here by Gauss-Hermite quadrature."""
import itertools

import numpy as np
import pytest

from oracle.dvm import D2V16, moment_matrix, equilibrium_moments, feq, moments


def maxwellian_moments(rho, ux, uy, T, b, order=24):
    """The 16 moment functionals of moment_matrix, integrated against
    rho (2 pi T)^(-b/2) exp(-(|v - u|^2 + |eta|^2) / (2T)) over v in R^2 and eta in R^(b-2)."""
    x, w = np.polynomial.hermite_e.hermegauss(order)   # weight exp(-x^2/2)
    w = w / np.sqrt(2 * np.pi)
    s = np.sqrt(T)
    out = np.zeros(16)
    extra = int(b) - 2
    for idx in itertools.product(range(order), repeat=2 + extra):
        wt = np.prod([w[i] for i in idx])
        vx = ux + s * x[idx[0]]
        vy = uy + s * x[idx[1]]
        eta2 = sum((s * x[i]) ** 2 for i in idx[2:])
        psi = vx * vx + vy * vy + eta2
        row = [1, vx, vy, psi, vx * vx, vx * vy, vy * vy, psi * vx, psi * vy,
               vx ** 3, vx * vx * vy, vx * vy * vy, vy ** 3, psi * vx * vx, psi * vx * vy, psi * vy * vy]
        out += wt * np.array(row)
    return rho * out


@pytest.mark.parametrize("b", [2, 3, 4])
def test_equilibrium_moments_are_maxwellian(b):
    order = 6
    for rho, ux, uy, T in [(1.0, 0.0, 0.0, 0.9), (0.7, 0.13, -0.21, 0.85), (1.6, -0.4, 0.05, 1.1)]:
        ref = maxwellian_moments(rho, ux, uy, T, b, order)
        got = equilibrium_moments(rho, ux, uy, T, float(b))
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_moment_matrix_rows_match_velocity_functionals(dvm):
    # row j of M applied to a single particle at velocity v_i equals the functional at v_i
    M = moment_matrix(dvm)
    assert M.shape == (16, 16)
    assert np.linalg.matrix_rank(M) == 16
    for i in range(16):
        vx, vy, e = dvm.vx[i], dvm.vy[i], dvm.eta[i]
        psi = vx * vx + vy * vy + e * e
        # psi v_x v_y and v_x^2 v_y, independently written
        assert M[14, i] == pytest.approx(psi * vx * vy, abs=1e-12)
        assert M[10, i] == pytest.approx(vx * vx * vy, abs=1e-12)


def test_velocity_set_geometry(dvm):
    # Kataoka-Tsutahara speeds 1, sqrt2, 3/sqrt2, 6: axes for 1 and 6, diagonals for the others
    speeds = np.sort(np.unique(np.round(np.hypot(dvm.vx, dvm.vy), 12)))
    assert np.allclose(speeds, [1.0, np.sqrt(2.0), 3.0 / np.sqrt(2.0), 6.0])
    diag = np.abs(np.abs(dvm.vx) - np.abs(dvm.vy)) < 1e-15
    assert list(diag) == [False] * 8 + [True] * 8
    assert np.allclose(dvm.v.sum(axis=0), 0.0)
    assert np.allclose(dvm.eta, [2.5] * 4 + [0.0] * 12)


@pytest.mark.parametrize("b", [2.0, 3.0])
def test_feq_reproduces_hydrodynamic_moments(dvm, b):
    rng = np.random.default_rng(3)
    rho = 0.5 + rng.random((3, 5))
    ux = 0.3 * rng.standard_normal((3, 5))
    uy = 0.3 * rng.standard_normal((3, 5))
    T = 0.8 + 0.3 * rng.random((3, 5))
    f = feq(dvm, rho, ux, uy, T, b)
    r2, ux2, uy2, T2 = moments(dvm, f, b)
    for a, c in [(rho, r2), (ux, ux2), (uy, uy2), (T, T2)]:
        assert np.allclose(a, c, rtol=1e-12, atol=1e-13)
    # all 16 moments, against quadrature of the Maxwellian at one node
    M = moment_matrix(dvm)
    ref = maxwellian_moments(rho[1, 2], ux[1, 2], uy[1, 2], T[1, 2], int(b), 6)
    assert np.allclose(M @ f[:, 1, 2], ref, rtol=1e-11, atol=1e-11)


def test_feq_is_fourth_degree_polynomial_in_u(dvm):
    # Sec. 2.1: f^eq is a polynomial of u up to fourth order: 5th differences vanish, 4th don't
    t = np.linspace(-0.3, 0.3, 9)
    d = np.array([0.6, -0.8])
    f = np.array([feq(dvm, 1.1, s * d[0], s * d[1], 0.9, 2.0) for s in t])  # (9, 16)
    d5 = np.diff(f, n=5, axis=0)
    d4 = np.diff(f, n=4, axis=0)
    assert np.max(np.abs(d5)) < 1e-11
    assert np.max(np.abs(d4)) > 1e-6


def test_feq_rotation_covariance(dvm):
    # rotating u by +90 degrees maps f_i^eq onto the velocity rotated by +90 degrees
    fu = feq(dvm, 1.2, 0.17, -0.09, 0.93, 2.0)
    fr = feq(dvm, 1.2, 0.09, 0.17, 0.93, 2.0)
    for i in range(16):
        rv = np.array([-dvm.vy[i], dvm.vx[i]])
        j = int(np.argmin(np.hypot(dvm.vx - rv[0], dvm.vy - rv[1])))
        assert fr[j] == pytest.approx(fu[i], abs=1e-12)
