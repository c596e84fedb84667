"""Pins of the oracle's forcing term (Eq. (2)), kinetic equation (Eq. (1)) and Runge-Kutta
step (Sec. 2.3) against closed forms derived by hand from the paper's definitions, exact
invariants, and exact decay/propagation rates."""
import numpy as np
import pytest

import oracle
from oracle.dvm import D2V16, feq, moments, moment_matrix
from oracle.model import Params, forcing_terms, rk2_step, init_feq, pressure_vdw
from oracle.diag import diagnostics


def _fields_1d(nx, ny, dx, build):
    x = np.arange(nx)[None, :] * dx * np.ones((ny, 1))
    L = nx * dx
    k = 2 * np.pi / L
    return build(x, k)


def _forcing(dvm, rho, ux, uy, T, p):
    fe = feq(dvm, rho, ux, uy, T, p.b)
    return forcing_terms(dvm, rho, ux, uy, T, fe, p), fe


def test_korteweg_form_of_B_in_1d(dvm):
    # rho = r0 + e cos(kx), u = 0, T uniform. By hand from the definitions after Eq. (2):
    # C = C_q = A = 0 and rho T B_x = (dP^w/drho - T) rho_x - M rho rho_xxx (Korteweg form),
    # with dP^w/drho = 9T/(3 - rho)^2 - 9 rho / 4 and M = K + H T.
    p = Params(K=5e-6, H=2e-6)
    nx, ny, T0, r0, e = 64, 4, 0.9, 1.1, 1e-3
    x = np.arange(nx)[None, :] * p.dx * np.ones((ny, 1))
    k = 2 * np.pi / (nx * p.dx)
    rho = r0 + e * np.cos(k * x)
    rx, rxxx = -e * k * np.sin(k * x), e * k ** 3 * np.sin(k * x)
    T = np.full_like(rho, T0)
    z = np.zeros_like(rho)
    (I, ex), fe = _forcing(dvm, rho, z, z, T, p)
    M = p.K + p.H * T0
    Bx = ((9 * T0 / (3 - rho) ** 2 - 9 * rho / 4 - T0) * rx - M * rho * rxxx) / (rho * T0)
    assert np.max(np.abs(ex["Bx"] - Bx)) < 1e-9 * np.max(np.abs(Bx))
    assert np.max(np.abs(ex["By"])) < 1e-12 * np.max(np.abs(Bx))
    for key in ("A", "C", "Cq"):
        assert np.max(np.abs(ex[key])) < 1e-10 * np.max(np.abs(Bx))
    Iref = -Bx[None] * dvm.vx[:, None, None] * fe
    assert np.max(np.abs(I - Iref)) < 1e-9 * np.max(np.abs(Iref))


@pytest.mark.parametrize("zeta", [0.0, 3e-3])
def test_compression_terms_of_C_in_1d(dvm, zeta):
    # rho, T uniform, u_x = U sin(kx): grad rho = 0 so Lambda = 0, and by hand
    # C = [rho^2 T u'/(3 - rho) - zeta u'^2] / (2 rho T^2), B_x = -zeta u''/(rho T), A = -2 C T.
    p = Params(zeta=zeta)
    nx, ny, T0, r0, U = 32, 2, 0.87, 0.8, 0.05
    x = np.arange(nx)[None, :] * p.dx * np.ones((ny, 1))
    k = 2 * np.pi / (nx * p.dx)
    ux = U * np.sin(k * x)
    u1, u2 = U * k * np.cos(k * x), -U * k * k * np.sin(k * x)
    rho, T, z = np.full_like(ux, r0), np.full_like(ux, T0), np.zeros_like(ux)
    (I, ex), fe = _forcing(dvm, rho, ux, z, T, p)
    C = (r0 * r0 * T0 * u1 / (3 - r0) - zeta * u1 * u1) / (2 * r0 * T0 * T0)
    scale = np.max(np.abs(C))
    assert np.max(np.abs(ex["C"] - C)) < 1e-10 * scale
    assert np.max(np.abs(ex["A"] + 2 * C * T0)) < 1e-10 * scale
    assert np.max(np.abs(ex["Bx"] + zeta * u2 / (r0 * T0))) < 1e-10 * max(scale, 1.0)
    assert np.max(np.abs(ex["Cq"])) < 1e-12 * scale


def test_heat_flux_term_Cq_in_1d(dvm):
    # rho uniform, u = 0, T = T0 + e cos(kx): C = 0, C_q = q (T_x^2 + T T_xx) / T^2 and
    # B_x = rho T_x / ((3 - rho) T), all by hand.
    p = Params(q=-0.05)
    nx, ny, T0, r0, e = 32, 2, 0.9, 1.2, 0.01
    x = np.arange(nx)[None, :] * p.dx * np.ones((ny, 1))
    k = 2 * np.pi / (nx * p.dx)
    T = T0 + e * np.cos(k * x)
    Tx, Txx = -e * k * np.sin(k * x), -e * k * k * np.cos(k * x)
    rho, z = np.full_like(T, r0), np.zeros_like(T)
    (I, ex), fe = _forcing(dvm, rho, z, z, T, p)
    Cq = p.q * (Tx * Tx + T * Txx) / (T * T)
    Bx = r0 * Tx / ((3 - r0) * T)
    assert np.max(np.abs(ex["Cq"] - Cq)) < 1e-9 * np.max(np.abs(Cq))
    assert np.max(np.abs(ex["Bx"] - Bx)) < 1e-9 * np.max(np.abs(Bx))
    assert np.max(np.abs(ex["C"])) < 1e-12 * np.max(np.abs(Cq))


@pytest.mark.parametrize("direction", [(1, 0), (1, 1), (2, 1)])
def test_interfacial_terms_of_C_along_a_direction(dvm, direction):
    # rho = r0 + e cos(xi), u = U sin(xi) n, T uniform, H = 0, with xi = k.r along a lattice
    # direction n. By hand (1D along n, primes = d/ds): rho T B = (dP^w/drho - T) rho' - K rho rho''',
    # 2 rho T^2 C = rho^2 T u'/(3 - rho) - K (rho rho' u')'.
    p = Params(K=5e-6)
    N, T0, r0, e, U = 32, 0.9, 1.0, 2e-3, 0.02
    mx, my = direction
    L = N * p.dx
    kv = 2 * np.pi / L * np.array([mx, my], dtype=float)
    k = np.hypot(*kv)
    n = kv / k
    X, Y = np.meshgrid(np.arange(N) * p.dx, np.arange(N) * p.dy)
    xi = kv[0] * X + kv[1] * Y
    rho = r0 + e * np.cos(xi)
    r1, r2, r3 = -e * k * np.sin(xi), -e * k * k * np.cos(xi), e * k ** 3 * np.sin(xi)
    u = U * np.sin(xi)
    u1, u2 = U * k * np.cos(xi), -U * k * k * np.sin(xi)
    T = np.full_like(rho, T0)
    (I, ex), fe = _forcing(dvm, rho, u * n[0], u * n[1], T, p)
    B = ((9 * T0 / (3 - rho) ** 2 - 9 * rho / 4 - T0) * r1 - p.K * rho * r3) / (rho * T0)
    d_rr1u1 = r1 * r1 * u1 + rho * r2 * u1 + rho * r1 * u2
    C = (rho * rho * T0 * u1 / (3 - rho) - p.K * d_rr1u1) / (2 * rho * T0 * T0)
    assert np.max(np.abs(ex["Bx"] - B * n[0])) < 1e-9 * np.max(np.abs(B))
    assert np.max(np.abs(ex["By"] - B * n[1])) < 1e-9 * np.max(np.abs(B))
    assert np.max(np.abs(ex["C"] - C)) < 1e-9 * np.max(np.abs(C))


def test_forcing_moment_identities(dvm):
    # sum_i I_i = 0 (mass) and sum_i (v_i - u) I_i = -rho T B (momentum) at every node,
    # from the equilibrium moments; random band-limited fields.
    p = Params(q=-0.01, zeta=1e-3, H=1e-6)
    rng = np.random.default_rng(11)
    N = 16

    def smooth(mean, amp):
        h = np.zeros((N, N), complex)
        h[:3, :3] = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        return mean + amp * np.fft.ifft2(h).real * N

    rho, ux, uy, T = smooth(1.0, 0.05), smooth(0.0, 0.02), smooth(0.0, 0.02), smooth(0.9, 0.01)
    (I, ex), fe = _forcing(dvm, rho, ux, uy, T, p)
    scale = np.max(np.abs(I))
    assert np.max(np.abs(I.sum(axis=0))) < 1e-12 * scale
    cx = dvm.vx[:, None, None] - ux
    cy = dvm.vy[:, None, None] - uy
    assert np.max(np.abs((cx * I).sum(0) + rho * T * ex["Bx"])) < 1e-11 * scale
    assert np.max(np.abs((cy * I).sum(0) + rho * T * ex["By"])) < 1e-11 * scale


def test_uniform_equilibrium_is_a_fixed_point(dvm):
    p = Params()
    shape = (8, 16)
    f = init_feq(dvm, np.full(shape, 1.3), np.full(shape, 0.07), np.full(shape, -0.02),
                 np.full(shape, 0.9), p)
    g = f
    for _ in range(3):
        g = rk2_step(dvm, g, p)
    assert np.max(np.abs(g - f)) < 1e-14 * np.max(np.abs(f))


def test_bgk_rk2_decay_rate(dvm):
    # uniform rho, u, T and f = f^eq + delta with delta carrying no mass, momentum or energy:
    # gradients vanish so I = 0 and advection is 0; Eq. (1) reduces to d delta/dt = -delta/tau,
    # and the two-stage step multiplies delta by 1 - z + z^2/2, z = dt/tau.
    p = Params(tau=2e-4, dt=1e-4)
    shape = (4, 8)
    rho, ux, uy, T = (np.full(shape, v) for v in (1.1, 0.05, -0.03, 0.92))
    fe = init_feq(dvm, rho, ux, uy, T, p)
    Cns = np.array([np.ones(16), dvm.vx, dvm.vy, dvm.psi])
    rng = np.random.default_rng(5)
    d = rng.standard_normal(16)
    d -= Cns.T @ np.linalg.solve(Cns @ Cns.T, Cns @ d)
    d *= 1e-3
    f = fe + d[:, None, None]
    g = rk2_step(dvm, f, p)
    z = p.dt / p.tau
    assert np.max(np.abs((g - fe) - (1 - z + z * z / 2) * d[:, None, None])) < 1e-13


def test_advection_only_propagation_rate(dvm):
    # collision and forcing off: each Fourier mode of f_i is multiplied per step by
    # R(-i dt k . v_i), R(z) = 1 + z + z^2/2 (two-stage Runge-Kutta), with k exact for a low mode.
    p = Params(collide=False, force=False, dt=2e-4)
    N = 32
    X, Y = np.meshgrid(np.arange(N) * p.dx, np.arange(N) * p.dy)
    kv = 2 * np.pi / (N * p.dx) * np.array([1.0, 2.0])
    xi = kv[0] * X + kv[1] * Y
    a = np.linspace(0.5, 1.0, 16)
    c = np.linspace(0.01, 0.02, 16)
    f = a[:, None, None] + c[:, None, None] * np.cos(xi)[None]
    g = rk2_step(dvm, f, p)
    th = p.dt * (kv[0] * dvm.vx + kv[1] * dvm.vy)
    R = 1 - 1j * th - th * th / 2
    ref = a[:, None, None] + c[:, None, None] * (R[:, None, None] * np.exp(1j * xi)[None]).real
    assert np.max(np.abs(g - ref)) < 1e-13


def test_mass_and_momentum_conservation_slab(dvm):
    import synthetic
    p = Params()
    rl, rv = oracle.coexistence(0.9)
    rho, ux, uy, T = synthetic.slab(32, 16, rl, rv, 0.9, width=2.0, noise=1e-4, seed=1)
    f = init_feq(dvm, rho, ux, uy, T, p)
    d0 = diagnostics(dvm, f, p)
    for _ in range(20):
        f = rk2_step(dvm, f, p)
    d1 = diagnostics(dvm, f, p)
    assert abs(d1["mass"] - d0["mass"]) < 1e-13 * d0["mass"]
    # momentum is conserved to rounding only (the forcing's momentum part is the spectral
    # divergence of S, which sums to zero on the periodic box): 1e-13 of the mass is a
    # rounding-level bound on any platform, far below what a wrong sign or term would give
    assert abs(d1["px"]) < 1e-13 * d0["mass"] and abs(d1["py"]) < 1e-13 * d0["mass"]
    # total energy drifts only slightly (the paper reports |de_T| ~ 1e-9 for this model)
    assert abs(d1["energy"] - d0["energy"]) < 1e-6 * abs(d0["energy"])


def test_vdw_critical_point():
    # Sec. 2.2's EOS has its critical point at rho_c = T_c = 1, P_c = 3/8:
    # dP/drho = d2P/drho2 = 0 there (central differences).
    h = 1e-4
    P = lambda r: pressure_vdw(r, 1.0)
    assert P(1.0) == pytest.approx(3.0 / 8.0, abs=1e-15)
    assert abs((P(1 + h) - P(1 - h)) / (2 * h)) < 1e-7
    assert abs((P(1 + h) - 2 * P(1.0) + P(1 - h)) / h ** 2) < 1e-6


def test_density_and_temperature_gradients_together(dvm):
    # rho = r0 + e cos(kx), T = T0 + eT cos(kx + 0.7), u = 0, H = 0. By hand:
    # Lambda_xx = K (rho_x^2/2 - rho rho_xx) + K rho rho_x T_x / T   (from -rho T rho_x d_x(K/T)),
    # rho T B_x = d_x(P^w - rho T) + d_x Lambda_xx, rho T^2 C_q = q d_x(rho T T_x), C = 0.
    p = Params(K=5e-6, q=-0.02)
    nx, ny, T0, r0, e, eT = 64, 2, 0.9, 1.05, 2e-3, 3e-3
    x = np.arange(nx)[None, :] * p.dx * np.ones((ny, 1))
    k = 2 * np.pi / (nx * p.dx)
    c, s = np.cos(k * x), np.sin(k * x)
    ct, st = np.cos(k * x + 0.7), np.sin(k * x + 0.7)
    rho, r1, r2, r3 = r0 + e * c, -e * k * s, -e * k * k * c, e * k ** 3 * s
    T, T1, T2 = T0 + eT * ct, -eT * k * st, -eT * k * k * ct
    z = np.zeros_like(rho)
    (I, ex), fe = _forcing(dvm, rho, z, z, T, p)
    K = p.K
    dP = 9 * T * r1 / (3 - rho) ** 2 + 3 * rho * T1 / (3 - rho) - 9 / 4 * rho * r1
    drT = r1 * T + rho * T1
    g = rho * r1 * T1 / T
    g1 = (r1 * r1 * T1 + rho * r2 * T1 + rho * r1 * T2) / T - rho * r1 * T1 * T1 / (T * T)
    dL = -K * rho * r3 + K * g1
    Bx = (dP - drT + dL) / (rho * T)
    Cq = p.q * (r1 * T * T1 + rho * T1 * T1 + rho * T * T2) / (rho * T * T)
    assert np.max(np.abs(ex["Bx"] - Bx)) < 1e-8 * np.max(np.abs(Bx))
    assert np.max(np.abs(ex["Cq"] - Cq)) < 1e-8 * np.max(np.abs(Cq))
    assert np.max(np.abs(ex["C"])) < 1e-12 * np.max(np.abs(Cq))
    # the grad(M/T) part alone is >= 100x the tolerance above (dropping or flipping it fails)
    assert np.min(np.abs(K * g1 / (rho * T))[np.abs(g1) > 0.5 * np.abs(g1).max()]) > 100 * 1e-8 * np.max(np.abs(Bx))


def test_euler_bgk_decay_rate(dvm):
    # forward Euler (the D2V33 runs' scheme, Sec. 3.2): the non-equilibrium part of a uniform
    # state is multiplied by 1 - z per step, z = dt/tau.
    p = Params(tau=4e-4, dt=1e-4, scheme="euler")
    shape = (4, 8)
    rho, ux, uy, T = (np.full(shape, v) for v in (0.9, -0.02, 0.04, 0.95))
    fe = init_feq(dvm, rho, ux, uy, T, p)
    Cns = np.array([np.ones(16), dvm.vx, dvm.vy, dvm.psi])
    d = np.random.default_rng(7).standard_normal(16)
    d -= Cns.T @ np.linalg.solve(Cns @ Cns.T, Cns @ d)
    d *= 1e-3
    g = rk2_step(dvm, fe + d[:, None, None], p)
    z = p.dt / p.tau
    assert np.max(np.abs((g - fe) - (1 - z) * d[:, None, None])) < 1e-13


def test_euler_advection_amplification(dvm):
    # collision and forcing off: forward Euler multiplies each Fourier mode of f_i by
    # 1 - i dt k . v_i (|.| > 1: the scheme amplifies pure advection, as expected of Euler).
    p = Params(collide=False, force=False, dt=2e-4, scheme="euler")
    N = 32
    X, Y = np.meshgrid(np.arange(N) * p.dx, np.arange(N) * p.dy)
    kv = 2 * np.pi / (N * p.dx) * np.array([2.0, -1.0])
    xi = kv[0] * X + kv[1] * Y
    a = np.linspace(0.4, 1.1, 16)
    c = np.linspace(0.02, 0.01, 16)
    f = a[:, None, None] + c[:, None, None] * np.sin(xi)[None]
    g = rk2_step(dvm, f, p)
    th = p.dt * (kv[0] * dvm.vx + kv[1] * dvm.vy)
    ref = a[:, None, None] + c[:, None, None] * ((1 - 1j * th)[:, None, None] * (-1j) * np.exp(1j * xi)[None]).real
    assert np.max(np.abs(g - ref)) < 1e-13


def test_isothermal_relaxation_to_the_thermostat(dvm):
    # isothermal mode: uniform state whose temperature moment T0 differs from T_iso. Gradients
    # vanish (I = 0, no advection), mass and momentum are conserved, so the target
    # f^eq(rho, u, T_iso) is fixed and f - f^eq(T_iso) is multiplied by 1 - z + z^2/2 per step.
    p = Params(tau=3e-4, dt=1e-4, T_iso=0.9)
    shape = (4, 4)
    rho, ux, uy = (np.full(shape, v) for v in (1.2, 0.03, 0.01))
    T0 = np.full(shape, 0.97)
    f0 = feq(dvm, rho, ux, uy, T0, p.b)
    target = feq(dvm, rho, ux, uy, np.full(shape, 0.9), p.b)
    f = f0.copy()
    z = p.dt / p.tau
    for n in range(1, 4):
        f = rk2_step(dvm, f, p)
        assert np.max(np.abs((f - target) - (1 - z + z * z / 2) ** n * (f0 - target))) < 1e-13
    r, vx, vy, T = moments(dvm, f, p.b)
    assert np.allclose(r, 1.2, rtol=0, atol=1e-14) and np.allclose(vx, 0.03, rtol=0, atol=1e-14)
    assert np.all(np.abs(T - 0.9) < np.abs(0.97 - 0.9))


def test_structure_factor_of_single_modes_and_parseval():
    # rho = 1 + a cos(2 pi (3 x + 4 y)/N): the DFT of rho - mean has two entries of modulus
    # a N^2 / 2 at (3, 4) and (-3, -4), both on shell 5, so S(5) = 2 (a N^2/2)^2 / N^2 / count(5)
    # and every other shell is 0. Parseval: sum_b S(b) count(b) = sum (rho - mean)^2 (all shells).
    from oracle.diag import structure_factor
    N, a = 32, 0.03
    x = np.arange(N)[None, :]
    y = np.arange(N)[:, None]
    rho = 1.0 + a * np.cos(2 * np.pi * (3 * x + 4 * y) / N)
    S, cnt = structure_factor(rho, 40)
    ref = 2 * (a * N * N / 2) ** 2 / (N * N) / cnt[5]
    assert S[5] == pytest.approx(ref, rel=1e-12)
    assert np.max(np.abs(np.delete(S, 5))) < 1e-20
    rng = np.random.default_rng(3)
    r = 1.0 + 0.01 * rng.standard_normal((16, 32))
    S, cnt = structure_factor(r, 64)
    assert np.sum(S * cnt) == pytest.approx(np.sum((r - r.mean()) ** 2), rel=1e-12)
    assert cnt.sum() == 16 * 32


def test_diagnostics_of_a_single_density_mode(dvm):
    # rho = rho0 + a sin(k x) with uniform u and T: every total is a closed form over the
    # periodic box of area A (sin averages to 0, sin^2 and cos^2 to 1/2; the spectral
    # derivative of a low mode is k cos(k x) to 1e-14 for the 16th-order k_eff):
    # mass = rho0 A, p = rho0 u A, e_T = A [rho0 T - 9/8 (rho0^2 + a^2/2) + K a^2 k^2 / 4
    # + rho0 |u|^2 / 2], max |u| = |u|.
    nx, ny, rho0, a, T, u = 32, 8, 1.1, 0.2, 0.95, (0.03, -0.04)
    p = Params()
    x = np.arange(nx)[None, :] * p.dx * np.ones((ny, 1))
    L = nx * p.dx
    k = 2 * np.pi / L
    rho = rho0 + a * np.sin(k * x)
    f = feq(dvm, rho, np.full_like(rho, u[0]), np.full_like(rho, u[1]), np.full_like(rho, T), p.b)
    d = diagnostics(dvm, f, p)
    A = L * ny * p.dy
    u2 = u[0] ** 2 + u[1] ** 2
    assert d["mass"] == pytest.approx(rho0 * A, rel=1e-13)
    assert d["px"] == pytest.approx(rho0 * u[0] * A, rel=1e-12)
    assert d["py"] == pytest.approx(rho0 * u[1] * A, rel=1e-12)
    eT = A * (rho0 * T - 9 / 8 * (rho0 ** 2 + a * a / 2) + p.K * a * a * k * k / 4 + rho0 * u2 / 2)
    assert d["energy"] == pytest.approx(eT, rel=1e-12)
    assert d["umax"] == pytest.approx(np.sqrt(u2), rel=1e-12)
