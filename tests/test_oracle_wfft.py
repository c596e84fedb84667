"""Pins of the oracle's spatial-derivative scheme (Sec. 2.3, Eq. (3)) against mathematics
that does not go through the oracle's own formula."""
import numpy as np
import pytest
import sympy

from oracle.wfft import C_KEFF, keff, deriv_multiplier, spectral_deriv, dft_deriv_matrix, dft_indices


def test_keff_coefficients_are_arcsin_series():
    # Eq. (3): the eight printed fractions are the Maclaurin coefficients of arcsin.
    x = sympy.symbols("x")
    ser = sympy.series(sympy.asin(x), x, 0, 17).removeO()
    for n, c in enumerate(C_KEFF):
        exact = ser.coeff(x, 2 * n + 1)
        assert c == pytest.approx(float(exact), rel=0, abs=1e-17)


def test_keff_is_sixteenth_order():
    # k - k_eff ~ c_8 phi^17: the log-log slope of the error between two moderate phi is ~17.
    N, dx = 4096, 1.0
    m = np.array([N * np.arcsin(0.5) / np.pi, N * np.arcsin(0.4) / np.pi])  # phi = 0.5, 0.4
    k = 2.0 * np.pi * m / (N * dx)
    err = k - keff(m, N, dx)
    assert np.all(err > 0)
    slope = np.log(err[0] / err[1]) / np.log(0.5 / 0.4)
    assert 17.0 <= slope <= 18.5
    # at phi = 1 the truncated series sums to 1.37..., i.e. k_eff/k = 0.8724 at Nyquist
    assert keff(N // 2, N, dx) / (np.pi / dx) == pytest.approx(0.8724, abs=5e-5)


@pytest.mark.parametrize("nx,ny", [(64, 64), (64, 32), (32, 128)])
def test_low_mode_derivatives_match_calculus(nx, ny):
    # smooth band-limited field: the spectral derivative equals the analytic one, since
    # k_eff(k) = k to machine precision for modes m <= 2 when N >= 32 (c_8 phi^16 < 1e-15).
    dx, dy = 0.013, 0.021
    x = np.arange(nx)[None, :] * dx
    y = np.arange(ny)[:, None] * dy
    Lx, Ly = nx * dx, ny * dy
    a, b = 2 * np.pi / Lx, 2 * np.pi / Ly
    h = 1.3 + np.sin(a * x) * np.cos(2 * b * y) + 0.4 * np.cos(2 * a * x + 0.3)
    hx = a * np.cos(a * x) * np.cos(2 * b * y) - 0.8 * a * np.sin(2 * a * x + 0.3)
    hy = -2 * b * np.sin(a * x) * np.sin(2 * b * y)
    hxx = -a * a * np.sin(a * x) * np.cos(2 * b * y) - 1.6 * a * a * np.cos(2 * a * x + 0.3)
    hxy = -2 * a * b * np.cos(a * x) * np.sin(2 * b * y)
    hyy = -4 * b * b * np.sin(a * x) * np.cos(2 * b * y)
    for (ox, oy), ref in {(1, 0): hx, (0, 1): hy, (2, 0): hxx, (1, 1): hxy, (0, 2): hyy}.items():
        got = spectral_deriv(h, ox, oy, dx, dy)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_high_mode_eigenvalue_and_nyquist():
    # derivative of a pure mode is k_eff(m) times the quadrature mode; Nyquist mode -> 0
    N, dx = 32, 0.1
    x = np.arange(N)
    for m in (5, 11, 15):
        h = np.sin(2 * np.pi * m * x / N)[None, :].repeat(2, axis=0)
        got = spectral_deriv(h, 1, 0, dx, 1.0)
        phi = np.sin(np.pi * m / N)
        # eigenvalue bracketed by the truncation of the arcsin series (all terms positive)
        ke = got[0] / np.cos(2 * np.pi * m * x / N)
        ke = ke[np.abs(np.cos(2 * np.pi * m * x / N)) > 0.5]
        assert np.ptp(ke) < 1e-10 * abs(ke[0])
        assert (2 / dx) * phi <= ke[0] <= (2 / dx) * np.arcsin(phi)
    nyq = np.cos(np.pi * x)[None, :].repeat(2, axis=0)
    assert np.max(np.abs(spectral_deriv(nyq, 1, 0, dx, 1.0))) < 1e-12
    assert np.max(np.abs(spectral_deriv(np.full((4, N), 3.0), 1, 0, dx, 1.0))) < 1e-12


def test_multiplier_is_odd_and_purely_imaginary():
    for N in (2, 4, 8, 64, 128):
        d = deriv_multiplier(N, 0.5)
        m = dft_indices(N)
        assert np.all(d.real == 0)
        for j in range(N):
            jj = np.where(m == -m[j])[0]
            if len(jj):
                assert abs(d[jj[0]] + d[j]) <= 1e-15 * abs(d[j]) or (m[j] == -N // 2 and d[j] == 0)


def _brute_force_deriv(h, ox, oy, dx, dy, alpha=0.0, p=36.0, terms=8):
    # sum_m d(m)^o exp(2 pi i m (a - b) / N) / N written out per output value, one axis at a
    # time: no FFT and no matrix shared with the oracle
    def axis_op(N, d, order):
        m = np.rint(np.fft.fftfreq(N) * N)
        phi = np.sin(np.pi * m / N)
        ke = (2.0 / d) * sum(c * phi ** (2 * n + 1) for n, c in enumerate(C_KEFF[:terms]))
        w = np.exp(-alpha * (np.abs(m) / (N / 2)) ** p) if alpha else np.ones(N)
        mult = (1j * ke * w) ** order
        mult[m == -N // 2] = 0.0
        a = np.arange(N)
        return np.array([[np.sum(mult * np.exp(2j * np.pi * m * (i - j) / N)).real / N for j in a] for i in a])
    out = h
    if ox:
        out = out @ axis_op(h.shape[1], dx, ox).T
    if oy:
        out = axis_op(h.shape[0], dy, oy) @ out
    return out


@pytest.mark.parametrize("nx,ny", [(8, 8), (16, 4), (4, 32), (2, 8), (128, 2), (64, 64)])
def test_fft_derivative_matches_brute_force_dft(nx, ny):
    # at N = 64 and 128 the operator is checked at the sizes the GPU parity tests run
    rng = np.random.default_rng(7)
    h = rng.standard_normal((ny, nx))
    dx, dy = 0.3, 0.7
    for ox, oy in [(1, 0), (0, 1), (2, 0), (0, 2), (1, 1)]:
        ref = _brute_force_deriv(h, ox, oy, dx, dy)
        got = spectral_deriv(h, ox, oy, dx, dy)
        tol = 1e-11 * max(1.0, np.abs(ref).max())
        assert np.allclose(got, ref, rtol=0, atol=tol)
        # the oracle's explicit-DFT back-end is the same operator
        assert np.allclose(spectral_deriv(h, ox, oy, dx, dy, backend="dft"), ref, rtol=0, atol=tol)
        if nx >= 64:
            assert np.allclose(spectral_deriv(h, ox, oy, dx, dy, 36.0, 36.0, 4, "dft"),
                               _brute_force_deriv(h, ox, oy, dx, dy, 36.0, 36.0, 4), rtol=0, atol=tol)


def test_dft_matrix_is_the_brute_force_sum():
    for N, order in ((16, 1), (32, 2), (128, 1)):
        D = dft_deriv_matrix(N, 0.25, order)
        ref = _brute_force_deriv(np.eye(N), order, 0, 0.25, 1.0)
        assert np.allclose(D.T, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_rk2_step_same_with_both_derivative_back_ends(dvm):
    # one Runge-Kutta step of a 32 x 16 noisy slab: the FFT and the explicit DFT back-ends
    # of Eq. (3) agree to round-off through the whole step (advection and forcing chain)
    import synthetic
    from oracle.model import Params, init_feq, rk2_step
    from oracle.maxwell import coexistence
    rl, rv = coexistence(0.9)
    fields = synthetic.slab(32, 16, rl, rv, 0.9, half_width=8, noise=1e-3, seed=3)
    p = Params()
    f = init_feq(dvm, *fields, p)
    a = rk2_step(dvm, f, p)
    p.deriv = "dft"
    b = rk2_step(dvm, f, p)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


def test_windowed_derivative_of_single_modes():
    # The window is a reading (the paper does not give W): pinned here to its stated form.
    # For a pure x-mode of index m and a pure y-mode of index n, the windowed first
    # derivative is the unwindowed one times exp(-alpha (|m|/(N/2))^p), computed here from the
    # closed form, and a derivative along x leaves a y-mode's window out entirely.
    nx, ny, dx, dy, alpha, p = 32, 16, 0.1, 0.2, 36.0, 8.0
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    for m in (3, 9, 14):
        h = np.sin(2 * np.pi * m * x / nx) * np.ones((ny, 1))
        plain = spectral_deriv(h, 1, 0, dx, dy)
        wind = spectral_deriv(h, 1, 0, dx, dy, alpha, p)
        w = np.exp(-alpha * (m / (nx / 2)) ** p)
        assert np.allclose(wind, w * plain, rtol=0, atol=1e-13 * np.max(np.abs(plain)))
        # second derivative carries the window twice (composition of first derivatives)
        wind2 = spectral_deriv(h, 2, 0, dx, dy, alpha, p)
        plain2 = spectral_deriv(h, 2, 0, dx, dy)
        assert np.allclose(wind2, w * w * plain2, rtol=0, atol=1e-13 * np.max(np.abs(plain2)))
    for n in (2, 5, 7):
        g = np.cos(2 * np.pi * n * y / ny) * np.sin(2 * np.pi * 3 * x / nx)
        plain = spectral_deriv(g, 1, 0, dx, dy)
        wind = spectral_deriv(g, 1, 0, dx, dy, alpha, p)
        assert np.allclose(wind, np.exp(-alpha * (3 / (nx / 2)) ** p) * plain, rtol=0, atol=1e-13)


def test_keff_with_four_terms_is_eighth_order():
    # the 8th-order scheme of the D2V33 runs (Sec. 3.2) keeps the first four terms:
    # k - k_eff ~ c_4 phi^9, log-log slope ~9; and it is the arcsin series truncated there.
    N, dx = 4096, 1.0
    m = np.array([N * np.arcsin(0.5) / np.pi, N * np.arcsin(0.4) / np.pi])
    k = 2.0 * np.pi * m / (N * dx)
    err = k - keff(m, N, dx, terms=4)
    slope = np.log(err[0] / err[1]) / np.log(0.5 / 0.4)
    assert np.all(err > 0) and 9.0 <= slope <= 10.5
    phi = 0.3
    x = sympy.symbols("x")
    ser = sympy.series(sympy.asin(x), x, 0, 9).removeO()
    mm = N * np.arcsin(phi) / np.pi
    assert keff(mm, N, 2.0, terms=4) == pytest.approx(float(ser.subs(x, phi)), rel=1e-14)


def test_solution_filter_of_single_modes(dvm):
    # the solution filter scales the 2D mode (m_x, m_y) of every field by W(m_x) W(m_y),
    # W(m) = exp(-alpha (|m|/(N/2))^p), written out here from its definition; the Nyquist index
    # is damped by exp(-alpha); a uniform field is untouched; the step ends with it
    from oracle.model import Params, solution_filter, rk2_step, init_feq
    nx, ny, alpha, p = 32, 16, 36.0, 8.0
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    P = Params(filter_alpha=alpha, filter_p=p)
    for mx, my in ((3, 2), (11, 5), (16, 0), (0, 8)):
        h = np.cos(2 * np.pi * (mx * x / nx + my * y / ny)) + 1.0
        f = np.repeat(h[None], 16, axis=0)
        w = np.exp(-alpha * (mx / (nx / 2)) ** p) * np.exp(-alpha * (my / (ny / 2)) ** p)
        out = solution_filter(f, P)
        ref = np.cos(2 * np.pi * (mx * x / nx + my * y / ny)) * w + 1.0
        assert np.allclose(out, np.repeat(ref[None], 16, axis=0), rtol=0, atol=1e-13)
    import oracle, synthetic
    rl, rv = oracle.coexistence(0.9)
    fields = synthetic.slab(32, 16, rl, rv, 0.9, half_width=8, noise=1e-3, seed=5)
    f0 = init_feq(dvm, *fields, P)
    P0 = Params()
    assert np.allclose(rk2_step(dvm, f0, P), solution_filter(rk2_step(dvm, f0, P0), P), rtol=0, atol=1e-15)
