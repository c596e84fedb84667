"""Sec. 2.3, Eq. (3): spatial derivatives by FFT with the 16th-order modified wavenumber.

Readings:
* Eq. (3) is circular as printed (k_x on both sides). It is read as
      k_eff(k) = (2/dx) * sum_{n=0}^{7} c_n phi^(2n+1),  phi = sin(k dx / 2),
  with k = 2 pi m / (N dx) for the DFT index m in [-N/2, N/2), the truncated Maclaurin
  series of arcsin(phi) / (dx/2); the same per axis with dy for k_y.
* The Nyquist index m = -N/2 gets a first-derivative multiplier of 0, so that the
  derivative of a real field stays real.
* Every derivative used by the model is one inverse transform of a spectrum times a
  product of first-derivative multipliers d(m) = i W(m) k_eff(m) of the two axes
  (second derivatives are d^2, mixed ones d_x d_y): compositions of first derivatives.
* The window W of the "windowed" FFT scheme is not specified in the paper. It is read
  as a per-axis exponential filter W(m) = exp(-alpha (|m|/(N/2))^p) (Hou and Li, J.
  Comput. Phys. 226 (2007): alpha = 36, p = 36) applied with each first derivative
  along that derivative's own axis; alpha = 0 (W = 1) is Eq. (3) exactly. Against the paper
  the window is "parity unpinned" (its form is a reading); tests pin it to this definition.
"""
import numpy as np

# Eq. (3): the eight coefficients as printed.
C_KEFF = np.array([1.0, 1.0 / 6.0, 3.0 / 40.0, 5.0 / 112.0, 35.0 / 1152.0,
                   63.0 / 2816.0, 231.0 / 13312.0, 143.0 / 10240.0])


def dft_indices(N):
    """DFT index m of each FFT output position, in [-N/2, N/2)."""
    return np.rint(np.fft.fftfreq(N) * N).astype(np.int64)


def keff(m, N, dx, terms=8):
    """Eq. (3): modified wavenumber of DFT index m on an N-point axis of spacing dx. `terms`
    keeps the first terms of the series (8: Eq. (3), 16th order; 4: the 8th-order scheme of
    the D2V33 runs of Sec. 3.2)."""
    phi = np.sin(np.pi * np.asarray(m, dtype=np.float64) / N)
    s = np.zeros_like(phi)
    for n, c in enumerate(C_KEFF[:terms]):
        s = s + c * phi ** (2 * n + 1)
    return (2.0 / dx) * s


def window(N, alpha, p):
    """Spectral window W(m) = exp(-alpha (|m| / (N/2))^p) of the windowed FFT scheme
    (exponential filter; alpha = 0 gives W = 1)."""
    m = np.abs(dft_indices(N)).astype(np.float64)
    if alpha == 0.0:
        return np.ones(N)
    return np.exp(-alpha * (m / (N / 2.0)) ** p)


def deriv_multiplier(N, dx, alpha=0.0, p=36.0, terms=8):
    """d(m) = i W(m) k_eff(m) per FFT position, zero at the Nyquist index."""
    m = dft_indices(N)
    d = 1j * keff(m, N, dx, terms) * window(N, alpha, p)
    if N % 2 == 0:
        d[m == -N // 2] = 0.0
    return d


def spectral_deriv(h, ox, oy, dx, dy, alpha=0.0, p=36.0, terms=8, backend="fft"):
    """Spectral derivative d^(ox) / dx^(ox) d^(oy) / dy^(oy) of a real field h of shape (ny, nx):
    the composition of the first-derivative operators of each axis. backend "fft": numpy's FFT
    of the whole field; "dft": the same operator as explicit DFT sums along each axis
    (dft_deriv_matrix, O(N) work per output value, no FFT)."""
    ny, nx = h.shape
    if backend == "dft":
        out = h
        if ox:
            out = out @ dft_deriv_matrix(nx, dx, ox, alpha, p, terms).T
        if oy:
            out = dft_deriv_matrix(ny, dy, oy, alpha, p, terms) @ out
        return np.array(out, dtype=np.float64, copy=True)
    mult = (deriv_multiplier(nx, dx, alpha, p, terms)[None, :] ** ox
            * deriv_multiplier(ny, dy, alpha, p, terms)[:, None] ** oy)
    return np.fft.ifft2(mult * np.fft.fft2(h)).real


_DFT_CACHE = {}


def dft_deriv_matrix(N, dx, order=1, alpha=0.0, p=36.0, terms=8):
    """Real N x N matrix of the same operator along one axis, built from the DFT sums (no FFT):
    D[a, b] = (1/N) sum_m d(m)^order exp(2 pi i m (a - b) / N). It is circulant, so its first
    column c[k] = (1/N) sum_m d(m)^order exp(2 pi i m k / N) is summed directly (N terms for
    each of the N values of k) and D[a, b] = c[(a - b) mod N]."""
    key = (N, float(dx), order, float(alpha), float(p), terms)
    if key not in _DFT_CACHE:
        m = dft_indices(N)
        d = deriv_multiplier(N, dx, alpha, p, terms) ** order
        k = np.arange(N)
        c = np.zeros(N, dtype=np.complex128)
        for j in range(N):
            c += d[j] * np.exp(2j * np.pi * ((m[j] * k) % N) / N)
        c = (c / N).real
        a = np.arange(N)
        _DFT_CACHE[key] = c[(a[:, None] - a[None, :]) % N]
    return _DFT_CACHE[key]
