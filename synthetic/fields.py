"""Seeded initial-condition generators.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the k-th output (k = 0, 1, ...)
of stream `seed` is mix(seed + (k + 1) * 0x9E3779B97F4A7C15) with the published
mixing function. A uniform double in [0, 1) takes the top 53 bits.
Noise is drawn in row-major order (y outer, x inner), one number per node.

Grid coordinates are integer node indices x = 0..nx-1, y = 0..ny-1; every array
returned is float64 with shape (ny, nx).
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, n, offset=0):
    """Outputs offset..offset+n-1 of the SplitMix64 stream started at `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed % (1 << 64)) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed, n, offset=0):
    """n doubles uniform in [0, 1): top 53 bits of SplitMix64 times 2^-53."""
    z = splitmix64(seed, n, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_sym(seed, n, amplitude, offset=0):
    """n doubles uniform in [-amplitude, amplitude)."""
    return amplitude * (2.0 * uniform01(seed, n, offset) - 1.0)


def _noise(seed, nx, ny, amplitude):
    if amplitude == 0.0:
        return np.zeros((ny, nx))
    return uniform_sym(seed, nx * ny, amplitude).reshape(ny, nx)


def slab(nx, ny, rho_l, rho_v, T, center=None, half_width=None, width=2.0,
         noise=0.0, seed=1):
    """Planar liquid slab along y: rho = rho_v + (rho_l - rho_v)/2 (1 + tanh((h - |x - c|)/w)),
    plus additive uniform noise of the given amplitude, u = 0, uniform T."""
    c = nx / 2.0 if center is None else center
    h = nx / 4.0 if half_width is None else half_width
    x = np.arange(nx, dtype=np.float64)[None, :]
    prof = rho_v + 0.5 * (rho_l - rho_v) * (1.0 + np.tanh((h - np.abs(x - c)) / width))
    rho = np.broadcast_to(prof, (ny, nx)).copy() + _noise(seed, nx, ny, noise)
    z = np.zeros((ny, nx))
    return rho, z, z.copy(), np.full((ny, nx), float(T))


def droplet(nx, ny, R, rho_l, rho_v, T, width=2.0, center=None, noise=0.0, seed=3):
    """Circular droplet of radius R at the box centre (or `center`): rho = rho_v +
    (rho_l - rho_v)/2 (1 + tanh((R - r)/w)), u = 0, uniform T."""
    cx, cy = (nx / 2.0, ny / 2.0) if center is None else center
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    rho = rho_v + 0.5 * (rho_l - rho_v) * (1.0 + np.tanh((R - r) / width))
    rho = rho + _noise(seed, nx, ny, noise)
    z = np.zeros((ny, nx))
    return rho, z, z.copy(), np.full((ny, nx), float(T))


def spinodal(nx, ny, rho0, amplitude, T, seed=2, multiplicative=True):
    """Uniform state rho0 with seeded noise: rho0 (1 + U[-a, a]) (multiplicative) or
    rho0 + U[-a, a] (additive); u = 0, uniform T."""
    n = _noise(seed, nx, ny, amplitude)
    rho = rho0 * (1.0 + n) if multiplicative else rho0 + n
    z = np.zeros((ny, nx))
    return rho, z, z.copy(), np.full((ny, nx), float(T))


def quench_temperatures(seed, count, lo=0.80, hi=0.95):
    """Per-instance quench temperatures uniform in [lo, hi), instance k taking output k."""
    return lo + (hi - lo) * uniform01(seed, count)
