"""The seeded input generators (shared by the oracle and the GPU tests; no arithmetic of the
method): SplitMix64 against the published reference outputs, the uniform mapping, and the
shapes and symmetries of the initial fields."""
import numpy as np

import synthetic
from synthetic.fields import splitmix64, uniform01


def test_splitmix64_reference_outputs():
    # the first outputs of the reference SplitMix64 generator started from state 0
    # (Steele, Lea & Flood 2014; the widely used public-domain C version by Vigna)
    assert [int(v) for v in splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # the stream is addressable: outputs k.. equal the tail of outputs 0..
    assert np.array_equal(splitmix64(7, 5, offset=3), splitmix64(7, 8)[3:])


def test_uniform01_range_and_moments():
    u = uniform01(11, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3 and abs(u.var() - 1 / 12) < 2e-3
    # 53-bit grid
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))


def test_fields_shapes_and_symmetry():
    rho, ux, uy, T = synthetic.slab(64, 8, 1.6, 0.4, 0.9, width=2.0)
    assert rho.shape == (8, 64) and np.all(ux == 0) and np.all(uy == 0) and np.all(T == 0.9)
    # a noise-free slab centred in the box is mirror-symmetric in x about the centre
    assert np.allclose(rho[:, 1:], rho[:, 1:][:, ::-1])
    assert rho.max() <= 1.6 + 1e-12 and rho.min() >= 0.4 - 1e-12
    d = synthetic.droplet(32, 32, 8, 1.6, 0.4, 0.9, width=2.0)[0]
    assert np.allclose(d, d.T) and d[16, 16] > 1.5 and d[0, 0] < 0.45
    s1 = synthetic.spinodal(16, 16, 1.0, 0.01, 0.9, seed=2)[0]
    s2 = synthetic.spinodal(16, 16, 1.0, 0.01, 0.9, seed=2)[0]
    assert np.array_equal(s1, s2) and np.abs(s1 - 1.0).max() <= 0.01
