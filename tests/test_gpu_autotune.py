"""The launch-shape autotuner (lbm_autotune, lbm_batch_autotune): it leaves the state
unchanged, and runs with the tuned shapes give bit-for-bit the results of the default
shapes (per-row and per-column work does not depend on the tiling)."""
import numpy as np
import pytest

import oracle
import synthetic

import paper_1403_3746_gb300 as lbm
from paper_1403_3746_gb300 import build as lbm_build

pytestmark = pytest.mark.gpu
PHASE = dict(tau=1e-4, dt=1e-4, dx=1 / 256, dy=1 / 256, K=5e-6, q=-0.004, b=2.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    lbm_build.build()


def droplet(n):
    rl, rv = oracle.coexistence(0.9)
    return synthetic.droplet(n, n, n / 4, rl, rv, 0.9, width=2.0)


@pytest.mark.parametrize("precision,n", [(lbm.LBM_MIXED, 256), (lbm.LBM_FP64, 128), (lbm.LBM_MIXED, 64)])
def test_autotune_keeps_state_and_results(precision, n):
    p = lbm.default_params(precision=precision, **PHASE)
    fields = droplet(n)
    with lbm.Simulation(n, n, p) as a, lbm.Simulation(n, n, p) as b:
        a.init(*fields)
        b.init(*fields)
        a.step(3)
        b.step(3)
        before = a.get_f()
        mom = a.moments()
        g0 = a.geometry()
        g, ms = a.autotune()
        print(f"n={n} precision={precision}: default {g0}, tuned {g}, ms {ms}")
        assert a.geometry() == g and all(t > 0 for t in (ms[0], ms[2]))
        assert np.array_equal(a.get_f(), before)
        for x, y in zip(a.moments(), mom):
            assert np.array_equal(x, y)
        a.step(5)
        b.step(5)
        assert np.array_equal(a.get_f(), b.get_f())


def test_batch_autotune():
    sizes = [(128, 128), (64, 64), (128, 128), (32, 64)]
    p = lbm.default_params(precision=lbm.LBM_MIXED, **PHASE)
    fields = [droplet(nx) if nx == ny else synthetic.spinodal(nx, ny, 1.0, 0.02, 0.9, seed=5) for nx, ny in sizes]
    out = []
    for tune in (False, True):
        with lbm.Batch(sizes, p) as bt:
            for k, f in enumerate(fields):
                bt.init(k, *f)
            bt.step(2)
            if tune:
                bt.autotune()
                print([bt.geometry(k) for k in range(len(sizes))])
            bt.step(4)
            out.append([bt.get_f(k) for k in range(len(sizes))])
    for x, y in zip(*out):
        assert np.array_equal(x, y)


def test_autotune_needs_state():
    with lbm.Simulation(32, 32, lbm.default_params(**PHASE)) as s:
        with pytest.raises(lbm.LbmError, match="call out of order"):
            s.autotune()


def test_graph_with_unequal_tile_shapes():
    # one step graph holds the column pass and the flux pass (the same kernel) with different
    # tile widths, and a second simulation of the same size launches it with other shapes in
    # between: every launch must still run (the kernel's shared-memory allowance is the
    # device maximum), with results bit for bit those of the default shapes
    n = 256
    p = lbm.default_params(precision=lbm.LBM_MIXED, **PHASE)
    fields = droplet(n)
    with lbm.Simulation(n, n, p) as a, lbm.Simulation(n, n, p) as b, lbm.Simulation(n, n, p) as c:
        for s in (a, b, c):
            s.init(*fields)
        a.set_geometry((64, 1, 1, 4))
        b.set_geometry((4, 2, 2, 64))
        assert a.geometry() == (64, 1, 1, 4)
        for _ in range(3):
            a.step(2)
            b.step(2)
            c.step(2)
        ref = c.get_f()
        assert np.array_equal(a.get_f(), ref) and np.array_equal(b.get_f(), ref)
        with pytest.raises(lbm.LbmError, match="not valid"):
            a.set_geometry((3, 1, 1, 4))
        with pytest.raises(lbm.LbmError, match="not valid"):
            a.set_geometry((64, 1, 3, 4))
