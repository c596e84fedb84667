"""Batches of independent simulations (lbm_batch_*) and the graph-launched step.

A batched instance is the same computation as a separate handle of the same size and
parameters (the row passes are row-local, the column passes take the instance from the
grid's z index), so its state must agree with a separate run bit for bit; one instance is
also checked against the FP64 oracle. lbm_step replays a captured CUDA graph unless
per-launch timing is on (direct launches): both must give identical states.
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

PHASE = dict(tau=1e-4, dt=1e-4, dx=1 / 256, dy=1 / 256, K=5e-6, q=-0.004, b=2.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    lbm_build.build()


def fields_for(k, nx, ny, T=0.9):
    """Instance k: a slab, a droplet or a spinodal state, each from its own seed."""
    rl, rv = oracle.coexistence(T)
    kind = k % 3
    if kind == 0:
        return synthetic.slab(nx, ny, rl, rv, T, center=nx / 2, half_width=nx / 4, width=2.0,
                              noise=1e-4, seed=100 + k)
    if kind == 1:
        return synthetic.droplet(nx, ny, min(nx, ny) / 4, rl, rv, T, width=2.0)
    return synthetic.spinodal(nx, ny, 1.0, 0.02, T, seed=200 + k)


def separate_run(fields, steps, p):
    ny, nx = fields[0].shape
    with lbm.Simulation(nx, ny, p) as s:
        s.init(*fields)
        s.step(steps)
        return s.get_f(), s.moments(), s.diagnostics()


@pytest.mark.parametrize("precision", [lbm.LBM_FP64, lbm.LBM_MIXED])
def test_batch_matches_separate_runs_bitwise(precision):
    sizes = [(64, 64), (32, 128), (64, 64), (128, 32), (64, 64), (32, 128), (16, 16)]
    p = lbm.default_params(precision=precision, **PHASE)
    steps = 12
    fields = [fields_for(k, nx, ny) for k, (nx, ny) in enumerate(sizes)]
    with lbm.Batch(sizes, p) as b:
        assert len(b) == len(sizes)
        for k, fl in enumerate(fields):
            b.init(k, *fl)
        b.step(steps // 2)
        b.step(steps - steps // 2)
        for k, fl in enumerate(fields):
            f_ref, m_ref, d_ref = separate_run(fl, steps, p)
            f_b = b.get_f(k)
            assert np.array_equal(f_b, f_ref), f"instance {k} {sizes[k]}: f differs"
            for a, r in zip(b.moments(k), m_ref):
                assert np.array_equal(a, r), f"instance {k}: moments differ"
            d = b.diagnostics(k)
            assert d["steps"] == steps
            for key in ("mass", "px", "py", "energy", "umax"):
                assert d[key] == d_ref[key], (k, key)


def test_batched_instance_against_oracle():
    sizes = [(32, 64), (32, 64), (64, 32)]
    p = lbm.default_params(**PHASE)
    steps = 6
    fields = [fields_for(k, nx, ny) for k, (nx, ny) in enumerate(sizes)]
    with lbm.Batch(sizes, p) as b:
        for k, fl in enumerate(fields):
            b.init(k, *fl)
        b.step(steps)
        op = oracle.Params(**PHASE)
        d = D2V16(op.eta0)
        for k in (1, 2):
            f = init_feq(d, *fields[k], op)
            for _ in range(steps):
                f = rk2_step(d, f, op)
            fg = b.get_f(k)
            floor = 1e-2 * np.max(np.abs(f))
            err = max(float(np.max(np.abs(fg[i] - f[i])) / max(np.max(np.abs(f[i])), floor)) for i in range(16))
            print(f"instance {k}: max f err {err:.3e}")
            assert err <= 1e-10


def test_reinit_one_instance_leaves_the_others():
    sizes = [(32, 32)] * 3
    p = lbm.default_params(**PHASE)
    fields = [fields_for(k, 32, 32) for k in range(3)]
    with lbm.Batch(sizes, p) as b:
        for k, fl in enumerate(fields):
            b.init(k, *fl)
        b.step(4)
        before = [b.get_f(k) for k in range(3)]
        b.init(1, *fields[0])
        assert np.array_equal(b.get_f(0), before[0])
        assert np.array_equal(b.get_f(2), before[2])
        assert b.diagnostics(1)["steps"] == 0 and b.diagnostics(0)["steps"] == 4
        b.step(4)
        # instance 1 now repeats instance 0's run from its initial state
        assert np.array_equal(b.get_f(1), before[0])


def test_batch_errors():
    p = lbm.default_params(**PHASE)
    with pytest.raises(lbm.LbmError, match="invalid argument"):
        lbm.Batch([], p)
    with pytest.raises(lbm.LbmError, match="powers of two"):
        lbm.Batch([(32, 32), (48, 32)], p)
    with lbm.Batch([(32, 32), (16, 16)], p) as b:
        b.init(0, *fields_for(0, 32, 32))
        with pytest.raises(lbm.LbmError, match="call out of order"):
            b.step(1)
        with pytest.raises(lbm.LbmError, match="call out of order"):
            b.get_f(1)
        with pytest.raises(lbm.LbmError, match="invalid argument"):
            b.diagnostics(2)
        with pytest.raises(ValueError):
            b.init(1, *fields_for(0, 32, 32))


@pytest.mark.parametrize("precision", [lbm.LBM_FP64, lbm.LBM_MIXED])
def test_graph_step_equals_direct_launches(precision):
    p = lbm.default_params(precision=precision, **PHASE)
    fl = fields_for(1, 128, 64)
    out = []
    for timing in (False, True):
        with lbm.Simulation(128, 64, p) as s:
            s.timing(timing)
            s.init(*fl)
            s.step(3)
            s.step(5)
            out.append(s.get_f())
            if timing:
                assert s.timing_read("update")[1] == 16
    assert np.array_equal(out[0], out[1])
