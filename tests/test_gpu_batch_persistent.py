"""The persistent batch form (LBM_BATCH_PERSISTENT): one kernel launch per step whose CTAs take
(stage, pass, size group, instance, tile) items from a queue, each waiting (bounded) for the
previous pass of its own instance. Every tile computes exactly what the per-pass kernels
compute, so the states must equal the graph form's and separate runs' bit for bit; a withheld
completion must end in LBM_ERR_TIMEOUT, not a hang."""
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


def fields_for(k, nx, ny):
    rl, rv = oracle.coexistence(0.9)
    if k % 2 == 0:
        return synthetic.droplet(nx, ny, min(nx, ny) / 4, rl, rv, 0.9, noise=1e-3, seed=300 + k)
    return synthetic.spinodal(nx, ny, 1.0, 0.02, 0.85 + 0.01 * (k % 5), seed=400 + k)


def run_batch(sizes, form, steps, **kw):
    p = lbm.default_params(precision=lbm.LBM_MIXED, **dict(PHASE, **kw))
    with lbm.Batch(sizes, p) as b:
        for k, (nx, ny) in enumerate(sizes):
            b.init(k, *fields_for(k, nx, ny))
        b.set_form(form)
        assert b.form() == form
        b.step(steps)
        b.synchronize()
        return [b.get_f(k) for k in range(len(sizes))], [b.diagnostics(k)["steps"] for k in range(len(sizes))]


@pytest.mark.parametrize("kw", [{}, dict(flags=lbm.LBM_FLAG_ISOTHERMAL, T_iso=0.9)])
def test_persistent_form_is_bitwise_the_graph_form(kw):
    sizes = [(128, 128), (256, 128), (128, 128), (512, 256), (128, 1024), (256, 128)]  # four sizes
    got, steps = run_batch(sizes, lbm.LBM_BATCH_PERSISTENT, 6, **kw)
    ref, _ = run_batch(sizes, lbm.LBM_BATCH_GRAPH, 6, **kw)
    assert steps == [6] * len(sizes)
    for k in range(len(sizes)):
        assert np.isfinite(got[k]).all()
        assert np.array_equal(got[k], ref[k]), (k, float(np.max(np.abs(got[k] - ref[k]))))
    # and a separate handle of one instance
    nx, ny = sizes[3]
    p = lbm.default_params(precision=lbm.LBM_MIXED, **dict(PHASE, **kw))
    with lbm.Simulation(nx, ny, p) as s:
        s.init(*fields_for(3, nx, ny))
        s.step(6)
        assert np.array_equal(s.get_f(), got[3])


def test_persistent_form_refuses_what_it_cannot_take():
    with lbm.Batch([(64, 64)], lbm.default_params(precision=lbm.LBM_MIXED)) as b:
        with pytest.raises(lbm.LbmError, match="unsupported"):
            b.set_form(lbm.LBM_BATCH_PERSISTENT)
    with lbm.Batch([(128, 128)], lbm.default_params()) as b:  # float64
        with pytest.raises(lbm.LbmError, match="unsupported"):
            b.set_form(lbm.LBM_BATCH_PERSISTENT)
    sizes = [(128, 128), (256, 256), (512, 512), (128, 256), (256, 128)]  # five sizes
    with lbm.Batch(sizes, lbm.default_params(precision=lbm.LBM_MIXED)) as b:
        with pytest.raises(lbm.LbmError, match="unsupported"):
            b.set_form(lbm.LBM_BATCH_PERSISTENT)


def test_withheld_completion_ends_in_a_timeout():
    sizes = [(128, 128), (256, 256)]
    p = lbm.default_params(precision=lbm.LBM_MIXED, **PHASE)
    with lbm.Batch(sizes, p) as b:
        for k, (nx, ny) in enumerate(sizes):
            b.init(k, *fields_for(k, nx, ny))
        b.set_form(lbm.LBM_BATCH_PERSISTENT)
        b.fault_inject(lbm.LBM_FAULT_WITHHOLD_COMPLETION, 400000)  # about 0.2 ms per wait
        b.step(1)
        with pytest.raises(lbm.LbmError) as ei:
            b.synchronize()
        assert ei.value.code == lbm.LBM_ERR_TIMEOUT
        b.synchronize()  # reported once; the batch stays usable
        b.fault_inject(lbm.LBM_FAULT_NONE)
        for k, (nx, ny) in enumerate(sizes):
            b.init(k, *fields_for(k, nx, ny))
        b.step(2)
        b.synchronize()
        got = [b.get_f(k) for k in range(len(sizes))]
    ref, _ = run_batch(sizes, lbm.LBM_BATCH_GRAPH, 2)
    for k in range(len(sizes)):
        assert np.array_equal(got[k], ref[k])
