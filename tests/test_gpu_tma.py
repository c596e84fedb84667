"""The TMA-fed column pass with two or one staging buffers (LBM_COL_TMA, LBM_COL_TMA1) and the
direct pass with L2 lookahead (LBM_COL_LOOKAHEAD) against the direct one: bit for bit the same
states over every legal tile width, in both precisions, for single grids and stacked batch
instances; the TMA pass's bounded waits end a starved launch with LBM_ERR_TIMEOUT instead of a
hang."""
import numpy as np
import pytest

import synthetic
import paper_1403_3746_gb300 as lbm
from paper_1403_3746_gb300 import build as lbm_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    lbm_build.build()


def _fields(nx, ny, seed=51):
    rl, rv = lbm.maxwell(0.9)
    rho, ux, uy, T = synthetic.droplet(nx, ny, min(nx, ny) / 4, rl, rv, 0.9, noise=1e-3, seed=seed)
    return rho, ux + 0.01 * np.sin(2 * np.pi * np.arange(nx) / nx)[None, :], uy, T


def _run(nx, ny, precision, W, kinds, steps=3):
    with lbm.Simulation(nx, ny, lbm.default_params(precision=precision)) as s:
        s.init(*_fields(nx, ny))
        g = list(s.geometry())
        g[0] = g[3] = W
        s.set_geometry(g)
        s.set_pass_kinds(kinds)
        assert s.pass_kinds()[:len(kinds)] == tuple(kinds)
        s.step(steps)
        return s.get_f()


@pytest.mark.parametrize("kind", [lbm.LBM_COL_TMA, lbm.LBM_COL_LOOKAHEAD, lbm.LBM_COL_TMA1])
@pytest.mark.parametrize("precision", [lbm.LBM_FP64, lbm.LBM_MIXED])
@pytest.mark.parametrize("nx,ny", [(64, 64), (256, 128), (32, 1024), (1024, 16), (16, 4096)])
def test_column_pass_kinds_are_bitwise_the_direct_one(kind, precision, nx, ny):
    es = 8 if precision == lbm.LBM_FP64 else 4
    plan = lbm.launch_plan(nx, ny, precision)
    widths = [w for w in (2, 4, 8, 16, 32) if w <= nx and w * es >= 16 and w * es <= 256]
    ref = _run(nx, ny, precision, plan["col_width"], (lbm.LBM_COL_DIRECT, lbm.LBM_COL_DIRECT))
    tried = 0
    for W in widths:
        try:
            got = _run(nx, ny, precision, W, (kind, kind))
        except lbm.LbmError as e:  # a width this shape cannot take (threads or shared memory)
            assert "not valid" in str(e) or "cannot take" in str(e), str(e)
            continue
        tried += 1
        assert np.array_equal(got, ref), (W, float(np.max(np.abs(got - ref))))
    assert tried >= 1


def test_default_one_buffer_tma_in_a_batch_matches_separate_runs():
    # columns of 2048 points take the one-buffer TMA form by default, here with three instances
    # stacked in one size group (tensor maps over the stacked rows) next to a second group
    sizes = [(16, 2048)] * 3 + [(32, 1024)] * 2
    p = lbm.default_params(precision=lbm.LBM_MIXED)
    with lbm.Batch(sizes, p) as b:
        for k, (nx, ny) in enumerate(sizes):
            b.init(k, *_fields(nx, ny, seed=70 + k))
        b.step(3)
        got = [b.get_f(k) for k in range(len(sizes))]
    for k, (nx, ny) in enumerate(sizes):
        with lbm.Simulation(nx, ny, p) as s:
            s.init(*_fields(nx, ny, seed=70 + k))
            s.set_pass_kinds((lbm.LBM_COL_DIRECT, lbm.LBM_COL_DIRECT))
            s.step(3)
            assert np.array_equal(s.get_f(), got[k]), k


def test_tma_in_a_batch_matches_separate_runs():
    sizes = [(64, 64)] * 3 + [(128, 32)] * 2
    p = lbm.default_params(precision=lbm.LBM_MIXED)
    with lbm.Batch(sizes, p) as b:
        for k, (nx, ny) in enumerate(sizes):
            b.init(k, *_fields(nx, ny, seed=60 + k))
        b.autotune()
        b.step(4)
        got = [b.get_f(k) for k in range(len(sizes))]
    for k, (nx, ny) in enumerate(sizes):
        with lbm.Simulation(nx, ny, p) as s:
            s.init(*_fields(nx, ny, seed=60 + k))
            s.set_pass_kinds((lbm.LBM_COL_TMA, lbm.LBM_COL_TMA))
            s.step(4)
            assert np.array_equal(s.get_f(), got[k]), k


@pytest.mark.parametrize("kind", [lbm.LBM_COL_TMA, lbm.LBM_COL_TMA1])
def test_starved_copies_end_in_a_timeout_not_a_hang(kind):
    nx = ny = 128
    with lbm.Simulation(nx, ny, lbm.default_params(precision=lbm.LBM_MIXED)) as s:
        s.init(*_fields(nx, ny))
        s.step(2)
        blob = s.get_state()
        ref_next = None
        s.set_pass_kinds((kind, kind))
        s.fault_inject(lbm.LBM_FAULT_STARVE_COPIES, 200000)  # about 0.1 ms per wait
        s.step(1)
        with pytest.raises(lbm.LbmError) as ei:
            s.synchronize()
        assert ei.value.code == lbm.LBM_ERR_TIMEOUT
        s.synchronize()  # reported once; the context stays usable
        # back to normal operation: resume from the checkpoint and step on
        s.fault_inject(lbm.LBM_FAULT_NONE)
        s.set_state(blob)
        s.step(1)
        s.synchronize()
        got = s.get_f()
    with lbm.Simulation(nx, ny, lbm.default_params(precision=lbm.LBM_MIXED)) as r:
        r.init(*_fields(nx, ny))
        r.step(3)
        ref_next = r.get_f()
    assert np.array_equal(got, ref_next)


@pytest.mark.parametrize("precision,nx,ny,widths", [
    (lbm.LBM_MIXED, 64, 1024, (32, 64)), (lbm.LBM_MIXED, 32, 2048, (16, 32)),
    (lbm.LBM_MIXED, 64, 4096, (8, 16)), (lbm.LBM_FP64, 32, 4096, (4, 8)), (lbm.LBM_FP64, 64, 512, (16, 32))])
def test_cluster_split_column_tiles_are_bitwise_the_plain_ones(precision, nx, ny, widths):
    # tiles wider than one CTA's threads: each line is split over a cluster of 2 or 4 CTAs that
    # exchange points through distributed shared memory; the arithmetic is unchanged
    plan = lbm.launch_plan(nx, ny, precision)
    ref = _run(nx, ny, precision, plan["col_width"], (lbm.LBM_COL_DIRECT, lbm.LBM_COL_DIRECT))
    for W in widths:
        got = _run(nx, ny, precision, W, (lbm.LBM_COL_DIRECT, lbm.LBM_COL_DIRECT))
        assert np.array_equal(got, ref), (W, float(np.max(np.abs(got - ref))))


@pytest.mark.parametrize("nx,ny,cs", [(2048, 8, 2), (4096, 8, 2), (4096, 8, 4)])
def test_cluster_split_update_rows_are_bitwise_the_plain_ones(nx, ny, cs):
    # float32 rows of 2048+ (4096 for four): a cluster of cs CTAs splits each row's line
    # transforms and node loop
    ref = _run(nx, ny, lbm.LBM_MIXED, 4, (lbm.LBM_COL_DIRECT, lbm.LBM_COL_DIRECT, 1))
    got = _run(nx, ny, lbm.LBM_MIXED, 4, (lbm.LBM_COL_DIRECT, lbm.LBM_COL_DIRECT, cs))
    assert np.array_equal(got, ref), float(np.max(np.abs(got - ref)))
    with lbm.Simulation(256, 8, lbm.default_params(precision=lbm.LBM_MIXED)) as s:
        s.init(*_fields(256, 8))
        with pytest.raises(lbm.LbmError, match="2048"):
            s.set_pass_kinds((lbm.LBM_COL_DIRECT, lbm.LBM_COL_DIRECT, 2))

