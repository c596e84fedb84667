"""Checkpoint and resume through the C ABI: k steps, lbm_get_state, k more steps equals 2k
uninterrupted steps bit for bit, on the same handle and on a fresh one, in both precisions and
for a batch instance; blobs of other sizes, parameters or corrupted headers are refused."""
import numpy as np
import pytest

import synthetic
import paper_1403_3746_gb300 as lbm
from paper_1403_3746_gb300 import build as lbm_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    lbm_build.build()


def _fields(nx, ny, seed=31):
    rl, rv = lbm.maxwell(0.9)
    rho, ux, uy, T = synthetic.droplet(nx, ny, nx / 4, rl, rv, 0.9, noise=1e-3, seed=seed)
    return rho, ux + 0.01 * np.sin(2 * np.pi * np.arange(nx) / nx)[None, :], uy, T


@pytest.mark.parametrize("precision", [lbm.LBM_FP64, lbm.LBM_MIXED])
def test_k_steps_checkpoint_k_steps_equals_2k_steps(precision):
    nx, ny, k = 64, 32, 7
    p = lbm.default_params(precision=precision)
    fields = _fields(nx, ny)
    with lbm.Simulation(nx, ny, p) as a:
        a.init(*fields)
        a.step(2 * k)
        f2k, m2k, d2k = a.get_f(), a.moments(), a.diagnostics()
    with lbm.Simulation(nx, ny, p) as b:
        b.init(*fields)
        b.step(k)
        blob = b.get_state()
        assert len(blob) == lbm.state_bytes(nx, ny, precision)
        b.step(3)  # moves on; the blob brings it back
        b.set_state(blob)
        assert b.diagnostics()["steps"] == k
        b.step(k)
        assert np.array_equal(b.get_f(), f2k)
        assert all(np.array_equal(x, y) for x, y in zip(b.moments(), m2k))
        assert b.diagnostics()["steps"] == 2 * k
    with lbm.Simulation(nx, ny, p) as c:  # a fresh handle, never initialised
        c.set_state(blob)
        c.step(k)
        assert np.array_equal(c.get_f(), f2k)
        d = c.diagnostics()
        assert d["steps"] == 2 * k and d["energy"] == d2k["energy"]


def test_batch_instance_resumes_bitwise():
    sizes = [(32, 32), (64, 32), (32, 32)]
    p = lbm.default_params(precision=lbm.LBM_MIXED)
    with lbm.Batch(sizes, p) as b:
        for i, (nx, ny) in enumerate(sizes):
            b.init(i, *_fields(nx, ny, seed=40 + i))
        b.step(5)
        blob = b.get_state(1)
        b.step(5)
        ref = b.get_f(1)
        b.set_state(1, blob)
        assert b.diagnostics(1)["steps"] == 5
    with lbm.Simulation(64, 32, p) as s:
        s.set_state(blob)
        s.step(5)
        assert np.array_equal(s.get_f(), ref)


def test_foreign_blobs_are_refused():
    p = lbm.default_params()
    with lbm.Simulation(32, 32, p) as a:
        a.init(*_fields(32, 32))
        a.step(2)
        blob = a.get_state()
        f = a.get_f()
        for other in (lbm.Simulation(64, 32, p), lbm.Simulation(32, 32, lbm.default_params(K=6e-6)),
                      lbm.Simulation(32, 32, lbm.default_params(precision=lbm.LBM_MIXED))):
            with other, pytest.raises(lbm.LbmError, match="invalid argument"):
                other.set_state(blob)
        bad = bytearray(blob)
        bad[0] = ord("X")
        with pytest.raises(lbm.LbmError, match="version-1"):
            a.set_state(bytes(bad))
        with pytest.raises(lbm.LbmError, match="truncated"):
            a.set_state(blob[:-8])
        nan = bytearray(blob)
        nan[64:72] = np.array([np.nan]).tobytes()
        with pytest.raises(lbm.LbmError, match="not finite"):
            a.set_state(bytes(nan))
        assert np.array_equal(a.get_f(), f)  # refused blobs change nothing


def _same_diag(got, ref, energy_rel):
    # the fused form sums the same per-node terms in another partition, and its d_x rho comes
    # from the macro pass's line (rho, T) instead of (rho, 0): the sums agree to rounding, the
    # energy's gradient part to float32 rounding of that derivative
    assert got["steps"] == ref["steps"]
    for k in ("mass", "px", "py", "umax"):
        assert got[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-14), k
    assert got["energy"] == pytest.approx(ref["energy"], rel=energy_rel), "energy"


def test_pipelined_diagnostics_match_the_blocking_call():
    # LBM_MIXED: each request rides on the next step's first macro pass (fused); the last one,
    # with no step after it, is computed on its own at lbm_diagnostics_end
    nx, ny = 128, 64
    p = lbm.default_params(precision=lbm.LBM_MIXED)
    with lbm.Simulation(nx, ny, p) as a, lbm.Simulation(nx, ny, p) as b:
        a.init(*_fields(nx, ny))
        b.init(*_fields(nx, ny))
        ref = []
        for _ in range(4):
            a.step(3)
            ref.append(a.diagnostics())
        got = []
        for k in range(4):
            b.step(3)
            b.diagnostics_begin()
            if k > 0:
                got.append(b.diagnostics_end())  # the previous step's request, while this one runs
        got.append(b.diagnostics_end())
        for g, r in zip(got, ref):
            _same_diag(g, r, 1e-7)
        assert np.array_equal(a.get_f(), b.get_f())  # the fused requests change nothing else
        with pytest.raises(lbm.LbmError, match="pending"):
            b.diagnostics_end()
        b.diagnostics_begin()
        b.diagnostics_begin()
        with pytest.raises(lbm.LbmError, match="two requests"):
            b.diagnostics_begin()


@pytest.mark.parametrize("precision,flags,filt", [(lbm.LBM_FP64, 0, 0.0), (lbm.LBM_MIXED, lbm.LBM_FLAG_EULER, 0.0),
                                                  (lbm.LBM_MIXED, 0, 36.0), (lbm.LBM_MIXED_RHO64, 0, 0.0),
                                                  (lbm.LBM_MIXED, lbm.LBM_FLAG_NO_FORCE, 0.0)])
def test_diagnostics_requests_in_every_form(precision, flags, filt):
    # fused (LBM_MIXED with the forcing chain) or standalone (the others): a request returns the
    # diagnostics of the state at lbm_diagnostics_begin, also when the state is replaced or
    # the step never comes
    nx, ny = 64, 64
    p = lbm.default_params(precision=precision, flags=flags, filter_alpha=filt)
    exact = precision != lbm.LBM_MIXED or flags & lbm.LBM_FLAG_NO_FORCE
    with lbm.Simulation(nx, ny, p) as s:
        s.init(*_fields(nx, ny))
        s.step(2)
        ref0 = s.diagnostics()
        blob = s.get_state()
        s.diagnostics_begin()
        s.step(1)  # the request rides on this step where it can
        ref1 = s.diagnostics()
        got0 = s.diagnostics_end()
        s.diagnostics_begin()  # no step follows: computed at lbm_diagnostics_end
        got1 = s.diagnostics_end()
        s.diagnostics_begin()
        s.set_state(blob)  # the state is replaced before any step: the request is of the old one
        s.step(1)
        got2 = s.diagnostics_end()
        assert s.diagnostics()["steps"] == 3
    if exact:
        assert got0 == ref0 and got1 == ref1 and got2 == ref1
    else:
        _same_diag(got0, ref0, 1e-7)
        assert got1 == ref1 and got2 == ref1
