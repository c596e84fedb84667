"""The allocation-free diagnostics entry point (lbm_diagnostics_noalloc) against the regular
one (lbm_diagnostics), through the C ABI.

Callers that cannot allocate device memory (an application whose GPU memory is owned by
another allocator or budgeted at start-up, a service that must not grow its footprint later)
use the variant with the library's built-in scratch array. It must give the same diagnostics
as lbm_diagnostics on the same state, on consecutive calls that reuse the shared scratch, for
the k_eff series the state was run with. This file is named to be collected last, so that a
run stopping at its first failure has run every other test.
"""
import numpy as np
import pytest

import synthetic
import paper_1403_3746_gb300 as lbm
from paper_1403_3746_gb300 import build as lbm_build

pytestmark = pytest.mark.gpu
KEYS = ("mass", "px", "py", "energy", "umax")


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    lbm_build.build()
    lbm.lib()
    return torch


def _state(torch, nx, ny, steps, seed, **kw):
    p = lbm.default_params(**kw)
    rho, ux, uy, T = synthetic.spinodal(nx, ny, 1.0, 0.02, 0.9, seed=seed)
    x = np.arange(nx)[None, :] / nx
    ux = ux + 0.02 * np.sin(2 * np.pi * x)
    sim = lbm.Simulation(nx, ny, p)
    sim.init(rho, ux, uy, T)
    sim.step(steps)
    ref = sim.diagnostics()
    dev = [torch.empty((ny, nx), dtype=torch.float64, device="cuda") for _ in range(4)]
    sim.moments_device(*dev)
    sim.synchronize()
    sim.close()
    return p, ref, dev


def _close(got, ref, energy_rel=1e-12):
    for k in KEYS:
        rel = energy_rel if k == "energy" else 1e-12
        assert got[k] == pytest.approx(ref[k], rel=rel, abs=1e-14), k


def test_noalloc_matches_lbm_diagnostics_on_two_calls(torch_cuda):
    torch = torch_cuda
    p, ref, dev = _state(torch, 256, 128, 4, seed=21)
    first = lbm.diagnostics_noalloc(p, *dev)
    second = lbm.diagnostics_noalloc(p, *dev)
    _close(first, ref)
    _close(second, ref)
    # a different grid and window in between, then the first state again
    p2, ref2, dev2 = _state(torch, 64, 512, 3, seed=22, win_alpha=36.0)
    _close(lbm.diagnostics_noalloc(p2, *dev2), ref2)
    _close(lbm.diagnostics_noalloc(p, *dev), ref)


def test_noalloc_with_the_eighth_order_series(torch_cuda):
    # keff_terms = 4 (the 8th-order variant of Sec. 3.2): the energy's |grad rho|^2 term uses
    # the same truncated series as the handle's own diagnostics
    torch = torch_cuda
    p, ref, dev = _state(torch, 128, 128, 3, seed=23, keff_terms=4)
    _close(lbm.diagnostics_noalloc(p, *dev), ref)
    p8 = lbm.default_params()
    other = lbm.diagnostics_noalloc(p8, *dev)
    assert other["energy"] != pytest.approx(ref["energy"], rel=1e-12)


def test_noalloc_on_a_mixed_precision_state(torch_cuda):
    # LBM_MIXED: lbm_diagnostics differentiates the float32 density, this call the float64
    # copy of it, so the energy agrees to float32 rounding of the gradient term only
    torch = torch_cuda
    p, ref, dev = _state(torch, 128, 64, 3, seed=24, precision=lbm.LBM_MIXED)
    _close(lbm.diagnostics_noalloc(p, *dev), ref, energy_rel=1e-5)


def test_noalloc_refuses_a_capturing_stream(torch_cuda):
    torch = torch_cuda
    p, ref, dev = _state(torch, 64, 64, 2, seed=25)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        with pytest.raises(lbm.LbmError, match="captured"):
            lbm.diagnostics_noalloc(p, *dev, stream=s.cuda_stream)
        x = dev[0] * 2.0  # the capture is still usable after the refusal
        g.capture_end()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(x, dev[0] * 2.0)
    _close(lbm.diagnostics_noalloc(p, *dev), ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    big = [torch.zeros((1024, 2048), dtype=torch.float64, device="cuda") for _ in range(4)]
    with pytest.raises(lbm.LbmError, match="exceeds"):
        lbm.diagnostics_noalloc(lbm.default_params(), *big)
    small = [torch.ones((64, 64), dtype=torch.float64, device="cuda") for _ in range(4)]
    with pytest.raises(lbm.LbmError, match="keff_terms"):
        lbm.diagnostics_noalloc(lbm.default_params(keff_terms=9), *small)
