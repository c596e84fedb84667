"""The allocation-free diagnostics entry point (lbm_diagnostics_noalloc) against the regular
one (lbm_diagnostics), through the C ABI.

Callers that cannot allocate device memory (for example during CUDA-graph stream capture,
or inside an application that owns all GPU memory) use the variant with the library's
built-in scratch array. It must give the same diagnostics as lbm_diagnostics on the same
state, on consecutive calls that reuse the shared scratch. This file is named to be
collected last, so that a run stopping at its first failure has run every other test.
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


def _close(got, ref):
    for k in KEYS:
        assert got[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-14), k


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


def test_noalloc_rejects_sizes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    big = [torch.zeros((1024, 2048), dtype=torch.float64, device="cuda") for _ in range(4)]
    with pytest.raises(lbm.LbmError, match="exceeds"):
        lbm.diagnostics_noalloc(lbm.default_params(), *big)
