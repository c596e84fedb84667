"""Large deformation of a rectangular droplet (Sec. 3.3) with the temperature held at 0.95
(isothermal mode): the 118 x 14 rectangle starts to contract along its length, mass is
conserved, and the mixed path follows the FP64 path."""
import numpy as np
import pytest

import paper_1403_3746_gb300 as lbm
from paper_1403_3746_gb300 import build as lbm_build
from paper_1403_3746_gb300 import droplet as dr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    lbm_build.build()


def test_rectangle_contracts_and_paths_agree():
    runs = {prec: dr.deform(20000, 10000, n=256, precision=prec) for prec in (lbm.LBM_FP64, lbm.LBM_MIXED)}
    for prec, r in runs.items():
        print(prec, [(round(x["t"], 2), round(x["aspect"], 4), f'{x["umax"]:.3e}') for x in r])
        assert all(x["finite"] for x in r)
        assert r[0]["aspect"] == pytest.approx(118 / 14, rel=5e-3)
        assert r[0]["aspect"] > r[1]["aspect"] > r[2]["aspect"]
    r64, r32 = runs[lbm.LBM_FP64], runs[lbm.LBM_MIXED]
    assert abs(r64[-1]["mass"] - r64[0]["mass"]) <= 1e-11 * r64[0]["mass"]
    assert abs(r32[-1]["mass"] - r32[0]["mass"]) <= 2e-6 * r32[0]["mass"]
    assert abs(r32[-1]["aspect"] / r64[-1]["aspect"] - 1) < 1e-2
    assert abs(r32[-1]["umax"] / r64[-1]["umax"] - 1) < 1e-2
