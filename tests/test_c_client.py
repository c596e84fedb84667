"""The C ABI from a plain C99 program (no C++, no Python): the header compiles as C, the
library links, and its host-only entry points (Maxwell construction, launch plan, error
strings) run without a device."""
import os
import shutil
import subprocess

import pytest

from paper_1403_3746_gb300 import build as lbm_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SOURCE = r"""
#include <stdio.h>
#include "lbm_d2v16.h"

int main(void) {
    double rl = 0.0, rv = 0.0;
    int plan[18];
    int rc = lbm_maxwell(0.95, &rl, &rv);
    printf("maxwell %d %.7f %.7f\n", rc, rl, rv);
    rc = lbm_launch_plan(1024, 1024, LBM_MIXED, plan);
    printf("plan %d %d %d %d\n", rc, plan[0], plan[7], plan[9]);
    rc = lbm_launch_plan(6, 8, LBM_MIXED, plan);
    printf("bad %d %s\n", rc, lbm_strerror(rc));
    return 0;
}
"""


def test_c99_client(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lbm_build.build()
    src = tmp_path / "client.c"
    src.write_text(C_SOURCE)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lbm_build.LIB)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-l:" + os.path.basename(lbm_build.LIB),
                    "-Wl,-rpath," + libdir], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    # the coexistence densities the paper prints at T = 0.95 (Sec. 3.3): 1.462 / 0.579
    rc, rl, rv = out[0].split()[1:]
    assert rc == "0" and abs(float(rl) - 1.462) < 5e-4 and abs(float(rv) - 0.579) < 5e-4
    # 1024^2 mixed: 16-column tiles, one row per update CTA, transforms in the update kernel
    assert out[1].split()[1:] == ["0", "16", "1", "0"]
    assert out[2].split()[1] == "-1" and "invalid argument" in out[2]
