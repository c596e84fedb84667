"""Writes spinodal256_<steps>.npz: the oracle's state after `steps` Runge-Kutta steps (2000 by
default; 5000, the whole quench of the parity workload, with --steps 5000) of the 256 x 256
spinodal quench (rho = 1 (1 + U[-0.01, 0.01]), seed 2, u = 0, T = 0.9; phase-separation set of
Sec. 3.2 with q = -0.004), sampled: rho, u_x, u_y, T on every 16th row and the 16 distributions on
every 64th row. Calls only the oracle and the input generators.

    python tests/golden/make_spinodal256.py [--steps 5000]
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synthetic  # noqa: E402
from oracle.dvm import D2V16  # noqa: E402
from oracle.model import Params, init_feq, rk2_step  # noqa: E402

N, SEED = 256, 2
MOMENT_ROWS = np.arange(0, N, 16)
F_ROWS = np.arange(0, N, 64)


def main():
    steps = int(sys.argv[sys.argv.index("--steps") + 1]) if "--steps" in sys.argv else 2000
    p = Params()
    d = D2V16(p.eta0)
    f = init_feq(d, *synthetic.spinodal(N, N, 1.0, 0.01, 0.9, seed=SEED), p)
    for _ in range(steps):
        f = rk2_step(d, f, p)
    rho, ux, uy, T = oracle.moments(d, f, p.b)
    np.savez_compressed(os.path.join(HERE, f"spinodal256_{steps}.npz"), steps=steps, seed=SEED,
                        moment_rows=MOMENT_ROWS, f_rows=F_ROWS, rho=rho[MOMENT_ROWS], ux=ux[MOMENT_ROWS],
                        uy=uy[MOMENT_ROWS], T=T[MOMENT_ROWS], f=f[:, F_ROWS, :],
                        u_scale=max(float(np.abs(ux).max()), float(np.abs(uy).max())))


if __name__ == "__main__":
    main()
