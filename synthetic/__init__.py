"""Seeded synthetic initial fields (rho, u_x, u_y, T) for the D2V16 liquid-vapour runs.

This package is shared by the CPU oracle, the tests and the benchmark. It holds no
arithmetic of the kinetic model: it only shapes initial macroscopic fields (a tanh
slab, a tanh droplet, a noisy uniform state) and draws seeded noise. Coexistence
densities are arguments, never computed here.
"""
from .fields import (  # noqa: F401
    splitmix64,
    uniform01,
    uniform_sym,
    slab,
    droplet,
    spinodal,
    quench_temperatures,
)
