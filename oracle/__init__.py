"""Plain FP64 CPU oracle of the D2V16-FFT-TLB liquid-vapour kinetic model (Gan, Xu et al.).

TEST INFRASTRUCTURE ONLY. This package is the correctness authority for the CUDA
library: only the tests, the smoke check and the benchmark's CPU-baseline /
reference arm may import or run it. The product library never calls it, and it
shares no code, table or constant with the CUDA path.

The oracle follows the paper's sections in order, written for readability, in
float64 numpy over whole fields:
  dvm.py      Sec. 2.1: the 16 discrete velocities, moments, the equilibrium f_eq
  wfft.py     Sec. 2.3, Eq. (3): 16th-order modified wavenumber, spectral derivatives
  model.py    Sec. 2.2, Eqs. (1)-(2): van der Waals EOS, stress Lambda, the forcing
              term I_i; Sec. 2.3: the two-stage Runge-Kutta step
  maxwell.py  Sec. 3.1: Maxwell construction for the van der Waals coexistence curve
  diag.py     Sec. 2.2 / 3.2: total mass, momentum, total energy e_T, max |u|, and the
              circularly averaged structure factor of the density

Readings of silent or garbled passages are listed where they are used.
Parity status: every function here is pinned by `tests/test_oracle_*.py` except the
full nonlinear trajectory of a phase-separating run, which the paper shows only as
figures ("parity unpinned" against the paper; its pins are conservation, fixed points,
closed-form decay rates and the Maxwell coexistence densities).
"""
from .dvm import D2V16, moment_matrix, equilibrium_moments, feq, moments  # noqa: F401
from .wfft import keff, deriv_multiplier, spectral_deriv, dft_deriv_matrix  # noqa: F401
from .model import Params, forcing_terms, rhs, rk2_step, run, pressure_vdw  # noqa: F401
from .maxwell import coexistence  # noqa: F401
from .diag import diagnostics  # noqa: F401
