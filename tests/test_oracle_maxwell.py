"""Pins of the oracle's Maxwell construction (Sec. 3.1) against the paper's printed
coexistence densities (Sec. 3.3) and textbook properties of the van der Waals fluid."""
import numpy as np
import pytest

from oracle.maxwell import coexistence
from oracle.model import pressure_vdw


def test_printed_coexistence_at_T095():
    # Sec. 3.3: at T = 0.95 the liquid and vapour densities are 1.462 and 0.579
    rl, rv = coexistence(0.95)
    assert round(rl, 3) == 1.462
    assert round(rv, 3) == 0.579


@pytest.mark.parametrize("T", [0.8, 0.85, 0.9, 0.95, 0.99])
def test_equal_pressure_and_chemical_potential(T):
    # chemical potential of the van der Waals free energy rho T ln(rho/(3 - rho)) - 9 rho^2/8
    mu = lambda r: T * np.log(r / (3 - r)) + 3 * T / (3 - r) - 9 * r / 4
    rl, rv = coexistence(T)
    assert rl > 1.0 > rv > 0.0
    assert pressure_vdw(rl, T) == pytest.approx(pressure_vdw(rv, T), rel=1e-11)
    assert mu(rl) == pytest.approx(mu(rv), rel=1e-10, abs=1e-11)


def test_mean_field_critical_scaling():
    # near T_c the van der Waals coexistence gap is 4 sqrt(1 - T) (mean-field exponent 1/2)
    for eps in (1e-4, 1e-5):
        rl, rv = coexistence(1.0 - eps)
        assert (rl - rv) / (4 * np.sqrt(eps)) == pytest.approx(1.0, abs=5 * np.sqrt(eps))
