"""The oracle against the values the paper prints (tests/golden/paper_values.json)."""
import json
import os
from fractions import Fraction

import numpy as np

from oracle.dvm import D2V16
from oracle.maxwell import coexistence
from oracle.wfft import C_KEFF

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_keff_coefficients_as_printed():
    vals = [float(Fraction(s)) for s in GOLD["keff_coefficients"]["values"]]
    assert np.array_equal(np.array(vals), C_KEFF)


def test_eta_as_printed():
    assert np.array_equal(D2V16(2.5).eta, np.array(GOLD["eta"]["values"], dtype=float))


def test_coexistence_as_printed():
    g = GOLD["coexistence_T095"]
    rl, rv = coexistence(g["T"])
    assert round(rl, g["decimals"]) == g["rho_l"] and round(rv, g["decimals"]) == g["rho_v"]
