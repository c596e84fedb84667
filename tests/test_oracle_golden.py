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


def test_stored_spinodal_state_is_the_generators():
    # the stored 2000-step oracle state: its recorded parameters, and sanity of the sampled
    # fields (the quench's density contrast after 2000 steps, T near 0.9, momentum near zero)
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "spinodal256_2000.npz"))
    assert int(g["steps"]) == 2000 and int(g["seed"]) == 2
    assert list(g["moment_rows"]) == list(range(0, 256, 16)) and list(g["f_rows"]) == list(range(0, 256, 64))
    assert g["f"].shape == (16, 4, 256) and g["rho"].shape == (16, 256)
    assert 0.95 < g["rho"].min() < 0.99 and 1.01 < g["rho"].max() < 1.05
    assert np.allclose(g["f"].sum(axis=0), g["rho"][::4], rtol=1e-12, atol=0)  # f rows 0, 64, 128, 192
    assert abs(g["T"].mean() - 0.9) < 0.01
