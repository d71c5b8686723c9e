"""The workload definitions carry the paper's printed constants (tests/golden)."""
import json
import os

import numpy as np

import workloads as W
from tests.independent import wagner_jones

HERE = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def test_paper_constants_in_workloads():
    g = _load("paper_constants.json")
    p = W.glider_params()
    assert np.allclose(p["x_d"], g["x_d"]["value"], rtol=0, atol=1e-15)
    assert np.allclose(p["q"], g["Q"]["value"])
    assert np.allclose(W.GLIDER_X0, g["x_g0"]["value"])
    assert p["shed_offset"] == g["shed_offset_fraction_of_chord"]["value"]
    assert p["dt"] == g["dt"]["value"]


def test_wagner_fit_coefficients():
    g = _load("wagner_jones.json")
    s = np.array([0.0, 1.0, 4.0, 16.0])
    ref = 1 - g["a1"] * np.exp(-g["b1"] * s) - g["a2"] * np.exp(-g["b2"] * s)
    assert np.allclose(wagner_jones(s), ref, rtol=1e-15)
    assert abs(wagner_jones(0.0) - 0.5) < 1e-12
