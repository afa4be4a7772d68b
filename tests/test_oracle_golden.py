"""Pins of the oracle against values the paper prints (tests/golden/)."""
import json
import os

import numpy as np

import oracle
from oracle.solver import TRParams
from oracle.spring1d import Spring1D

HERE = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def test_table2_shear_moduli_match_lame():
    """Table 2 prints E, mu and nu for each phase; the oracle's mu = E/(2(1+nu))
    must reproduce the printed mu to the printed digit."""
    g = _load("table2_material_properties.json")
    for row in g["rows"]:
        _, mu = oracle.lame(row["E"], row["nu"])
        assert abs(mu - row["mu"]) <= g["printed_digits_mu"], row["name"]


def test_spring_eigenvalues_printed_form():
    g = _load("spring_example_sec31.json")
    for a in g["alphas"]:
        s = Spring1D(k=g["k"], gamma0=g["gamma0"], alpha=a)
        K = s.nodal_stiffness(np.array([g["xbar"]] * 3))  # damage spring post-peak
        w = np.sort(np.linalg.eigvalsh(K))
        np.testing.assert_allclose(w, np.sort([0.0, 3 * g["k"], (2 * a + 1) * g["k"]]), atol=1e-12)
        assert (w.min() < -1e-12) == (a < -0.5)


def test_solver_constants_are_the_printed_ones():
    g = _load("spring_example_sec31.json")
    assert TRParams().restart_thr == g["restart_threshold"]["value"]
