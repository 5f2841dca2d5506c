"""The stored expected values under tests/golden/ (read by the benchmark, which may not
run the oracle) equal a fresh computation by the oracle, and the stored modes are
what they claim to be: stationary points of f with -Hess f positive definite,
passing the quality gate of Eq. 1."""
import os
import sys

import numpy as np
import pytest

from oracle import objectives as OB
from paper_2606_26164_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_modes as G  # noqa: E402


@pytest.mark.parametrize("name", G.MODE_WORKLOADS)
def test_stored_modes_are_current_and_are_modes(name):
    stored = np.load(G.path("modes_" + name))
    fresh = G.modes_of(name)
    for k in ("x", "f", "neg_hess"):
        np.testing.assert_allclose(stored[k], fresh[k], rtol=1e-10, atol=1e-12)
    obj = I.WORKLOADS[name](n=16).objective
    x = stored["x"]
    g = OB.grad(obj, x)
    assert np.abs(g).max() <= 1e-8 * max(1.0, np.abs(stored["neg_hess"]).max())
    for H in stored["neg_hess"]:
        assert np.linalg.eigvalsh(H).min() > 0
    assert np.all(stored["f"] >= stored["f"].max() + np.log(0.1) - 1e-12)


def test_stored_exact_mixture_values_are_current():
    stored = np.load(G.path("exact_mixture256_d64"))
    fresh = G.exact_mixture256()
    for k in ("rows", "x", "f", "g"):
        np.testing.assert_allclose(stored[k], fresh[k], rtol=1e-12, atol=0)
