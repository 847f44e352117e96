"""The convergence study on the GPU (Sec. 4.1-4.2, Table 1) through the C ABI
against the oracle's study on the same graph, meshes and noise: the error of
every mesh level agrees, and so the rates; the rates sit at the theory."""
import numpy as np
import pytest

import grf_inputs as gi
from oracle import convergence as cv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
grf = pytest.importorskip("paper_2605_02670_gb300")
from paper_2605_02670_gb300 import convergence as gc  # noqa: E402


def _graph():
    g = gi.Graph(4, np.array([0, 1, 2, 2]), np.array([1, 2, 0, 3]),
                 np.array([1.0, 1.0, 1.0, 0.5]))
    return g, np.array([2, 2, 2, 1])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("beta", [0.375, 0.75])
def test_strong_errors_match_oracle(precision, beta):
    g, base = _graph()
    args = (g, base, [2, 3, 4, 5], 9, beta, 1.0, 100, 7)
    hs, eg = gc.strong_errors(*args, precision=precision)
    ho, eo = cv.strong_errors(*args)
    np.testing.assert_allclose(hs, ho)
    # errors are differences of fields; the fields match to 1e-4 (mixed) / 1e-6
    np.testing.assert_allclose(eg, eo, rtol=1e-3 if precision == "mixed" else 1e-5)
    assert abs(gc.rate(hs, eg) - (2 * beta - 0.5)) < 0.06


def test_covariance_errors_match_oracle():
    g, base = _graph()
    args = (g, base, [1, 2, 3, 4], 7, 0.5, 1.0)
    hs, eg = gc.covariance_errors(*args, precision="fp64")
    _, eo = cv.covariance_errors(*args)
    np.testing.assert_allclose(eg, eo, rtol=1e-5)
    assert abs(gc.rate(hs, eg) - 1.5) < 0.1
