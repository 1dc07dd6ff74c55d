"""Pins of the oracle's GLL rule and derivative matrix (Section 4.2,
Eq. numerical_integ and Eq. deriv_u): closed forms and polynomial exactness."""
import math
import os

import numpy as np
import pytest

from oracle import gll

GOLD = os.path.join(os.path.dirname(__file__), "golden", "gll_p4.txt")


def test_p4_closed_form():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    val = {"-1": -1.0, "1": 1.0, "0": 0.0,
           "-sqrt(3/7)": -math.sqrt(3 / 7), "sqrt(3/7)": math.sqrt(3 / 7)}
    x_ref = np.array([val[r[0]] for r in rows])
    w_ref = np.array([int(r[1]) / int(r[2]) for r in rows])
    x = gll.gll_nodes(4)
    np.testing.assert_allclose(x, x_ref, rtol=0, atol=1e-15)
    np.testing.assert_allclose(gll.gll_weights(4), w_ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
def test_weights_sum_and_exactness(p):
    x = gll.gll_nodes(p)
    w = gll.gll_weights(p)
    assert abs(w.sum() - 2.0) < 1e-14
    assert np.all(np.diff(x) > 0) and x[0] == -1.0 and x[-1] == 1.0
    # exact for monomials up to degree 2p-1
    for k in range(2 * p):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(w @ x ** k - exact) < 1e-13, (p, k)
    # and not for degree 2p (the rule has only 2p-1 degrees of exactness)
    k = 2 * p
    assert abs(w @ x ** k - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("p", range(1, 9))
def test_derivative_matrix_on_polynomials(p):
    x = gll.gll_nodes(p)
    D = gll.derivative_matrix(x)
    np.testing.assert_allclose(D @ np.ones(p + 1), 0.0, atol=1e-12)
    for k in range(1, p + 1):
        np.testing.assert_allclose(D @ x ** k, k * x ** (k - 1), atol=1e-11)


def test_lagrange_dual_system():
    """Eq. dual_sys: the nodal basis is the identity at its own nodes."""
    x = gll.gll_nodes(5)
    np.testing.assert_allclose(gll.lagrange_values(x, x), np.eye(6), atol=1e-14)
