"""Pins of the quadrature rules: exactness against the closed-form monomial integrals."""
import math

import numpy as np
import pytest

from oracle import quadrature as Q


def _mons(d):
    return [(a, b, c) for a in range(d + 1) for b in range(d + 1 - a) for c in range(d + 1 - a - b)]


def _exact(a, b, c):
    # a! b! c! / (a+b+c+3)!  written independently of the oracle's helper
    return math.gamma(a + 1) * math.gamma(b + 1) * math.gamma(c + 1) / math.gamma(a + b + c + 4)


@pytest.mark.parametrize("degree,npts", [(1, 1), (2, 4), (4, 14), (5, 14)])
def test_exactness(degree, npts):
    x, w = Q.rule(degree)
    assert len(w) == npts
    assert np.all(w > 0)
    lam0 = 1 - x.sum(axis=1)
    assert np.all(x > 0) and np.all(lam0 > 0)
    for a, b, c in _mons(degree):
        got = np.dot(w, x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c)
        assert abs(got - _exact(a, b, c)) < 1e-15, (a, b, c)


@pytest.mark.parametrize("degree,top", [(1, 1), (2, 2), (5, 5)])
def test_degree_is_not_overstated(degree, top):
    x, w = Q.rule(degree)
    errs = [abs(np.dot(w, x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c) - _exact(a, b, c))
            for a, b, c in _mons(top + 1) if a + b + c == top + 1]
    assert max(errs) > 1e-8


def test_degree2_closed_form():
    x, w = Q.rule(2)
    a = (5 - np.sqrt(5)) / 20
    assert np.allclose(np.sort(np.unique(np.round(x, 14))), np.sort(np.unique(np.round([a, 1 - 3 * a], 14))))
    assert np.allclose(w, 1 / 24)
