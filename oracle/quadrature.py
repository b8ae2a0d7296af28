"""Quadrature rules on the reference tetrahedron {(0,0,0),(1,0,0),(0,1,0),(0,0,1)} (volume 1/6).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper takes Xiao-Gimbutas rules (Sections 3, 6.3 and 7.4: 11 points for
degree 4, 4 points for degree 2); their nodes are not printed.  Reading used
here: rules of the stated degree derived from the moment equations.
  * degree 1: the centroid rule.
  * degree 2: the symmetric 4-point rule, barycentric (b,a,a,a) and its
    permutations, a = (5 - sqrt 5)/20, b = 1 - 3a, weights 1/24 (closed form).
  * degree 4 (and 5): a fully symmetric 14-point rule, exact to degree 5, with
    orbits (a1,a1,a1,1-3a1) x4, (a2,a2,a2,1-3a2) x4 and (b,b,1/2-b,1/2-b) x6;
    its six parameters solve the moment equations by Gauss-Newton here.
Pinned by: exactness on every monomial x^a y^b z^c with a+b+c <= degree
against the closed form a! b! c! / (a+b+c+3)!, positivity of the weights,
points inside the tetrahedron (tests/test_oracle_quadrature.py).
"""
from __future__ import annotations

import functools
import itertools
import math

import numpy as np


def monomial_integral(a: int, b: int, c: int) -> float:
    """Exact integral of x^a y^b z^c over the reference tetrahedron."""
    return math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)


def _orbit_s31(a: float) -> np.ndarray:
    bary = []
    for pos in range(4):
        lam = [a] * 4
        lam[pos] = 1.0 - 3.0 * a
        bary.append(lam)
    return np.array(bary)[:, 1:]


def _orbit_s22(b: float) -> np.ndarray:
    c = 0.5 - b
    bary = set()
    for perm in itertools.permutations([b, b, c, c]):
        bary.add(perm)
    return np.array(sorted(bary))[:, 1:]


def _rule14(theta):
    a1, w1, a2, w2, b, w3 = theta
    pts = np.concatenate([_orbit_s31(a1), _orbit_s31(a2), _orbit_s22(b)], axis=0)
    w = np.concatenate([np.full(4, w1), np.full(4, w2), np.full(6, w3)])
    return pts, w


def _monomials(deg: int):
    return [(a, b, c) for a in range(deg + 1) for b in range(deg + 1 - a) for c in range(deg + 1 - a - b)]


def _residual(theta, mons):
    pts, w = _rule14(theta)
    return np.array([np.dot(w, pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c) - monomial_integral(a, b, c)
                     for a, b, c in mons])


@functools.lru_cache(maxsize=None)
def _solve_rule14():
    mons = _monomials(5)
    theta = np.array([0.1, 1.0 / 84, 0.3, 1.0 / 84, 0.45, 1.0 / 84])
    for _ in range(100):
        r = _residual(theta, mons)
        jac = np.empty((len(mons), 6))
        for p in range(6):
            h = 1e-7
            tp = theta.copy(); tp[p] += h
            tm = theta.copy(); tm[p] -= h
            jac[:, p] = (_residual(tp, mons) - _residual(tm, mons)) / (2 * h)
        step = np.linalg.lstsq(jac, -r, rcond=None)[0]
        theta = theta + step
        if np.max(np.abs(step)) < 1e-17:
            break
    return tuple(theta)


def rule(degree: int):
    """(points (nq,3), weights (nq,)) of the rule of the given degree (1, 2, 4 or 5)."""
    if degree <= 1:
        return np.array([[0.25, 0.25, 0.25]]), np.array([1.0 / 6.0])
    if degree == 2:
        a = (5.0 - math.sqrt(5.0)) / 20.0
        return _orbit_s31(a), np.full(4, 1.0 / 24.0)
    if degree in (3, 4, 5):
        return _rule14(np.array(_solve_rule14()))
    raise ValueError("unsupported quadrature degree %d" % degree)
