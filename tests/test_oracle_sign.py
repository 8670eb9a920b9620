"""Pins for the sign/step approximation (Section 5.4.2; Table 2 defines the
margin 2^-alpha and precision beta vocabulary): the default stage polynomial
is derived here from its closed form, and the composite margin found by the
oracle's grid search is checked against bisection on the monotone map."""
import math

import numpy as np
import pytest

from oracle import query


def test_f3_closed_form():
    # f3(x) = sum_{i=0}^{3} C(2i,i)/4^i * x (1 - x^2)^i, expanded with numpy polynomials
    x = np.polynomial.Polynomial([0, 1])
    f = sum(math.comb(2 * i, i) / 4 ** i * x * (1 - x ** 2) ** i for i in range(4))
    c = f.coef
    assert np.allclose(c[[1, 3, 5, 7]], query.F3) and np.allclose(c[[0, 2, 4, 6]], 0)


def test_f3_properties():
    xs = np.linspace(-1, 1, 2001)
    v = query.odd_poly(query.F3, xs)
    assert abs(query.odd_poly(query.F3, 1.0) - 1.0) < 1e-15
    assert np.allclose(v, -v[::-1])
    # derivative is 35/16 (1 - x^2)^3 >= 0: monotone on [-1, 1], maps [-1,1] into itself
    h = 1e-6
    d = (query.odd_poly(query.F3, xs[1:-1] + h) - query.odd_poly(query.F3, xs[1:-1] - h)) / (2 * h)
    assert np.allclose(d, 35 / 16 * (1 - xs[1:-1] ** 2) ** 3, atol=1e-6)
    assert np.all(np.abs(v) <= 1 + 1e-15)


def bisect_margin(stages, tol):
    lo, hi = 0.0, 1.0          # composite is increasing on [0,1]; find composite(x) = 1 - tol
    for _ in range(200):
        mid = (lo + hi) / 2
        if 1.0 - query.composite_sign(stages, mid) > tol:
            lo = mid
        else:
            hi = mid
    return hi


@pytest.mark.parametrize("nst,tol", [(1, 0.5), (3, 0.5), (1, 2.0 ** -12), (3, 2.0 ** -12), (5, 2.0 ** -12)])
def test_margin_grid_equals_bisection(nst, tol):
    st = [query.F3] * nst
    g = query.sign_margin(st, tol)
    b = bisect_margin(st, tol)
    assert abs(g - b) <= 2.0 / (1 << 20)
    # every point beyond the margin is within tol of sign; a point just inside is not
    xs = np.linspace(g, 1, 10001)
    assert np.all(np.abs(query.composite_sign(st, xs) - 1) <= tol)
    assert abs(query.composite_sign(st, g * 0.99) - 1) > tol


def test_step_affine():
    z = np.array([-0.9, -0.3, 0.3, 0.9])
    u = (query.composite_sign([query.F3] * 5, z) + 1) / 2
    assert np.all(np.abs(u - (z > 0)) < 2.0 ** -8)
