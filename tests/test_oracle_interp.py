"""Pins of the oracle's interpolation layer (Sec. 3) against closed forms and
independent definitions.  CPU only."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def test_chebyshev_points_closed_form(orc):
    # Eq. Chebyshev_points on [-1, 1]: cos(k pi / n); n = 4 written out by hand.
    s = orc.cheb_points(4)
    h = math.sqrt(0.5)
    np.testing.assert_allclose(s, [1.0, h, 0.0, -h, -1.0], rtol=0, atol=3e-16)
    # n = 1: the two ends only; n = 2: ends and centre.
    np.testing.assert_allclose(orc.cheb_points(1), [1.0, -1.0], atol=0)
    np.testing.assert_allclose(orc.cheb_points(2), [1.0, 0.0, -1.0], atol=3e-16)


def test_chebyshev_points_interval_map(orc):
    # Sec. 3: t -> (a + b + t (b - a)) / 2 sends 1 -> b, -1 -> a and keeps order.
    for n in (1, 3, 8, 13):
        s = orc.cheb_points(n, 2.0, 5.0)
        assert s[0] == 5.0 and s[-1] == 2.0
        assert np.all(np.diff(s) < 0)
        ref = orc.cheb_points(n)
        np.testing.assert_allclose(s, 3.5 + 1.5 * ref, rtol=0, atol=1e-15)


def _brute_weights(s):
    # definition in Eq. Barycentric-1D: w_k = 1 / prod_{j != k} (s_k - s_j)
    n1 = len(s)
    return np.array([1.0 / np.prod([s[k] - s[j] for j in range(n1) if j != k])
                     for k in range(n1)])


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 8, 12, 16])
def test_simple_weights_match_definition_up_to_common_factor(orc, n):
    # Eq. barycentric_weights vs the definition: equal up to one common
    # factor (scale invariance, Sec. 3), on [-1, 1] and on a mapped interval.
    ws = orc.bary_weights(n)
    assert ws[0] == 0.5 and abs(ws[-1]) == 0.5
    assert np.all(np.abs(ws[1:-1]) == 1.0)
    for a, b in ((-1.0, 1.0), (0.3, 0.31), (-40.0, 7.0)):
        wb = _brute_weights(orc.cheb_points(n, a, b))
        ratio = wb / ws
        np.testing.assert_allclose(ratio, ratio[0], rtol=1e-11)


def _lagrange_product(s, t):
    # Eq. Lagrange_polynomial, written as the plain product form
    n1 = len(s)
    return np.array([np.prod([(t - s[j]) / (s[k] - s[j]) for j in range(n1) if j != k])
                     for k in range(n1)])


@pytest.mark.parametrize("n", [1, 2, 5, 8, 11])
def test_barycentric_equals_product_form(orc, n):
    rng = np.random.default_rng(5)
    a, b = -0.7, 1.9
    s = orc.cheb_points(n, a, b)
    w = orc.bary_weights(n)
    for t in rng.uniform(a, b, 25):
        L = orc.bary_basis(s, w, t)
        np.testing.assert_allclose(L, _lagrange_product(s, t), rtol=0, atol=2e-13)
        assert abs(L.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("n", [1, 4, 9])
def test_coincident_point_rule(orc, n):
    # L_k(s_j) = delta_jk through the flag branch (Sec. 3, Algorithm 1).
    s = orc.cheb_points(n, -3.0, 2.0)
    w = orc.bary_weights(n)
    for j in range(n + 1):
        L = orc.bary_basis(s, w, s[j])
        e = np.zeros(n + 1)
        e[j] = 1.0
        assert np.array_equal(L, e)
    # just outside the tolerance the ordinary branch runs and stays finite
    t = s[1] + 1e-300
    L = orc.bary_basis(s, w, t)
    assert np.all(np.isfinite(L))


def test_degenerate_interval_all_points_coincide(orc):
    # zero-width box: every s_k equals a; the last flagged k carries the weight
    s = orc.cheb_points(4, 0.25, 0.25)
    L = orc.bary_basis(s, orc.bary_weights(4), 0.25)
    assert L.sum() == 1.0 and L[-1] == 1.0


@pytest.mark.parametrize("n", [2, 6, 10])
def test_interpolation_reproduces_polynomials(orc, n):
    # Sec. 2: the interpolant of a polynomial of degree <= n is exact.
    rng = np.random.default_rng(n)
    s = orc.cheb_points(n, -0.4, 1.3)
    w = orc.bary_weights(n)
    coef = rng.standard_normal(n + 1)
    p = np.polynomial.polynomial.Polynomial(coef)
    for t in rng.uniform(-0.4, 1.3, 10):
        L = orc.bary_basis(s, w, t)
        assert abs(L @ p(s) - p(t)) < 1e-12 * max(1.0, abs(p(t)))
    # and it is not exact for degree n + 1 (the test above is sensitive)
    q = np.polynomial.polynomial.Polynomial(np.r_[np.zeros(n + 1), 1.0])
    t = 0.123
    L = orc.bary_basis(s, w, t)
    assert abs(L @ q(s) - q(t)) > 1e-8
