"""Pins of the oracle's regularized Stokes kernels (Sec. 7) and direct sum:
hand-computed values, eps -> 0 limits to the Stokes kernels, and calculus
identities of the MRS functions (divergence-free Stokeslet velocity; angular
velocity = half the curl of the velocity).  CPU only."""
import math

import numpy as np
import pytest

ST, RO, SR, POLY = 0, 1, 2, 99
C = 1.0 / (8.0 * math.pi)


@pytest.mark.parametrize("eps", [0.5, 0.01, 1e-3])
def test_mrs_functions_at_zero(orc, eps):
    # Eq. MRS_kernels at r = 0 by hand: H1 = 1/(4 pi eps), H2 = 1/(8 pi eps^3),
    # Q = 5/(8 pi eps^3), D1 = 10/(8 pi eps^3), D2 = 21/(8 pi eps^5).
    H = orc.mrs_functions(0.0, eps)
    ref = [1 / (4 * math.pi * eps), C / eps**3, 5 * C / eps**3, 10 * C / eps**3,
           21 * C / eps**5]
    np.testing.assert_allclose(H, ref, rtol=1e-14)


def test_mrs_functions_stokes_limit(orc):
    # eps = 0 at r = 2: H1 = 1/(8 pi r), H2 = 1/(8 pi r^3), Q = 2/(8 pi r^3),
    # D1 = -2/(8 pi r^3), D2 = 6/(8 pi r^5).
    r = 2.0
    H = orc.mrs_functions(r * r, 0.0)
    ref = [C / r, C / r**3, 2 * C / r**3, -2 * C / r**3, 6 * C / r**5]
    np.testing.assert_allclose(H, ref, rtol=1e-14)


def test_mrs_function_values_hand_computed(orc):
    # r = 1, eps = 1: rho^2 = 2.  H1 = 3/(8 pi 2^1.5), H2 = 1/(8 pi 2^1.5),
    # Q = 7/(8 pi 2^2.5), D1 = 1/(8 pi 2^3.5), D2 = 27/(8 pi 2^3.5).
    H = orc.mrs_functions(1.0, 1.0)
    ref = [3 * C / 2**1.5, C / 2**1.5, 7 * C / 2**2.5, 1 * C / 2**3.5, 27 * C / 2**3.5]
    np.testing.assert_allclose(H, ref, rtol=1e-14)


def _rand_pair(seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(3), g.standard_normal(3), g.standard_normal(6)


@pytest.mark.parametrize("seed", range(4))
def test_stokeslet_limit(orc, seed):
    # eps -> 0: u = (f + (f.dhat) dhat) / (8 pi r), the Stokeslet.
    x, y, f = _rand_pair(seed)
    d = x - y
    r = np.linalg.norm(d)
    ref = C * (f[:3] / r + (f[:3] @ d) * d / r**3)
    u = orc.kernel_apply(ST, 1e-9, x, y, f[:3])
    np.testing.assert_allclose(u, ref, rtol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_rotlet_limit(orc, seed):
    # eps -> 0: u = n x d / (8 pi r^3) (rotlet) and
    # w = (-n / r^3 + 3 (n.d) d / r^5) / (16 pi), half the curl of that rotlet.
    x, y, f = _rand_pair(seed)
    n = f[:3]
    d = x - y
    r = np.linalg.norm(d)
    u = orc.kernel_apply(RO, 1e-9, x, y, n)
    np.testing.assert_allclose(u[:3], C * np.cross(n, d) / r**3, rtol=1e-12)
    np.testing.assert_allclose(u[3:], (-n / r**3 + 3 * (n @ d) * d / r**5) / (16 * math.pi),
                               rtol=1e-11)


@pytest.mark.parametrize("seed", range(3))
def test_stokeslet_rotlet_is_sum_of_parts(orc, seed):
    # Eq. MRS_2 = Stokeslet + rotlet terms + (1/2)(f x d) Q in w
    x, y, f = _rand_pair(seed)
    eps = 0.3
    d = x - y
    H = orc.mrs_functions(d @ d, eps)
    u_sr = orc.kernel_apply(SR, eps, x, y, f)
    u_s = orc.kernel_apply(ST, eps, x, y, f[:3])
    u_r = orc.kernel_apply(RO, eps, x, y, f[3:])
    np.testing.assert_allclose(u_sr[:3], u_s + u_r[:3], rtol=1e-14)
    np.testing.assert_allclose(u_sr[3:], u_r[3:] + 0.5 * np.cross(f[:3], d) * H[2],
                               rtol=1e-13, atol=1e-15)


def _velocity(orc, kernel, eps, x, y, f):
    return orc.kernel_apply(kernel, eps, x, y, f)[:3]


def _fd_jacobian(orc, kernel, eps, x, y, f, h=1e-5):
    J = np.empty((3, 3))  # J[a, b] = d u_a / d x_b
    for b in range(3):
        e = np.zeros(3)
        e[b] = h
        J[:, b] = (_velocity(orc, kernel, eps, x + e, y, f)
                   - _velocity(orc, kernel, eps, x - e, y, f)) / (2 * h)
    return J


@pytest.mark.parametrize("eps", [0.05, 0.3, 1.0])
def test_regularized_stokeslet_is_divergence_free(orc, eps):
    # div u = 0 for Eq. Velocity_1 at any eps (H1'/r + 4 H2 + r H2' = 0).
    x, y, f = _rand_pair(11)
    J = _fd_jacobian(orc, ST, eps, x * 0.4, y * 0.4, f[:3])
    scale = np.abs(J).max()
    assert abs(np.trace(J)) < 1e-8 * scale


@pytest.mark.parametrize("eps", [0.05, 0.3, 1.0])
def test_angular_velocity_is_half_curl(orc, eps):
    # Eq. AngularVelocity equals (1/2) curl of Eq. Velocity_2 for finite eps;
    # this pins Q, D1, D2 and the reading 1/4 [n.d] d D2 of the garbled term.
    x, y, f = _rand_pair(12)
    x, y = 0.4 * x, 0.4 * y
    J = _fd_jacobian(orc, SR, eps, x, y, f)
    curl = np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])
    w = orc.kernel_apply(SR, eps, x, y, f)[3:]
    np.testing.assert_allclose(w, 0.5 * curl, rtol=1e-7, atol=1e-9 * np.abs(w).max())


def test_stokeslet_reciprocity(orc):
    # the Stokeslet tensor is symmetric: f_a . u(x_a; f_b at x_b) = f_b . u(x_b; f_a at x_a)
    g = np.random.default_rng(3)
    xa, xb, fa, fb = g.standard_normal((4, 3))
    lhs = fa @ orc.kernel_apply(ST, 0.2, xa, xb, fb)
    rhs = fb @ orc.kernel_apply(ST, 0.2, xb, xa, fa)
    assert abs(lhs - rhs) < 1e-14 * abs(lhs)


def test_test_poly_kernel_value(orc):
    # prod_l (1 + x_l y_l / 2)^3 times f
    x = np.array([1.0, -2.0, 0.5])
    y = np.array([0.5, 0.25, 2.0])
    f = np.array([1.0, 2.0, -1.0])
    p = (1 + 0.25) ** 3 * (1 - 0.25) ** 3 * (1 + 0.5) ** 3
    np.testing.assert_allclose(orc.kernel_apply(POLY, 0.0, x, y, f), p * f, rtol=1e-15)


@pytest.mark.parametrize("kernel", [ST, RO, SR])
def test_direct_sum_is_sum_of_pairs_and_keeps_self_term(orc, kernel):
    g = np.random.default_rng(7)
    x = g.uniform(-1, 1, (5, 3))
    w = g.uniform(-1, 1, (5, orc.kernel_win(kernel)))
    eps = 0.1
    out = orc.direct(kernel, eps, x, x, w)
    for i in range(5):
        ref = sum(orc.kernel_apply(kernel, eps, x[i], x[j], w[j]) for j in range(5))
        np.testing.assert_allclose(out[i], ref, rtol=1e-14, atol=1e-14)
    # self term: a lone particle moves with f H1(0) = f / (4 pi eps)
    if kernel == ST:
        lone = orc.direct(ST, eps, x[:1], x[:1], w[:1])
        np.testing.assert_allclose(lone[0], w[0] / (4 * math.pi * eps), rtol=1e-14)


def test_rel_l2_definition(orc):
    ud = np.array([[3.0, 4.0, 0.0], [0.0, 0.0, 0.0]])
    ut = np.array([[3.0, 4.0, 1.0], [0.0, 0.0, 0.0]])
    assert abs(orc.rel_l2(ud, ut) - 1.0 / 5.0) < 1e-16
