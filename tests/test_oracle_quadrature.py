"""Pins of the oracle's closed-form inner integrals against textbook values,
brute-force adaptive quadrature and the Poisson equation."""
import numpy as np
import pytest
from scipy import integrate

from oracle import quadrature as Q

LO = np.zeros(3)
HI = np.ones(3)


def test_cube_centre_textbook_value():
    # potential at the centre of a unit cube: 3 ln((sqrt3+1)/(sqrt3-1)) - pi/2
    exact = 3.0 * np.log((np.sqrt(3) + 1) / (np.sqrt(3) - 1)) - np.pi / 2
    assert abs(Q.box_potential(np.full(3, 0.5), LO, HI) - exact) < 1e-13


def test_cube_corner_from_centre_by_scaling():
    # Phi_[0,1]^3(0) = Phi_[-1,1]^3(0) / 8 = 4 Phi_[-1/2,1/2]^3(0) / 8
    centre = Q.box_potential(np.full(3, 0.5), LO, HI)
    for corner in ([0, 0, 0], [1, 1, 1], [1, 0, 1]):
        assert abs(Q.box_potential(np.array(corner, float), LO, HI) - centre / 2) < 1e-13


def test_square_centre_textbook_value():
    exact = 4.0 * np.log(1.0 + np.sqrt(2.0))
    assert abs(Q.rect_potential(np.array([0.5, 0.5, 0.0]), 2, 0.0, LO, HI) - exact) < 1e-13


@pytest.mark.parametrize("p", [[2.3, -0.7, 1.9], [1.3, 0.5, 0.5], [-0.2, 1.1, 0.4]])
def test_exterior_points_against_high_order_gauss(p):
    p = np.array(p)
    P, W = Q.box_gauss_points(LO, HI, 40)
    R = np.linalg.norm(P - p, axis=1)
    tol = 1e-10 if np.min(R) > 0.5 else 1e-5
    assert abs(Q.box_potential(p, LO, HI) - np.sum(W / R)) < tol * np.sum(W / R)
    for d in range(3):
        ref = np.sum(W * P[:, d] / R)
        assert abs(Q.box_linear_potential(p, LO, HI, d) - ref) < tol * abs(ref)
    for axis in range(3):
        P2, W2 = Q.rect_gauss_points(axis, 0.3, LO, HI, 40)
        R2 = np.linalg.norm(P2 - p, axis=1)
        ref = np.sum(W2 / R2)
        assert abs(Q.rect_potential(p, axis, 0.3, LO, HI) - ref) < 1e-4 * ref
        ref = np.sum(W2 * R2)
        assert abs(Q.rect_R_integral(p, axis, 0.3, LO, HI) - ref) < 1e-8 * ref


def _interior_brute(p, weight=None):
    """int_box w(r')/|r'-p| by splitting the box at p into 8 sub-boxes; in each,
    the z integral of 1/R is the textbook asinh and x, y use adaptive QUADPACK."""
    total = 0.0
    for x0, x1 in ((0.0, p[0]), (p[0], 1.0)):
        for y0, y1 in ((0.0, p[1]), (p[1], 1.0)):
            def f(y, x):
                rho = np.hypot(x - p[0], y - p[1])
                if weight is None:
                    return np.arcsinh((1.0 - p[2]) / rho) + np.arcsinh(p[2] / rho)
                return weight(x) * (np.arcsinh((1.0 - p[2]) / rho) + np.arcsinh(p[2] / rho))
            v, _ = integrate.dblquad(f, x0, x1, y0, y1, epsabs=1e-11, epsrel=1e-11)
            total += v
    return total


@pytest.mark.parametrize("p", [[0.31, 0.62, 0.47], [0.9, 0.15, 0.55]])
def test_interior_points_against_adaptive_quadrature(p):
    p = np.array(p)
    assert abs(Q.box_potential(p, LO, HI) - _interior_brute(p)) < 1e-8
    ref = _interior_brute(p, weight=lambda x: x)
    assert abs(Q.box_linear_potential(p, LO, HI, 0) - ref) < 1e-8


def test_poisson_equation():
    # Laplacian of the box potential is -4 pi inside and 0 outside
    e = 1e-3
    for p, lap in (([0.4, 0.55, 0.3], -4 * np.pi), ([1.6, 0.5, -0.4], 0.0)):
        p = np.array(p)
        acc = -6 * Q.box_potential(p, LO, HI)
        for d in range(3):
            dp = np.zeros(3)
            dp[d] = e
            acc += Q.box_potential(p + dp, LO, HI) + Q.box_potential(p - dp, LO, HI)
        assert abs(acc / e ** 2 - lap) < 1e-3


def test_in_plane_rectangle_against_adaptive_quadrature():
    p = np.array([0.3, 0.8, 0.0])
    ref = 0.0
    for x0, x1 in ((0.0, 0.3), (0.3, 1.0)):
        # inner y integral of 1/sqrt(u^2+v^2) in closed form (asinh), outer adaptive
        f = lambda x: np.arcsinh((1.0 - 0.8) / abs(x - 0.3)) + np.arcsinh(0.8 / abs(x - 0.3))
        ref += integrate.quad(f, x0, x1, epsabs=1e-12, limit=200)[0]
    assert abs(Q.rect_potential(p, 2, 0.0, LO, HI) - ref) < 1e-9
    refR, _ = integrate.dblquad(lambda y, x: np.hypot(x - 0.3, y - 0.8), 0, 1, 0, 1, epsabs=1e-12)
    assert abs(Q.rect_R_integral(p, 2, 0.0, LO, HI) - refR) < 1e-9


def test_broadcasting_over_elements():
    pts = np.random.default_rng(0).uniform(-1, 2, (5, 7, 3))
    lo = np.random.default_rng(1).uniform(-1, 0, (5, 1, 3))
    hi = lo + 0.7
    v = Q.box_potential(pts, lo, hi)
    for i in range(5):
        for j in range(7):
            assert abs(v[i, j] - Q.box_potential(pts[i, j], lo[i, 0], hi[i, 0])) < 1e-12
