"""Pins for the oracle's 1-D quantities against the definitions they come from.

The flux coefficients s_k, the generator q_k, the Toeplitz matrix T, the
stiffness B, the scaling eta and the mass matrix A_n are all re-derived here
from the finite-volume definitions of Sec. 1-2 (Riemann-Liouville derivatives
of the hat functions at the half nodes, cell integrals of the hat functions)
by numerical quadrature, which shares nothing with the closed forms in the
oracle.  A dropped term, wrong sign or transposed index in the oracle fails one
of these.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import tfde_oracle as o


def _frac_int_weighted(x, lo, hi, d, side):
    """integral_lo^hi |x - s|^{d-1} ds by adaptive quadrature; the singular end
    (s = x) gets scipy's algebraic weight."""
    if hi <= lo:
        return 0.0
    if side == "left":   # s < x, weight (x - s)^{d-1}
        if hi >= x:
            return integrate.quad(lambda s: 1.0, lo, x, weight="alg", wvar=(0.0, d - 1.0),
                                  epsabs=1e-15, epsrel=1e-13)[0]
        return integrate.quad(lambda s: (x - s) ** (d - 1.0), lo, hi, epsabs=1e-15, epsrel=1e-13)[0]
    else:                # s > x, weight (s - x)^{d-1}
        if lo <= x:
            return integrate.quad(lambda s: 1.0, x, hi, weight="alg", wvar=(d - 1.0, 0.0),
                                  epsabs=1e-15, epsrel=1e-13)[0]
        return integrate.quad(lambda s: (s - x) ** (d - 1.0), lo, hi, epsabs=1e-15, epsrel=1e-13)[0]


def left_rl_of_hat(p, x, d, h=1.0, a=0.0):
    """(d^{1-d}/dx^{1-d} phi_p)(x) = (1/Gamma(d)) int_a^x (x-s)^{d-1} phi_p'(s) ds
    (Sec. 1 definition; phi_p(a) = 0 lets the derivative move inside)."""
    xp = a + p * h
    up = _frac_int_weighted(x, xp - h, min(xp, x), d, "left")      # phi' = +1/h
    dn = _frac_int_weighted(x, xp, min(xp + h, x), d, "left")      # phi' = -1/h
    return (up - dn) / (h * math.gamma(d))


def right_rl_of_hat(p, x, d, h=1.0, a=0.0):
    """(d^{1-d}/d(-x)^{1-d} phi_p)(x) = -(1/Gamma(d)) int_x^b (s-x)^{d-1} phi_p'(s) ds."""
    xp = a + p * h
    up = _frac_int_weighted(x, max(xp - h, x), xp, d, "right")
    dn = _frac_int_weighted(x, max(xp, x), xp + h, d, "right")
    return -(up - dn) / (h * math.gamma(d))


@pytest.mark.parametrize("d", [0.1, 0.5, 0.9])
def test_s_k_are_rl_derivatives_of_hats(d):
    """Sec. 2: left derivative of phi_p at x_{i+1/2} equals
    s_{i-p+1} / (h^{1-d} Gamma(d+1)); right derivative at x_{i-1/2} equals
    s_{p-i+1} / (h^{1-d} Gamma(d+1))."""
    s = o.s_coefficients(d, 12)
    c = 1.0 / math.gamma(d + 1.0)  # h = 1
    p = 20
    for m in range(0, 12):
        i = p - 1 + m
        got = left_rl_of_hat(p, i + 0.5, d)
        assert got == pytest.approx(c * s[m], rel=2e-9, abs=1e-12)
        i2 = p + 1 - m
        got2 = right_rl_of_hat(p, i2 - 0.5, d)
        assert got2 == pytest.approx(c * s[m], rel=2e-9, abs=1e-12)
    # zero where the support does not reach the evaluation point
    assert abs(left_rl_of_hat(p, p - 1.5, d)) < 1e-14


@pytest.mark.parametrize("d,kp,km", [(0.3, 1.0, 1.0), (0.7, 2.0, 0.5), (0.55, 19.0, 21.0)])
def test_fv_flux_matrix_from_first_principles(d, kp, km):
    """Row i of Eq. (fvm_sol) in 1-D: the flux jump -(dt/2)(1/h)[D phi_p] over the
    dual cell, D = k_+ d^{1-d}_x - k_- d^{1-d}_{-x}, must equal eta B[i, p]."""
    n, dt = 6, 0.1
    h = 1.0 / (n + 1)
    prob = o.Problem(n=(n, n, n), delta=(d, d, d), kp=(kp,) * 3, km=(km,) * 3, dt=dt)
    etaB = prob.eta[0] * prob.B[0]
    for i in range(1, n + 1):
        for p in range(1, n + 1):
            xm, xp = (i - 0.5) * h, (i + 0.5) * h

            def D(x):
                return kp * left_rl_of_hat(p, x, d, h) - km * right_rl_of_hat(p, x, d, h)

            jump = D(xp) - D(xm)
            got = -(dt / 2.0) * jump / h
            assert got == pytest.approx(etaB[i - 1, p - 1], rel=5e-8, abs=1e-9)


def test_mass_matrix_from_cell_integrals():
    """(1/h) int_{x_{i-1/2}}^{x_{i+1/2}} phi_p = A_n[i, p] (Sec. 2, mass display)."""
    n = 7
    h = 1.0 / (n + 1)
    A = o.mass_A(n)

    def hat(p, x):
        return max(0.0, 1.0 - abs(x - p * h) / h)

    for i in range(1, n + 1):
        for p in range(1, n + 1):
            val = integrate.quad(lambda x: hat(p, x), (i - 0.5) * h, (i + 0.5) * h,
                                 points=[(p - 1) * h, p * h, (p + 1) * h], epsabs=1e-15)[0] / h
            assert val == pytest.approx(A[i - 1, p - 1], abs=1e-13)


def test_toeplitz_layout():
    """Eq. (T_ni): diagonal q_1, superdiagonal q_0, subdiagonals q_2..q_n, zero above."""
    n = 9
    q = o.q_coefficients(0.4, n)
    T = o.toeplitz_T(q, n)
    assert np.all(np.diag(T) == q[1])
    assert np.all(np.diag(T, 1) == q[0])
    for m in range(2, n + 1):
        assert np.all(np.diag(T, -(m - 1)) == q[m])
    assert np.all(np.triu(T, 2) == 0.0)
    assert T[n - 1, 0] == q[n]


def test_limits_delta_to_zero_and_one():
    """delta -> 0: q = (-1, 2, -1, 0, ...) (the standard 3-point Laplacian);
    delta -> 1: q = (-1/2, 0, 1/2, 0, ...)."""
    n = 8
    q0 = o.q_coefficients(1e-12, n)
    np.testing.assert_allclose(q0[:3], [-1.0, 2.0, -1.0], atol=1e-10)
    np.testing.assert_allclose(q0[3:], 0.0, atol=1e-10)
    q1 = o.q_coefficients(1.0 - 1e-12, n)
    np.testing.assert_allclose(q1[:3], [-0.5, 0.0, 0.5], atol=1e-10)
    np.testing.assert_allclose(q1[3:], 0.0, atol=1e-10)


@pytest.mark.parametrize("d", [0.05, 0.2, 0.35, 0.5, 0.65, 0.8, 0.95])
def test_coefficient_lemmas(d):
    """Lemma coef_prop1 (i)-(iii) and Lemma coef_prop2, n = 2048; plus the
    telescoping identity sum_{k=0}^{n} q_k = -s_n (so the series sums to 0)."""
    n = 2048
    q = o.q_coefficients(d, n)
    s = o.s_coefficients(d, n)
    assert q[1] > 0
    assert q[0] + q[2] < 0
    assert np.all(q[3:] < 0)
    # (iii): q_1 + sum_{k != 1, k <= m} q_k > 0 for every m >= 2
    partial = q[1] + q[0] + np.cumsum(q[2:])
    assert np.all(partial > 0)
    # coef_prop2: q_0 + q_2 < q_3 < q_4 < ...
    assert q[0] + q[2] < q[3]
    assert np.all(np.diff(q[3:]) > 0)
    # (ii): telescoping
    assert math.fsum(q) == pytest.approx(-s[n], rel=1e-9, abs=1e-15)
    assert abs(s[n]) < 2.0 * n ** (d - 2.0)


@pytest.mark.parametrize("d", [0.15, 0.5, 0.85])
def test_q_k_against_cancellation_free_integral(d):
    """For k >= 3, q_k = -Delta^3 g(k - 5/2) with g(x) = x^d, and
    Delta^3 g(a) = int_0^3 B2(t) g'''(a + t) dt (B2: quadratic B-spline).  The
    integral has no cancellation, so it checks the high-precision difference
    formula (Eq. (coef_expression)) to full FP64 accuracy."""
    q = o.q_coefficients(d, 600)
    g3 = lambda x: d * (d - 1.0) * (d - 2.0) * x ** (d - 3.0)
    pieces = [(0.0, 1.0, lambda t: 0.5 * t * t),
              (1.0, 2.0, lambda t: 0.5 * (-2.0 * t * t + 6.0 * t - 3.0)),
              (2.0, 3.0, lambda t: 0.5 * (3.0 - t) ** 2)]
    xg, wg = np.polynomial.legendre.leggauss(40)   # each piece is analytic for a >= 1/2
    for k in [3, 4, 7, 20, 100, 599, 600]:
        a = k - 2.5
        val = 0.0
        for lo, hi, w in pieces:
            t = 0.5 * (hi - lo) * xg + 0.5 * (hi + lo)
            val += 0.5 * (hi - lo) * math.fsum(wg * w(t) * g3(a + t))
        assert -val == pytest.approx(q[k], rel=2e-13)


def test_eta_scaling():
    """eta = dt / (2 Gamma(d+1) h^{2-d}) for a few hand-computed values."""
    assert o.eta(0.5, 0.25, 0.1) == pytest.approx(0.1 / (2 * math.gamma(1.5) * 0.25 ** 1.5), rel=1e-15)
    # h = 1, dt = 2 -> 1/Gamma(d+1); Gamma(2) = 1
    assert o.eta(1.0, 1.0, 2.0) == pytest.approx(1.0)
