"""Pins for the oracle's Krylov solvers and CN time loop: dense LU brute force,
the iteration counts printed in Tables 3 and 4 of the paper, the
manufactured-solution source term against a quadrature of its definition, and
the convergence orders stated in the Sec. 2 remark."""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import tfde_oracle as o
import tfde_inputs as inp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_iteration_counts.json")


@pytest.mark.parametrize("sym", [True, False])
def test_krylov_solution_matches_dense_lu(sym):
    p = o.Problem(n=(5, 6, 7), delta=(0.3, 0.6, 0.8), kp=(1.0, 1.5, 2.0),
                  km=(1.0, 1.5, 2.0) if sym else (0.5, 1.0, 0.6), dt=0.2)
    b = inp.uniform_vector(p.shape, 11)
    x_ref = np.linalg.solve(o.dense_A(p), b.ravel()).reshape(p.shape)
    tau = o.build_tau(p)
    A = lambda v: o.apply_A(p, v)
    Pi = lambda r: o.apply_Pinv(tau, r)
    if sym:
        x, info = o.pcg(A, Pi, b, np.zeros_like(b), 1e-14, 500)
    else:
        x, info = o.gmres_left(A, Pi, b, np.zeros_like(b), 1e-14, 500, 20, "true")
    assert info.converged
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-12
    # restarted GMRES with a short restart converges to the same solution
    x2, info2 = o.gmres_left(A, Pi, b, np.zeros_like(b), 1e-13, 500, 3, "true")
    assert info2.restarts > 1 and np.linalg.norm(x2 - x_ref) / np.linalg.norm(x_ref) < 1e-11


def test_delta_to_zero_tau_is_exact():
    """delta -> 0 makes every T tridiagonal Toeplitz, already in the tau algebra,
    so P = A and PCG converges in one iteration."""
    p = o.Problem(n=(6, 6, 6), delta=(1e-13,) * 3, kp=(1.0,) * 3, km=(1.0,) * 3, dt=0.1)
    b = inp.uniform_vector(p.shape, 12)
    tau = o.build_tau(p)
    x, info = o.pcg(lambda v: o.apply_A(p, v), lambda r: o.apply_Pinv(tau, r), b,
                    np.zeros_like(b), 1e-10, 50)
    assert info.iters == 1


def _example2(deltas, np1, kp, km):
    n = np1 - 1
    M = np1 // 2
    return o.Problem(n=(n, n, n), delta=deltas, kp=kp, km=km, dt=1.0 / M), M


@pytest.mark.parametrize("key", ["0.1,0.2,0.3", "0.4,0.5,0.6", "0.7,0.8,0.9", "0.1,0.5,0.9"])
def test_table3_table4_iteration_counts(key):
    """Example 2 with the settings of Sec. 4 (tol 1e-9, zero initial guess,
    restart 20, M = (n+1)/2): PCG(tau), CG and PGMRES(tau) average iteration
    counts of Tables 3 and 4 for n+1 = 8, 16, 32."""
    g = json.load(open(GOLDEN))
    deltas = tuple(float(v) for v in key.split(","))
    for idx, np1 in enumerate(g["n_plus_1"]):
        p, M = _example2(deltas, np1, (5.0,) * 3, (5.0,) * 3)
        r = o.cn_solve(p, o.exact_u(p, 0.0, "sin"), M, tol=1e-9, phi="sin", x0="zero")
        assert np.mean(r.iters) == g["table3_pcg_tau"][key][idx]
        # unpreconditioned CG column (identity preconditioner)
        u, its = o.exact_u(p, 0.0, "sin"), []
        for m in range(1, M + 1):
            b = o.rhs(p, u, o.source_cell_average(p, (m - 0.5) * p.dt, "sin"))
            u, info = o.pcg(lambda v: o.apply_A(p, v), lambda r_: r_, b, np.zeros_like(b), 1e-9, 10 ** 6)
            its.append(info.iters)
        assert abs(np.mean(its) - g["table3_cg"][key][idx]) <= 0.5
        pn, M = _example2(deltas, np1, (19.0, 21.0, 23.0), (21.0, 23.0, 25.0))
        r = o.cn_solve(pn, o.exact_u(pn, 0.0, "sin"), M, tol=1e-9, phi="sin", x0="zero",
                       criterion="preconditioned")
        assert np.mean(r.iters) == g["table4_pgmres_tau"][key][idx]


@pytest.mark.parametrize("d,kp,km", [(0.3, 1.0, 1.0), (0.75, 2.0, 0.5), (0.5, 19.0, 21.0)])
def test_source_series_is_the_conservative_operator(d, kp, km):
    """S_d(x) = d/dx [k_+ D^{1-d}_x P - k_- D^{1-d}_{-x} P](x), evaluated by
    quadrature from the Riemann-Liouville definitions (Sec. 1):
    (1/Gamma(d)) [k_+ int_0^x (x-s)^{d-1} P''(s) ds + k_- int_x^1 (s-x)^{d-1} P''(s) ds]."""
    P2 = lambda s: 2.0 - 12.0 * s + 12.0 * s * s
    for x in [0.03, 0.2, 0.5, 0.77, 0.99]:
        left = integrate.quad(P2, 0.0, x, weight="alg", wvar=(0.0, d - 1.0))[0]
        right = integrate.quad(P2, x, 1.0, weight="alg", wvar=(d - 1.0, 0.0))[0]
        ref = (kp * left + km * right) / math.gamma(d)
        assert o.S_series(x, d, kp, km) == pytest.approx(ref, rel=1e-10, abs=1e-12)


def test_source_cell_average_against_quadrature():
    """F^{m-1/2} (exact cell averages) against 3-D Gauss-Legendre quadrature of
    the pointwise source over a few dual cells."""
    p = o.Problem(n=(9, 7, 8), delta=(0.3, 0.6, 0.8), kp=(1.0, 2.0, 1.0), km=(0.5, 2.0, 1.5), dt=0.1)
    t = 0.35
    F = o.source_cell_average(p, t, "sin")
    xg, wg = np.polynomial.legendre.leggauss(24)

    def f(x, y, z):
        ph, dph = o.TIME_FACTORS["sin"]
        Px, Py, Pz = o.P_poly(x), o.P_poly(y), o.P_poly(z)
        S = (o.S_series(x, 0.3, 1.0, 0.5) * Py * Pz + Px * o.S_series(y, 0.6, 2.0, 2.0) * Pz
             + Px * Py * o.S_series(z, 0.8, 1.0, 1.5))
        return dph(t) * Px * Py * Pz - ph(t) * S

    for (k, j, i) in [(0, 0, 0), (3, 2, 4), (7, 6, 8), (4, 0, 8)]:
        c = [(i + 1) * p.h[0], (j + 1) * p.h[1], (k + 1) * p.h[2]]
        pts = [c[a] + 0.5 * p.h[a] * xg for a in range(3)]
        X, Y, Z = np.meshgrid(pts[0], pts[1], pts[2], indexing="ij")
        W = wg[:, None, None] * wg[None, :, None] * wg[None, None, :]
        avg = np.sum(W * f(X, Y, Z)) / 8.0
        assert F[k, j, i] == pytest.approx(avg, rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("case", ["sym", "nonsym"])
def test_space_convergence_order(case):
    """Remark after Eq. (coef_expression): second order in space when
    k_+ = k_-, at least min(1 + delta_i) otherwise (fixed small dt)."""
    if case == "sym":
        d, kp, km, need = (0.5, 0.5, 0.5), (1.0,) * 3, (1.0,) * 3, 1.8
    else:
        d, kp, km, need = (0.3, 0.6, 0.8), (1.0,) * 3, (0.5,) * 3, 1.25
    errs = []
    for np1 in [8, 16, 32]:
        n = np1 - 1
        p = o.Problem(n=(n, n, n), delta=d, kp=kp, km=km, dt=1.0 / 32)
        r = o.cn_solve(p, o.exact_u(p, 0.0, "exp"), 32, tol=1e-12, phi="exp")
        errs.append(np.sqrt(np.mean((r.u - o.exact_u(p, 1.0, "exp")) ** 2)))
    assert math.log2(errs[1] / errs[2]) > need
    assert math.log2(errs[0] / errs[1]) > need


def test_time_convergence_order():
    """Eq. (CN): second order in time.  Successive differences on one grid
    (M, 2M, 4M) cancel the spatial error: ratio ~ 4."""
    p0 = dict(n=(9, 9, 9), delta=(0.4, 0.5, 0.6), kp=(1.0,) * 3, km=(1.0,) * 3)
    sols = []
    for M in [4, 8, 16]:
        p = o.Problem(dt=1.0 / M, **p0)
        sols.append(o.cn_solve(p, o.exact_u(p, 0.0, "sin"), M, tol=1e-13, phi="sin").u)
    ratio = np.linalg.norm(sols[0] - sols[1]) / np.linalg.norm(sols[1] - sols[2])
    assert 3.5 < ratio < 4.5


GOLDEN_2D = os.path.join(os.path.dirname(__file__), "golden", "paper_iteration_counts_2d.json")


def _example1(deltas, np1, kp, km):
    n = np1 - 1
    M = np1 // 8
    return o.Problem(n=(n, n, 1), delta=(deltas[0], deltas[1], 0.5), kp=(kp[0], kp[1], 1.0),
                     km=(km[0], km[1], 1.0), dt=1.0 / M, dim=2), M


def test_two_dimensional_operator_is_the_2d_kronecker_form():
    """The 2-D problem (Example 1) against its own Kronecker form written out:
    A = A2 (x) A1 + eta_1 A2 (x) B1 + eta_2 B2 (x) A1, with no third axis."""
    p = o.Problem(n=(5, 4, 1), delta=(0.3, 0.7, 0.5), kp=(1.0, 2.0, 1.0), km=(0.5, 3.0, 1.0), dt=0.1, dim=2)
    T1 = o.toeplitz_T(o.q_coefficients(0.3, 5), 5)
    T2 = o.toeplitz_T(o.q_coefficients(0.7, 4), 4)
    B1, B2 = 1.0 * T1 + 0.5 * T1.T, 2.0 * T2 + 3.0 * T2.T
    A1, A2 = o.mass_A(5), o.mass_A(4)
    e1 = o.eta(0.3, 1.0 / 6, 0.1)
    e2 = o.eta(0.7, 1.0 / 5, 0.1)
    A = np.kron(A2, A1) + e1 * np.kron(A2, B1) + e2 * np.kron(B2, A1)
    np.testing.assert_allclose(o.dense_A(p), A, rtol=1e-14, atol=1e-15)
    v = inp.uniform_vector(p.shape, 3)
    np.testing.assert_allclose(o.apply_A(p, v).ravel(), A @ v.ravel(), rtol=1e-13, atol=1e-14)
    # P of Eq. (pre_definition) in 2-D and its diagonalised form agree
    P = o.dense_P_from_definition(p)
    tau = o.build_tau(p)
    np.testing.assert_allclose(o.apply_P(tau, v).ravel(), P @ v.ravel(), rtol=1e-12, atol=1e-13)
    assert p.symmetric is False


@pytest.mark.parametrize("key", ["0.1,0.2", "0.4,0.5", "0.8,0.9", "0.1,0.9"])
def test_table1_table2_iteration_counts_2d(key):
    """Example 1 with the settings of Sec. 4: PCG(tau) and PGMRES(tau) average
    iteration counts of Tables 1 and 2 for n+1 = 64 and 128 (the GPU tests
    cover 256 and 512)."""
    g = json.load(open(GOLDEN_2D))
    deltas = tuple(float(v) for v in key.split(","))
    for idx, np1 in enumerate(g["n_plus_1"][:2]):
        p, M = _example1(deltas, np1, (5.0, 5.0), (5.0, 5.0))
        r = o.cn_solve(p, o.exact_u(p, 0.0, "4exp"), M, tol=1e-9, phi="4exp", x0="zero")
        assert np.mean(r.iters) == g["table1_pcg_tau"][key][idx]
        pn, M = _example1(deltas, np1, (19.0, 21.0), (21.0, 23.0))
        r = o.cn_solve(pn, o.exact_u(pn, 0.0, "4exp"), M, tol=1e-9, phi="4exp", x0="zero",
                       criterion="preconditioned")
        assert np.mean(r.iters) == g["table2_pgmres_tau"][key][idx]
