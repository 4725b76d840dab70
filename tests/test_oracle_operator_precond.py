"""Pins for the oracle's 3-D operator (Eq. (linear_sys)) and the tau
preconditioner (Eq. (pre_definition) / Eq. (diag_tau_pre)) against explicit
Kronecker products, closed forms and the spectral statements of Sec. 3."""
import math

import numpy as np
import pytest
from scipy import linalg

from oracle import tfde_oracle as o
import tfde_inputs as inp


def _prob(n=(3, 4, 5), delta=(0.3, 0.6, 0.8), kp=(1.0, 1.0, 1.0), km=(1.0, 1.0, 1.0), dt=0.1):
    return o.Problem(n=n, delta=delta, kp=kp, km=km, dt=dt)


@pytest.mark.parametrize("sym", [True, False])
def test_apply_A_matches_kronecker_matrix(sym):
    """Axis-by-axis application == the N x N matrix built with np.kron."""
    p = _prob(kp=(1.0, 2.0, 0.7), km=(1.0, 2.0, 0.7) if sym else (0.5, 1.0, 1.9))
    v = inp.uniform_vector(p.shape, 1)
    A = o.dense_A(p)
    np.testing.assert_allclose(o.apply_A(p, v).ravel(), A @ v.ravel(), rtol=1e-13, atol=1e-13)
    # lexicographic order: a unit vector at (i, j, k) sits at i + n1 (j + n2 k)
    e = np.zeros(p.shape)
    e[2, 1, 0] = 1.0
    col = 0 + p.n[0] * (1 + p.n[1] * 2)
    np.testing.assert_allclose(o.apply_A(p, e).ravel(), A[:, col], rtol=1e-14, atol=1e-15)
    assert np.allclose(A, A.T) == sym


def test_rhs_is_the_cn_right_hand_side():
    """b = (A_N - stiffness) u + dt F = 2 A_N u - A u + dt F."""
    p = _prob()
    u = inp.uniform_vector(p.shape, 2)
    F = inp.uniform_vector(p.shape, 3)
    AN = np.kron(p.M[2], np.kron(p.M[1], p.M[0]))
    ref = 2 * AN @ u.ravel() - o.dense_A(p) @ u.ravel() + p.dt * F.ravel()
    np.testing.assert_allclose(o.rhs(p, u, F).ravel(), ref, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3, 8, 17])
def test_dst_orthogonal_symmetric_and_diagonalises_mass(n):
    S = o.dst_matrix(n)
    np.testing.assert_allclose(S, S.T, atol=1e-15)
    np.testing.assert_allclose(S @ S, np.eye(n), atol=1e-14)
    D = S @ o.mass_A(n) @ S
    np.testing.assert_allclose(D, np.diag(o.mass_eigenvalues(n)), atol=1e-14)
    lam = o.mass_eigenvalues(n)
    assert np.all(lam > 0.5) and np.all(lam < 1.0)   # Lemma tridiag_eig


@pytest.mark.parametrize("d", [0.1, 0.45, 0.9])
@pytest.mark.parametrize("n", [2, 3, 10, 33])
def test_tau_matrix_is_diagonalised_with_printed_eigenvalues(d, n):
    """tau(H(T)) = H(T) - Hankel is diagonalised by S_n and its eigenvalues are
    the (corrected) formula of Lemma 1D_tau_SPD; all positive."""
    q = o.q_coefficients(d, n)
    T = o.toeplitz_T(q, n)
    H = 0.5 * (T + T.T)
    tau = o.tau_matrix_of_symmetric_toeplitz(H[:, 0])
    S = o.dst_matrix(n)
    D = S @ tau @ S
    off = D - np.diag(np.diag(D))
    assert np.abs(off).max() < 1e-14
    np.testing.assert_allclose(np.diag(D), o.tau_eigenvalues(q, n), rtol=1e-12, atol=1e-15)
    assert np.all(o.tau_eigenvalues(q, n) > 0)


@pytest.mark.parametrize("d", [0.05, 0.3, 0.6, 0.95])
def test_one_dim_tau_spectrum_lemma(d):
    """Lemma monotony_coefficients via (1D_bound): eig(tau(H)^{-1} H) in (1/2, 3/2)."""
    for n in [4, 16, 64]:
        q = o.q_coefficients(d, n)
        T = o.toeplitz_T(q, n)
        H = 0.5 * (T + T.T)
        tau = o.tau_matrix_of_symmetric_toeplitz(H[:, 0])
        ev = linalg.eigh(H, tau, eigvals_only=True)
        assert ev.min() > 0.5 and ev.max() < 1.5


def test_preconditioner_definition_matches_diagonalised_form():
    """Eq. (pre_definition) as explicit Kronecker sums == S_N Lambda S_N
    (Eq. (diag_tau_pre)); apply_Pinv inverts it; lambda_min(P) > 1/8
    (Lemma spd_tau_pre)."""
    p = _prob(n=(4, 3, 5), kp=(1.0, 2.0, 0.7), km=(0.5, 1.0, 1.9))
    Pd = o.dense_P_from_definition(p)
    tau = o.build_tau(p)
    v = inp.uniform_vector(p.shape, 5)
    np.testing.assert_allclose(o.apply_P(tau, v).ravel(), Pd @ v.ravel(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(o.apply_Pinv(tau, o.apply_P(tau, v)), v, rtol=1e-12, atol=1e-13)
    assert np.linalg.eigvalsh(Pd).min() > 1.0 / 8.0
    assert tau.Lam.min() > 1.0 / 8.0


def _spectral_case(n, d, kp, km, dt=0.05):
    p = o.Problem(n=(n, n, n), delta=d, kp=kp, km=km, dt=dt)
    A = o.dense_A(p)
    Pd = o.dense_P_from_definition(p)
    w, U = np.linalg.eigh(Pd)
    Pmh = U @ np.diag(w ** -0.5) @ U.T
    return p, A, Pd, Pmh


@pytest.mark.parametrize("d", [(0.1, 0.2, 0.3), (0.5, 0.5, 0.5), (0.7, 0.8, 0.9), (0.1, 0.5, 0.9)])
def test_cg_spectral_theorem(d):
    """Theorem CG_bounded_sprctrum: symmetric case, eig(P^{-1/2} A P^{-1/2}) in (1/2, 3/2)."""
    for n, dt in [(5, 0.05), (7, 1.0)]:
        _, A, Pd, _ = _spectral_case(n, d, (5.0,) * 3, (5.0,) * 3, dt)
        ev = linalg.eigh(A, Pd, eigvals_only=True)
        assert ev.min() > 0.5 and ev.max() < 1.5


@pytest.mark.parametrize("d,kp,km", [((0.1, 0.2, 0.3), (19.0, 21.0, 23.0), (21.0, 23.0, 25.0)),
                                     ((0.7, 0.8, 0.9), (1.0, 1.0, 1.0), (0.5, 0.5, 0.5)),
                                     ((0.3, 0.6, 0.8), (2.0, 0.5, 1.5), (0.5, 2.0, 1.0))])
def test_nonsymmetric_spectral_lemmas_and_gmres_rate(d, kp, km):
    """Lemma prop:eigen_S: eig(P^{-1/2} H(A) P^{-1/2}) in (1/2, 3/2);
    Lemma eigen_Skew: rho(P^{-1/2} S(A) P^{-1/2}) <= varsigma;
    Theorem theorem_main: the GMRES residual on the two-sided system obeys
    ||r_k|| <= omega^k ||r_0||, omega = sqrt((2 + 4 s^2)/(3 + 4 s^2))."""
    n = 5
    p, A, Pd, Pmh = _spectral_case(n, d, kp, km, dt=0.5)
    Hs = 0.5 * (A + A.T)
    Sk = 0.5 * (A - A.T)
    evH = np.linalg.eigvalsh(Pmh @ Hs @ Pmh)
    assert evH.min() > 0.5 and evH.max() < 1.5
    sig = 1.5 * max(math.tan(d[i] * math.pi / 2) * abs(kp[i] - km[i]) / (kp[i] + km[i]) for i in range(3))
    rho = np.abs(np.linalg.eigvals(Pmh @ Sk @ Pmh)).max()
    assert rho <= sig + 1e-12
    omega = math.sqrt((2 + 4 * sig ** 2) / (3 + 4 * sig ** 2))
    Z = Pmh @ A @ Pmh
    rhs = Pmh @ inp.uniform_vector(p.shape, 7).ravel()
    # GMRES iterate k minimises ||w - Z x|| over the Krylov space K_k(Z, w) (x0 = 0)
    Kr = [rhs]
    r0 = np.linalg.norm(rhs)
    for k in range(1, 9):
        Q, _ = np.linalg.qr(np.array(Kr).T)
        y, *_ = np.linalg.lstsq(Z @ Q, rhs, rcond=None)
        rk = np.linalg.norm(rhs - Z @ Q @ y)
        assert rk <= omega ** k * r0 * (1 + 1e-10)
        Kr.append(Z @ Kr[-1])


@pytest.mark.parametrize("d", [0.2, 0.5, 0.8])
def test_skew_vs_hermitian_quadratic_forms(d):
    """Lemma Her_Skew_Her: |v* S(T) v| <= tan(d pi/2) v* H(T) v, i.e. the
    generalised eigenvalues of (i S(T), H(T)) lie in [-tan, tan]."""
    for n in [3, 12, 40]:
        q = o.q_coefficients(d, n)
        T = o.toeplitz_T(q, n)
        ev = linalg.eigh(1j * 0.5 * (T - T.T), 0.5 * (T + T.T), eigvals_only=True)
        assert np.abs(ev).max() <= math.tan(d * math.pi / 2) + 1e-12


@pytest.mark.parametrize("sym", [True, False])
def test_pointwise_operator_matches_kronecker_rows(sym):
    """apply_A_at (used by the full-size sampled GPU checks) against rows of
    the explicit N x N Kronecker matrices of Eq. (linear_sys): op "A" is a
    row of A, op "RHS" a row of the right-hand-side operator 2 A_N - A, at
    random points of a 7 x 6 x 5 grid that include every face and corner."""
    p = _prob(n=(7, 6, 5), kp=(1.0, 2.0, 0.7), km=(1.0, 2.0, 0.7) if sym else (0.5, 1.0, 1.9))
    v = inp.uniform_vector(p.shape, 11)
    A = o.dense_A(p)
    AN = np.kron(p.M[2], np.kron(p.M[1], p.M[0]))
    R = 2.0 * AN - A
    rng = np.random.default_rng(5)
    pts = [(int(rng.integers(0, p.n[2])), int(rng.integers(0, p.n[1])), int(rng.integers(0, p.n[0])))
           for _ in range(40)]
    pts += [(0, 0, 0), (p.n[2] - 1, p.n[1] - 1, p.n[0] - 1), (0, p.n[1] - 1, 0), (p.n[2] - 1, 0, p.n[0] - 1)]
    rows = [i + p.n[0] * (j + p.n[1] * k) for (k, j, i) in pts]
    np.testing.assert_allclose(o.apply_A_at(p, v, pts, "A"), A[rows] @ v.ravel(), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(o.apply_A_at(p, v, pts, "RHS"), R[rows] @ v.ravel(), rtol=1e-13, atol=1e-14)
    # and the RHS branch is the oracle's right-hand side without a source
    np.testing.assert_allclose(o.apply_A_at(p, v, pts, "RHS"),
                               np.array([o.rhs(p, v, None)[k, j, i] for (k, j, i) in pts]), rtol=1e-13, atol=1e-14)
