"""Plain FP64 CPU oracle for the CN-FV tau-preconditioned Krylov method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The product (the CUDA library and its binding) never calls it, and it
shares no code with the product.

It restates, slowly and literally, what the paper (Qu, Lei, Hon, Huang,
"Optimal preconditioning techniques for finite volume approximation of
three-dimensional conservative space-fractional diffusion equations") computes:

* Sec. 2, Eq. (CN) and Eq. (fvm_sol): Crank-Nicolson in time, finite volumes with
  the piecewise-linear nodal basis in space;
* Sec. 2, Eq. (coef_expression) and the s_k display after it: the flux
  coefficients s_k and the Toeplitz generator q_k;
* Sec. 2, Eq. (T_ni), Eq. (stiff_matrix), Eq. (tridiag_matrix): T, B, A_n and eta;
* Sec. 2, Eq. (original_matrix_form) / Eq. (linear_sys): the system A u^m = b^m;
* Sec. 3, Eq. (pre_definition), Eq. (diag_tau_pre): the tau preconditioner
  P = S_N Lambda S_N with the 1-D DST-I matrix S_n;
* Sec. 3, Lemma 1D_tau_SPD: the tau eigenvalues from the first column of H(T)
  (the printed sum is garbled; the reading used here is
  lambda_k = q_1 + (q_0+q_2) cos(theta_k) + sum_{j=2}^{n-1} q_{j+1} cos(j theta_k));
* Sec. 3.1 / 3.2 and Sec. 4: PCG for k_+ = k_-, left-preconditioned restarted
  GMRES(20) otherwise;
* Sec. 4, Example 2: the manufactured 3-D solution and its Gamma-series source.

Array convention: a 3-D grid function is an ndarray of shape (n3, n2, n1)
indexed [k, j, i] (z, y, x), so that C order is the paper's lexicographic
ordering with x fastest (Sec. 2, the definition of u^m).

Every routine is FP64.  Library primitives used as steps: numpy matmul /
tensordot, numpy.linalg (only in tests), math.gamma, decimal arithmetic.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from decimal import Decimal, localcontext

import numpy as np

# --------------------------------------------------------------------------
# Sec. 2: flux coefficients s_k and Toeplitz generator q_k
# --------------------------------------------------------------------------


def s_coefficients_decimal(delta: float, n: int, digits: int = 60) -> list:
    """s_k^{(delta)} for k = 0..n as Decimals (Sec. 2, display defining s_k).

    s_0 = (1/2)^d, s_1 = (3/2)^d - 2 (1/2)^d,
    s_k = (k+1/2)^d - 2 (k-1/2)^d + (k-3/2)^d  (2 <= k <= n).
    Evaluated with ``digits`` significant decimal digits because the second
    difference of k^d cancels about log10(k^2) digits.
    """
    with localcontext() as ctx:
        ctx.prec = digits
        d = Decimal(delta)  # the exact binary value of the FP64 delta
        half = Decimal(1) / Decimal(2)

        def pw(x: Decimal) -> Decimal:
            return x ** d

        s = []
        for k in range(n + 1):
            if k == 0:
                s.append(pw(half))
            elif k == 1:
                s.append(pw(Decimal(3) * half) - 2 * pw(half))
            else:
                kk = Decimal(k)
                s.append(pw(kk + half) - 2 * pw(kk - half) + pw(kk - 3 * half))
        return s


def q_coefficients_decimal(delta: float, n: int, digits: int = 60) -> list:
    """q_k^{(delta)} for k = 0..n as Decimals, Eq. (coef_expression):
    q_0 = -s_0, q_k = s_{k-1} - s_k (1 <= k <= n)."""
    s = s_coefficients_decimal(delta, n, digits)
    with localcontext() as ctx:
        ctx.prec = digits
        q = [-s[0]]
        for k in range(1, n + 1):
            q.append(s[k - 1] - s[k])
    return q


def s_coefficients(delta: float, n: int) -> np.ndarray:
    """s_k (k = 0..n), high-precision evaluation rounded once to FP64."""
    return np.array([float(v) for v in s_coefficients_decimal(delta, n)], dtype=np.float64)


def q_coefficients(delta: float, n: int) -> np.ndarray:
    """q_k (k = 0..n), high-precision evaluation rounded once to FP64."""
    return np.array([float(v) for v in q_coefficients_decimal(delta, n)], dtype=np.float64)


# --------------------------------------------------------------------------
# Sec. 2: the 1-D matrices
# --------------------------------------------------------------------------


def toeplitz_T(q: np.ndarray, n: int) -> np.ndarray:
    """T_n^{(delta)} of Eq. (T_ni): lower Hessenberg Toeplitz with
    T[i, j] = q_{i-j+1} when 0 <= i-j+1 <= n, else 0 (0-based i, j).
    The diagonal is q_1, the superdiagonal q_0, the first column q_1..q_n."""
    T = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        for j in range(n):
            m = i - j + 1
            if 0 <= m <= n:
                T[i, j] = q[m]
    return T


def stiffness_B(T: np.ndarray, kp: float, km: float) -> np.ndarray:
    """B_n = k_+ T + k_- T^T, Eq. (stiff_matrix)."""
    return kp * T + km * T.T


def mass_A(n: int) -> np.ndarray:
    """A_n = tridiag(1, 6, 1) / 8, Eq. (tridiag_matrix)."""
    A = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        A[i, i] = 6.0 / 8.0
        if i > 0:
            A[i, i - 1] = 1.0 / 8.0
        if i + 1 < n:
            A[i, i + 1] = 1.0 / 8.0
    return A


def eta(delta: float, h: float, dt: float) -> float:
    """eta_delta = dt / (2 Gamma(delta+1) h^(2-delta)), Sec. 2 after Eq. (original_matrix_form)."""
    return dt / (2.0 * math.gamma(delta + 1.0) * h ** (2.0 - delta))


def dst_matrix(n: int) -> np.ndarray:
    """S_n with [S_n]_{jk} = sqrt(2/(n+1)) sin(j k pi / (n+1)), 1 <= j,k <= n (Sec. 3)."""
    j = np.arange(1, n + 1, dtype=np.float64)
    return math.sqrt(2.0 / (n + 1)) * np.sin(np.outer(j, j) * math.pi / (n + 1))


def mass_eigenvalues(n: int) -> np.ndarray:
    """Eigenvalues of A_n in the order S_n diagonalises it:
    (6 + 2 cos(k pi/(n+1))) / 8, k = 1..n (tridiagonal Toeplitz closed form;
    Lemma tridiag_eig gives the enclosing interval (1/2, 1))."""
    k = np.arange(1, n + 1, dtype=np.float64)
    return (6.0 + 2.0 * np.cos(k * math.pi / (n + 1))) / 8.0


def tau_eigenvalues(q: np.ndarray, n: int) -> np.ndarray:
    """Eigenvalues of tau(H(T_n)) (Lemma 1D_tau_SPD), k = 1..n:
    lambda_k = q_1 + (q_0+q_2) cos(theta_k) + sum_{j=2}^{n-1} q_{j+1} cos(j theta_k),
    theta_k = k pi / (n+1).  This is t_0 + 2 sum_j t_j cos(j theta_k) for the first
    column t = [q_1, (q_0+q_2)/2, q_3/2, ..., q_n/2] of H(T_n) (proof of
    Theorem CG_bounded_sprctrum)."""
    lam = np.zeros(n, dtype=np.float64)
    for kk in range(1, n + 1):
        th = kk * math.pi / (n + 1)
        v = q[1]
        if n >= 2:
            v += (q[0] + q[2]) * math.cos(th)
        for j in range(2, n):
            v += q[j + 1] * math.cos(j * th)
        lam[kk - 1] = v
    return lam


def tau_matrix_of_symmetric_toeplitz(t: np.ndarray) -> np.ndarray:
    """tau(T) for a symmetric Toeplitz T with first column t (length n):
    T minus the Hankel matrix whose first column is (t_2, ..., t_{n-1}, 0, 0)
    and whose last column is its reverse (0, 0, t_{n-1}, ..., t_2).  With
    s = i + j (0-based) the Hankel entry is t_{s+2} for s <= n-3, zero for
    s in {n-2, n-1, n}, and t_{2n-s} for s >= n+1.  This is the natural tau
    approximation cited in Sec. 3 (Bini and Di Benedetto)."""
    n = len(t)
    T = np.empty((n, n))
    H = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            T[i, j] = t[abs(i - j)]
            s = i + j
            if s <= n - 3:
                H[i, j] = t[s + 2]
            elif s >= n + 1:
                H[i, j] = t[2 * n - s]
    return T - H


# --------------------------------------------------------------------------
# Problem definition (Sec. 1 and Sec. 2)
# --------------------------------------------------------------------------


@dataclass
class Problem:
    """One 3-D problem: grid, fractional orders, diffusivities and time step.

    n = (n1, n2, n3) interior points per axis (x, y, z); lo/hi the box Omega;
    delta = (alpha, beta, gamma); kp/km = k_{i,+}, k_{i,-}; dt the CN step."""

    n: tuple
    delta: tuple
    kp: tuple
    km: tuple
    dt: float
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    # dim = 2: the two-dimensional problem of Sec. 4, Example 1 (n[2] must be
    # 1): the system of Eq. (linear_sys) without the third axis, i.e. its
    # Kronecker form with the third mass factor the 1 x 1 identity and no
    # third stiffness term
    dim: int = 3
    # derived
    h: tuple = field(init=False)
    q: list = field(init=False)
    T: list = field(init=False)
    B: list = field(init=False)
    M: list = field(init=False)
    eta: tuple = field(init=False)

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        self.h = tuple((self.hi[a] - self.lo[a]) / (self.n[a] + 1) for a in range(3))
        self.q = [q_coefficients(self.delta[a], self.n[a]) for a in range(3)]
        self.T = [toeplitz_T(self.q[a], self.n[a]) for a in range(3)]
        self.B = [stiffness_B(self.T[a], self.kp[a], self.km[a]) for a in range(3)]
        self.M = [mass_A(self.n[a]) for a in range(3)]
        self.eta = tuple(eta(self.delta[a], self.h[a], self.dt) for a in range(3))
        if self.dim == 2:
            if self.n[2] != 1:
                raise ValueError("a 2-D problem has n[2] = 1")
            self.M[2] = np.ones((1, 1))
            self.B[2] = np.zeros((1, 1))
            self.eta = (self.eta[0], self.eta[1], 0.0)

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])

    @property
    def symmetric(self) -> bool:
        """k_{i,+} = k_{i,-} for every axis (Sec. 2 remark after Eq. (linear_sys))."""
        return all(self.kp[a] == self.km[a] for a in range(self.dim))

    def nodes(self, axis: int) -> np.ndarray:
        """Interior nodes x_p = a + p h, p = 1..n (Sec. 2)."""
        return self.lo[axis] + self.h[axis] * np.arange(1, self.n[axis] + 1, dtype=np.float64)


# --------------------------------------------------------------------------
# Kronecker-structured application.  Axis a in {0: x, 1: y, 2: z}.
# --------------------------------------------------------------------------


def apply_along(Mat: np.ndarray, v: np.ndarray, axis: int) -> np.ndarray:
    """(I (x) .. (x) Mat (x) .. (x) I) v with Mat acting on the given axis of the
    grid function v[k, j, i]; axis 0 = x (last array index), 2 = z (first)."""
    arr_axis = 2 - axis
    out = np.tensordot(Mat, v, axes=([1], [arr_axis]))  # contracted axis becomes first
    return np.moveaxis(out, 0, arr_axis)


def apply_mass_all(prob: Problem, v: np.ndarray) -> np.ndarray:
    """A_N v = (A_{n3} (x) A_{n2} (x) A_{n1}) v (Sec. 2, notation A_N)."""
    out = apply_along(prob.M[0], v, 0)
    out = apply_along(prob.M[1], out, 1)
    return apply_along(prob.M[2], out, 2)


def stiffness_terms(prob: Problem, v: np.ndarray) -> np.ndarray:
    """eta_a A3 A2 B1 v + eta_b A3 B2 A1 v + eta_c B3 A2 A1 v, the three
    Kronecker terms of Eq. (linear_sys) (without A_N)."""
    M, B, e = prob.M, prob.B, prob.eta
    t1 = apply_along(M[2], apply_along(M[1], apply_along(B[0], v, 0), 1), 2)
    t2 = apply_along(M[2], apply_along(B[1], apply_along(M[0], v, 0), 1), 2)
    t3 = apply_along(B[2], apply_along(M[1], apply_along(M[0], v, 0), 1), 2)
    return e[0] * t1 + e[1] * t2 + e[2] * t3


def apply_A(prob: Problem, v: np.ndarray) -> np.ndarray:
    """A v with A = A_N + sum of the three stiffness terms, Eq. (linear_sys)."""
    return apply_mass_all(prob, v) + stiffness_terms(prob, v)


def rhs(prob: Problem, u_prev: np.ndarray, F: np.ndarray | None) -> np.ndarray:
    """b^m = (A_N - stiffness terms) u^{m-1} + dt F^{m-1/2}, Eq. (linear_sys)
    (the tau multiplying F there is the time step)."""
    b = apply_mass_all(prob, u_prev) - stiffness_terms(prob, u_prev)
    if F is not None:
        b = b + prob.dt * F
    return b


def dense_A(prob: Problem) -> np.ndarray:
    """The N x N matrix of Eq. (original_matrix_form) by explicit Kronecker
    products (small grids only)."""
    M, B, e = prob.M, prob.B, prob.eta
    AN = np.kron(M[2], np.kron(M[1], M[0]))
    return (AN + e[0] * np.kron(M[2], np.kron(M[1], B[0]))
            + e[1] * np.kron(M[2], np.kron(B[1], M[0]))
            + e[2] * np.kron(B[2], np.kron(M[1], M[0])))


# --------------------------------------------------------------------------
# Sec. 3: the tau preconditioner
# --------------------------------------------------------------------------


@dataclass
class TauPreconditioner:
    """P = S_N Lambda S_N, Eq. (diag_tau_pre)."""

    S: list
    Lam: np.ndarray  # shape (n3, n2, n1)


def build_tau(prob: Problem) -> TauPreconditioner:
    """Lambda = LA3 LA2 LA1 + sum_i eta_i (k_{i+}+k_{i-}) (.. Lambda_i^delta ..)
    from the 1-D eigenvalue arrays (Eq. (diag_tau_pre))."""
    a = [mass_eigenvalues(prob.n[ax]) for ax in range(3)]
    lam = [tau_eigenvalues(prob.q[ax], prob.n[ax]) for ax in range(3)]
    c = [prob.eta[ax] * (prob.kp[ax] + prob.km[ax]) for ax in range(3)]
    if prob.dim == 2:   # the absent third axis: identity mass factor, no stiffness term
        a[2] = np.ones(1)
        c[2] = 0.0
    A1, A2, A3 = (a[0][None, None, :], a[1][None, :, None], a[2][:, None, None])
    L1, L2, L3 = (lam[0][None, None, :], lam[1][None, :, None], lam[2][:, None, None])
    Lam = A3 * A2 * A1 + c[0] * A3 * A2 * L1 + c[1] * A3 * L2 * A1 + c[2] * L3 * A2 * A1
    S = [dst_matrix(prob.n[ax]) for ax in range(3)]
    return TauPreconditioner(S=S, Lam=Lam)


def apply_S_N(S: list, v: np.ndarray) -> np.ndarray:
    """S_N v with S_N = S_{n3} (x) S_{n2} (x) S_{n1} (direct dense DST-I per axis)."""
    out = apply_along(S[0], v, 0)
    out = apply_along(S[1], out, 1)
    return apply_along(S[2], out, 2)


def apply_Pinv(tau: TauPreconditioner, r: np.ndarray) -> np.ndarray:
    """z = P^{-1} r = S_N Lambda^{-1} S_N r (S_n is symmetric and S_n^2 = I)."""
    return apply_S_N(tau.S, apply_S_N(tau.S, r) / tau.Lam)


def apply_P(tau: TauPreconditioner, v: np.ndarray) -> np.ndarray:
    """P v = S_N Lambda S_N v."""
    return apply_S_N(tau.S, apply_S_N(tau.S, v) * tau.Lam)


def dense_P_from_definition(prob: Problem) -> np.ndarray:
    """P of Eq. (pre_definition): every B_i replaced by
    (k_{i+}+k_{i-}) tau(H(T_i)), mass factors kept (small grids only)."""
    M = prob.M
    taus = []
    for ax in range(3):
        T = prob.T[ax]
        H = 0.5 * (T + T.T)
        taus.append((prob.kp[ax] + prob.km[ax]) * tau_matrix_of_symmetric_toeplitz(H[:, 0]))
    e = prob.eta
    AN = np.kron(M[2], np.kron(M[1], M[0]))
    return (AN + e[0] * np.kron(M[2], np.kron(M[1], taus[0]))
            + e[1] * np.kron(M[2], np.kron(taus[1], M[0]))
            + e[2] * np.kron(taus[2], np.kron(M[1], M[0])))


# --------------------------------------------------------------------------
# Krylov solvers (Sec. 3.1, 3.2; settings of Sec. 4)
# --------------------------------------------------------------------------


@dataclass
class SolveInfo:
    iters: int = 0        # PCG iterations, or total GMRES inner (Arnoldi) steps
    restarts: int = 0
    relres: float = float("nan")   # final true relative residual ||b - A x|| / ||b||
    converged: bool = False


def _dot(a, b):
    return float(np.dot(a.ravel(), b.ravel()))


def _norm(a):
    return math.sqrt(_dot(a, a))


def pcg(A, Minv, b, x0, tol, maxit):
    """Textbook preconditioned conjugate gradients for the SPD system (Sec. 3.1).

    A, Minv: callables on grid functions.  Stops when ||r_j|| <= tol ||b|| for
    the recursively updated residual and then confirms with the true residual
    (continuing from it if the confirmation fails), as MATLAB's pcg does."""
    info = SolveInfo()
    x = x0.copy()
    nb = _norm(b)
    if nb == 0.0:
        info.relres, info.converged = 0.0, True
        return np.zeros_like(b), info
    r = b - A(x)
    if _norm(r) <= tol * nb:
        info.relres, info.converged = _norm(r) / nb, True
        return x, info
    z = Minv(r)
    p = z.copy()
    rz = _dot(r, z)
    while info.iters < maxit:
        Ap = A(p)
        alpha = rz / _dot(p, Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        info.iters += 1
        if _norm(r) <= tol * nb:
            rt = b - A(x)
            if _norm(rt) <= tol * nb:
                info.relres, info.converged = _norm(rt) / nb, True
                return x, info
            r = rt  # continue from the true residual
            z = Minv(r)
            p = z.copy()
            rz = _dot(r, z)
            continue
        z = Minv(r)
        rz_new = _dot(r, z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    info.relres = _norm(b - A(x)) / nb
    return x, info


def gmres_left(A, Minv, b, x0, tol, maxit, restart=20, criterion="preconditioned"):
    """Restarted GMRES(restart) on the left-preconditioned system
    P^{-1} A u = P^{-1} b, Eq. (one_side_system); modified Gram-Schmidt Arnoldi
    and Givens rotations (Saad's textbook form).

    criterion "preconditioned": stop when ||P^{-1}(b - A x)|| <= tol ||P^{-1} b||
    (the rule MATLAB's gmres applies with a left preconditioner, Sec. 4);
    "true": additionally require ||b - A x|| <= tol ||b|| at termination.
    maxit counts inner (Arnoldi) steps."""
    info = SolveInfo()
    x = x0.copy()
    nb = _norm(b)
    if nb == 0.0:
        info.relres, info.converged = 0.0, True
        return np.zeros_like(b), info
    pb = _norm(Minv(b))

    def accepted(x):
        pr = _norm(Minv(b - A(x)))
        if pr > tol * pb:
            return False
        return criterion != "true" or _norm(b - A(x)) <= tol * nb

    while info.iters < maxit:
        r = Minv(b - A(x))
        beta = _norm(r)
        if beta <= tol * pb and accepted(x):
            info.converged = True
            break
        V = [r / beta]
        R = np.zeros((restart + 1, restart))   # Hessenberg, rotated in place to R
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        k_used = 0
        for j in range(restart):
            w = Minv(A(V[j]))
            for i in range(j + 1):
                R[i, j] = _dot(w, V[i])
                w = w - R[i, j] * V[i]
            hnext = _norm(w)
            R[j + 1, j] = hnext
            for i in range(j):  # previous rotations on the new column
                t = cs[i] * R[i, j] + sn[i] * R[i + 1, j]
                R[i + 1, j] = -sn[i] * R[i, j] + cs[i] * R[i + 1, j]
                R[i, j] = t
            den = math.hypot(R[j, j], R[j + 1, j])
            cs[j] = R[j, j] / den
            sn[j] = R[j + 1, j] / den
            R[j, j] = den
            R[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            info.iters += 1
            k_used = j + 1
            if abs(g[j + 1]) <= tol * pb or info.iters >= maxit or hnext == 0.0:
                break
            V.append(w / hnext)
        y = np.zeros(k_used)   # back substitution R y = g
        for i in range(k_used - 1, -1, -1):
            y[i] = (g[i] - np.dot(R[i, i + 1:k_used], y[i + 1:k_used])) / R[i, i]
        for i in range(k_used):
            x = x + y[i] * V[i]
        info.restarts += 1
        if accepted(x):
            info.converged = True
            break
    info.relres = _norm(b - A(x)) / nb
    return x, info


# --------------------------------------------------------------------------
# Sec. 4, Example 2: manufactured solution u = phi(t) P(x) P(y) P(z),
# P(x) = x^2 (1-x)^2 on (0,1), and its source term
#   f = phi'(t) P P P - phi(t) [S_a(x) P(y) P(z) + P(x) S_b(y) P(z) + P(x) P(y) S_c(z)],
#   S_d(x) = sum_{k=0}^{2} (-1)^{2-k} C(2,k) Gamma(5-k)/Gamma(3-k+d)
#            [k_+ x^{2-k+d} + k_- (1-x)^{2-k+d}].
# phi(t) = sin(t+1) in the paper's Example 2; phi(t) = exp(-t) in the
# exp-decay variant of the same example.
# --------------------------------------------------------------------------

TIME_FACTORS = {
    # name: (phi, phi')
    "sin": (lambda t: math.sin(t + 1.0), lambda t: math.cos(t + 1.0)),
    "exp": (lambda t: math.exp(-t), lambda t: -math.exp(-t)),
    "4exp": (lambda t: 4.0 * math.exp(t), lambda t: 4.0 * math.exp(t)),   # Example 1 (2-D)
}


def P_poly(x):
    """P(x) = x^2 (1-x)^2."""
    return x * x * (1.0 - x) ** 2


def S_series(x, d, kp, km):
    """S_d(x): the conservative fractional operator applied to P (Example 2)."""
    out = 0.0
    for k in range(3):
        coef = (-1.0) ** (2 - k) * math.comb(2, k) * math.gamma(5 - k) / math.gamma(3 - k + d)
        p = 2 - k + d
        out = out + coef * (kp * x ** p + km * (1.0 - x) ** p)
    return out


def exact_u(prob: Problem, t: float, phi: str = "exp") -> np.ndarray:
    """Nodal values of the manufactured solution at time t."""
    x, y, z = (prob.nodes(a) for a in range(3))
    Pz = P_poly(z) if prob.dim == 3 else np.ones(1)
    return TIME_FACTORS[phi][0](t) * (Pz[:, None, None] * P_poly(y)[None, :, None]
                                      * P_poly(x)[None, None, :])


def _cell_avg_power(a, b, p):
    """(1/(b-a)) * integral_a^b x^p dx for 0 <= a < b (exact antiderivative;
    b^{p+1} - a^{p+1} written as a^{p+1} expm1((p+1) log1p((b-a)/a)) when a > 0
    so that thin cells keep full relative accuracy)."""
    h = b - a
    out = np.empty_like(a)
    pos = a > 0
    aa = a[pos]
    out[pos] = aa ** (p + 1.0) * np.expm1((p + 1.0) * np.log1p(h[pos] / aa)) / ((p + 1.0) * h[pos])
    out[~pos] = b[~pos] ** (p + 1.0) / ((p + 1.0) * h[~pos])
    return out


def cell_average_P(prob: Problem, axis: int) -> np.ndarray:
    """(1/h) integral over [x_{i-1/2}, x_{i+1/2}] of P(x) = x^2 - 2 x^3 + x^4."""
    xc = prob.nodes(axis)
    h = prob.h[axis]
    a, b = xc - 0.5 * h, xc + 0.5 * h
    return _cell_avg_power(a, b, 2.0) - 2.0 * _cell_avg_power(a, b, 3.0) + _cell_avg_power(a, b, 4.0)


def cell_average_S(prob: Problem, axis: int) -> np.ndarray:
    """(1/h) integral over the dual cell of S_delta(x) (exact antiderivatives)."""
    xc = prob.nodes(axis)
    h = prob.h[axis]
    a, b = xc - 0.5 * h, xc + 0.5 * h
    d, kp, km = prob.delta[axis], prob.kp[axis], prob.km[axis]
    out = np.zeros_like(xc)
    for k in range(3):
        coef = (-1.0) ** (2 - k) * math.comb(2, k) * math.gamma(5 - k) / math.gamma(3 - k + d)
        p = 2 - k + d
        # the (1-x)^p part: substitute y = 1 - x, cell [1-b, 1-a]
        out += coef * (kp * _cell_avg_power(a, b, p) + km * _cell_avg_power(1.0 - b, 1.0 - a, p))
    return out


def source_cell_average(prob: Problem, t: float, phi: str = "exp") -> np.ndarray:
    """F^{m-1/2} at time t: f_{ijk} = (h1 h2 h3)^{-1} * integral of f over the
    dual cell (Sec. 2, the definition of F^{m-1/2}).  f is a sum of separable
    products, so the cell average is the same sum of products of 1-D cell
    averages, each integrated exactly."""
    ph, dph = TIME_FACTORS[phi]
    Px, Py, Pz = (cell_average_P(prob, a) for a in range(3))
    Sx, Sy, Sz = (cell_average_S(prob, a) for a in range(3))
    if prob.dim == 2:   # Example 1: u = phi(t) P(x) P(y), no third factor
        Pz, Sz = np.ones(1), np.zeros(1)
    X = lambda v: v[None, None, :]
    Y = lambda v: v[None, :, None]
    Z = lambda v: v[:, None, None]
    PPP = Z(Pz) * Y(Py) * X(Px)
    SPP = Z(Pz) * Y(Py) * X(Sx) + Z(Pz) * Y(Sy) * X(Px) + Z(Sz) * Y(Py) * X(Px)
    return dph(t) * PPP - ph(t) * SPP


# --------------------------------------------------------------------------
# Sec. 2, Eq. (CN) / Eq. (linear_sys): the time loop
# --------------------------------------------------------------------------


@dataclass
class CNResult:
    u: np.ndarray
    iters: list
    relres: list


def cn_solve(prob: Problem, u0: np.ndarray, M: int, *, tol: float, phi: str | None = "exp",
             x0: str = "prev", maxit: int | None = None, restart: int = 20,
             criterion: str = "true", sources=None) -> CNResult:
    """March u^0 -> u^M with one linear solve per step, t_m = m dt.

    phi: manufactured source time factor ("exp" / "sin"), or None for f = 0;
    ``sources`` may instead give a callable t -> F array.  x0 = "prev" starts
    each solve from u^{m-1}, "zero" from 0 (MATLAB's default).  PCG when
    k_+ = k_- on every axis, else left-preconditioned GMRES(restart)."""
    tau = build_tau(prob)
    Aop = lambda v: apply_A(prob, v)
    Pinv = lambda r: apply_Pinv(tau, r)
    if maxit is None:
        maxit = int(np.prod(prob.n))
    u = u0.copy()
    iters, relres = [], []
    for m in range(1, M + 1):
        th = (m - 0.5) * prob.dt
        if sources is not None:
            F = sources(th)
        elif phi is not None:
            F = source_cell_average(prob, th, phi)
        else:
            F = None
        b = rhs(prob, u, F)
        xs = u if x0 == "prev" else np.zeros_like(u)
        if prob.symmetric:
            u, info = pcg(Aop, Pinv, b, xs, tol, maxit)
        else:
            crit = "preconditioned" if criterion == "preconditioned" else "true"
            u, info = gmres_left(Aop, Pinv, b, xs, tol, maxit, restart, crit)
        iters.append(info.iters)
        relres.append(info.relres)
    return CNResult(u=u, iters=iters, relres=relres)


def apply_A_at(prob: Problem, v: np.ndarray, points, op: str = "A") -> np.ndarray:
    """(A v) or (RHS operator v) at the given (k, j, i) points, one by one, from
    the Kronecker form of Eq. (linear_sys): every term is a product of three
    1-D rows, so each output needs only the <= 3 x 3 x n block of v under the
    non-zero pattern of its rows (the mass rows are tridiagonal)."""
    sgn = 1.0 if op == "A" else -1.0
    M, B, e = prob.M, prob.B, prob.eta
    out = np.empty(len(points))
    for idx, (k, j, i) in enumerate(points):
        terms = [(1.0, M[2][k], M[1][j], M[0][i]),
                 (sgn * e[0], M[2][k], M[1][j], B[0][i]),
                 (sgn * e[1], M[2][k], B[1][j], M[0][i]),
                 (sgn * e[2], B[2][k], M[1][j], M[0][i])]
        total = 0.0
        for c, rz, ry, rx in terms:
            kk, jj, ii = np.nonzero(rz)[0], np.nonzero(ry)[0], np.nonzero(rx)[0]
            blk = v[np.ix_(kk, jj, ii)]
            total += c * np.einsum("a,b,c,abc->", rz[kk], ry[jj], rx[ii], blk)
        out[idx] = total
    return out
