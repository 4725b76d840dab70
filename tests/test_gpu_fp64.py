"""GPU parity of the plain-FP64 path (TFDE_FP64) against the oracle, through
the C ABI.  Sizes span several 64-wide tiles with ragged tails, degenerate
1-point axes, and the full n = 256 size on sampled outputs."""
import math

import numpy as np
import pytest

from oracle import tfde_oracle as o
import tfde_inputs as inp
from gpu_helpers import relerr, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2511_21198_gb300 import build
    build.build()
    from paper_2511_21198_gb300 import tfde
    tfde.load()
    return tfde


class Case:
    def __init__(self, T, n, delta, kp, km, dt, prec=0):
        self.T = T
        self.params = T.make_params(n, delta, kp, km, dt)
        self.h = T.tfde_assemble(self.params, prec)
        self.o = o.Problem(n=n, delta=delta, kp=kp, km=km, dt=dt)

    def close(self):
        self.T.tfde_destroy(self.h)


CASES = [
    ((5, 6, 7), (0.3, 0.6, 0.8), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), 0.1),
    ((16, 16, 16), (0.5, 0.5, 0.5), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), 1 / 16),
    ((70, 9, 12), (0.7, 0.2, 0.9), (2.0, 0.5, 1.5), (0.5, 2.0, 1.0), 0.05),
    ((3, 67, 5), (0.4, 0.45, 0.6), (1.0, 1.0, 1.0), (0.5, 0.5, 0.5), 0.2),
    ((4, 5, 66), (0.9, 0.1, 0.5), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), 0.3),
    ((1, 1, 1), (0.5, 0.5, 0.5), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), 0.1),
    ((1, 9, 2), (0.2, 0.5, 0.8), (1.0, 2.0, 1.0), (1.5, 2.0, 0.5), 0.1),
    # n + 1 prime on every axis (101, 5, 31): the DST-I transform length has no small factor
    ((100, 4, 30), (0.35, 0.65, 0.95), (1.5, 1.0, 1.0), (0.7, 1.0, 2.0), 0.02),
    ((130, 3, 2), (0.6, 0.3, 0.5), (1.0,) * 3, (1.0,) * 3, 0.05),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])))
def test_matvec_and_precond_parity(T, case):
    c = Case(T, *case)
    try:
        v = inp.uniform_vector(c.o.shape, 21)
        x = to_dev(v)
        y = to_dev(np.zeros_like(v))
        T.tfde_matvec(c.h, T.TFDE_OP_A, x, y)
        assert relerr(to_host(y), o.apply_A(c.o, v)) < 1e-13
        T.tfde_matvec(c.h, T.TFDE_OP_RHS, x, y)
        assert relerr(to_host(y), o.rhs(c.o, v, None)) < 1e-13
        T.tfde_precond(c.h, x, y)
        tau = o.build_tau(c.o)
        assert relerr(to_host(y), o.apply_Pinv(tau, v)) < 1e-13
        # in-place preconditioner (z aliases r)
        T.tfde_precond(c.h, x, x)
        assert relerr(to_host(x), o.apply_Pinv(tau, v)) < 1e-13
        for a in range(3):
            q, lam, eta = T.tfde_coefficients(c.h, a, c.o.n[a])
            np.testing.assert_allclose(q, c.o.q[a], rtol=5e-15)
            assert eta == pytest.approx(c.o.eta[a], rel=1e-15)
    finally:
        c.close()


@pytest.mark.parametrize("sym", [True, False])
def test_solvers_match_dense_solution(T, sym):
    n = (12, 10, 14)
    c = Case(T, n, (0.3, 0.6, 0.8), (1.0, 1.5, 2.0), (1.0, 1.5, 2.0) if sym else (0.5, 1.0, 0.6), 0.2)
    try:
        b = inp.uniform_vector(c.o.shape, 31)
        xref = np.linalg.solve(o.dense_A(c.o), b.ravel()).reshape(c.o.shape)
        bd = to_dev(b)
        x = to_dev(np.zeros_like(b))
        if sym:
            info = T.tfde_pcg(c.h, bd, x, 1e-13, 500)
        else:
            info = T.tfde_pgmres(c.h, bd, x, 20, 1e-13, 500)
        assert info.relres <= 1e-13
        assert relerr(to_host(x), xref) < 1e-11
        # restarted GMRES with a short restart also converges
        if not sym:
            x2 = to_dev(np.zeros_like(b))
            info = T.tfde_pgmres(c.h, bd, x2, 3, 1e-12, 500)
            assert info.restarts > 1 and relerr(to_host(x2), xref) < 1e-10
    finally:
        c.close()


def test_source_term_matches_oracle(T):
    c = Case(T, (9, 7, 8), (0.3, 0.6, 0.8), (1.0, 2.0, 1.0), (0.5, 2.0, 1.5), 0.1)
    try:
        t = 0.35
        F = to_dev(np.zeros(c.o.shape))
        T.tfde_source_example2(c.h, math.cos(t + 1.0), -math.sin(t + 1.0), F)
        assert relerr(to_host(F), o.source_cell_average(c.o, t, "sin")) < 1e-13
    finally:
        c.close()


def _gpu_trajectory(T, c, M, tol, u0):
    u = to_dev(u0)
    un = to_dev(np.zeros_like(u0))
    F = to_dev(np.zeros_like(u0))
    iters = []
    for m in range(1, M + 1):
        th = (m - 0.5) * c.o.dt
        T.tfde_source_example2(c.h, -math.exp(-th), -math.exp(-th), F)
        info = T.tfde_cn_step(c.h, u, F, None, un, tol)
        assert info.relres <= tol
        iters.append(info.iters)
        u, un = un, u
    return to_host(u), iters


def test_cn_trajectory_n16_exp(T):
    """The 16^3 symmetric workload (delta = 0.5, k = 1, 16 steps, tol 1e-8)
    against the oracle running the same PCG from the same previous step."""
    n, M = 16, 16
    c = Case(T, (n, n, n), (0.5, 0.5, 0.5), (1.0,) * 3, (1.0,) * 3, 1.0 / M)
    try:
        u0 = o.exact_u(c.o, 0.0, "exp")
        ug, it_g = _gpu_trajectory(T, c, M, 1e-8, u0)
        r = o.cn_solve(c.o, u0, M, tol=1e-8, phi="exp")
        assert it_g == r.iters
        assert relerr(ug, r.u) < 1e-10
        ex = o.exact_u(c.o, 1.0, "exp")
        err_g = np.abs(ug - ex).max()
        assert err_g == pytest.approx(np.abs(r.u - ex).max(), rel=1e-6)   # same discretisation error
        assert err_g / np.abs(ex).max() < 0.03
    finally:
        c.close()


@pytest.mark.parametrize("n", [(20, 18, 16), (67, 11, 37)], ids=lambda n: "x".join(map(str, n)))
@pytest.mark.parametrize("sym", [True, False])
def test_cn_step_tight_parity(T, sym, n):
    """One step from the same u^{m-1}, both sides to a 1e-13 true residual:
    relative error <= 1e-12 (the all-FP64 parity gate).  The second grid is
    ragged against every tile of the fused mass stencil (64 x 8 x 32 points)
    and spans two of its z chunks."""
    c = Case(T, n, (0.3, 0.6, 0.8), (1.0,) * 3, (1.0,) * 3 if sym else (0.5,) * 3, 0.02)
    try:
        u0 = inp.smoothed_uniform(c.o.shape, 2)
        b = o.rhs(c.o, u0, None)
        tau = o.build_tau(c.o)
        A = lambda v: o.apply_A(c.o, v)
        Pi = lambda r: o.apply_Pinv(tau, r)
        if sym:
            xo, _ = o.pcg(A, Pi, b, u0, 1e-13, 1000)
        else:
            xo, _ = o.gmres_left(A, Pi, b, u0, 1e-13, 1000, 20, "true")
        un = to_dev(np.zeros_like(u0))
        info = T.tfde_cn_step(c.h, to_dev(u0), None, None, un, 1e-13)
        assert info.relres <= 1e-13
        assert relerr(to_host(un), xo) < 1e-12
    finally:
        c.close()


def test_argument_errors(T):
    c = Case(T, (6, 6, 6), (0.5,) * 3, (1.0,) * 3, (0.5,) * 3, 0.1)
    try:
        x = to_dev(np.ones(c.o.shape))
        y = to_dev(np.zeros(c.o.shape))
        host = np.zeros(c.o.shape)
        with pytest.raises(T.TfdeError) as e:
            T.tfde_matvec(c.h, T.TFDE_OP_A, host.ctypes.data, y)
        assert e.value.status == T.TFDE_EINVAL
        with pytest.raises(T.TfdeError) as e:
            T.tfde_pcg(c.h, x, y, 1e-8, 10)       # non-symmetric problem
        assert e.value.status == T.TFDE_EINVAL
        with pytest.raises(T.TfdeError) as e:
            T.tfde_pgmres(c.h, x, y, 20, -1.0, 10)
        assert e.value.status == T.TFDE_EINVAL
        with pytest.raises(T.TfdeError) as e:
            T.tfde_matvec(c.h, T.TFDE_OP_A, x, x)
        assert e.value.status == T.TFDE_EINVAL
        info = T.tfde_pgmres(c.h, x, y, 20, 1e-14, 2, check=False)
        assert info.status == T.TFDE_ENOCONV and info.iters == 2
        bad = T.make_params((4, 4, 4), (1.5, 0.5, 0.5), (1,) * 3, (1,) * 3, 0.1)
        with pytest.raises(T.TfdeError) as e:
            T.tfde_assemble(bad)
        assert e.value.status == T.TFDE_EINVAL
        # zero right-hand side gives x = 0 without iterating
        z = to_dev(np.zeros(c.o.shape))
        info = T.tfde_pgmres(c.h, z, x, 20, 1e-8, 10)
        assert info.iters == 0 and float(np.abs(to_host(x)).max()) == 0.0
    finally:
        c.close()


def test_full_size_matvec_sampled_and_precond_eigenvector(T):
    """n = 256 (the benchmark size), FP64 path: 64 sampled outputs of A v
    computed one by one by the oracle, and P^{-1} applied to a DST-I
    eigenvector (a separable sine product), which must return it divided by
    its eigenvalue Lambda(a, b, c)."""
    n = 256
    c = Case(T, (n, n, n), (0.7, 0.7, 0.7), (1.0,) * 3, (1.0,) * 3, 1.0 / 20)
    try:
        rng = np.random.default_rng(5)
        v = inp.smoothed_uniform(c.o.shape, 3)
        y = to_dev(np.zeros_like(v))
        T.tfde_matvec(c.h, T.TFDE_OP_A, to_dev(v), y)
        yh = to_host(y)
        pts = [tuple(int(t) for t in rng.integers(0, n, 3)) for _ in range(60)]
        pts += [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 128), (255, 0, 1)]
        ref = o.apply_A_at(c.o, v, pts)
        got = np.array([yh[p] for p in pts])
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(yh).max()
        a, b_, cc = 3, 200, 77
        S = [o.dst_matrix(n)[:, m] for m in (a, b_, cc)]   # columns = eigenvectors
        r = S[2][:, None, None] * S[1][None, :, None] * S[0][None, None, :]
        tau = o.build_tau(c.o)
        lam = tau.Lam[cc, b_, a]
        z = to_dev(np.zeros_like(r))
        T.tfde_precond(c.h, to_dev(r), z)
        assert relerr(to_host(z), r / lam) < 1e-12
    finally:
        c.close()


def test_stiffness_operator(T):
    """TFDE_OP_STIFF gives the three Kronecker stiffness terms of Eq. (linear_sys) alone."""
    c = Case(T, (9, 8, 7), (0.3, 0.6, 0.8), (1.0, 2.0, 0.5), (0.5, 2.0, 1.5), 0.1)
    try:
        v = inp.uniform_vector(c.o.shape, 71)
        y = to_dev(np.zeros_like(v))
        T.tfde_matvec(c.h, T.TFDE_OP_STIFF, to_dev(v), y)
        assert relerr(to_host(y), o.stiffness_terms(c.o, v)) < 1e-13
    finally:
        c.close()


@pytest.mark.parametrize("sym", [True, False])
def test_cn_advance_matches_cn_step(T, sym):
    """The chained in-place advance (A u^{m-1} = b^{m-1} - r^{m-1}) follows the
    same trajectory as independent CN steps; an intervening solver call or a
    different buffer breaks the chain and forces a full restart."""
    n, M = (12, 10, 8), 6
    c = Case(T, n, (0.4, 0.6, 0.8), (1.0,) * 3, (1.0,) * 3 if sym else (0.5, 0.7, 0.9), 1.0 / M)
    try:
        u0 = o.exact_u(c.o, 0.0, "exp")
        F = to_dev(np.zeros_like(u0))
        ua = to_dev(u0)
        us, un = to_dev(u0), to_dev(np.zeros_like(u0))
        for m in range(1, M + 1):
            th = (m - 0.5) * c.o.dt
            T.tfde_source_example2(c.h, -math.exp(-th), -math.exp(-th), F)
            ia = T.tfde_cn_advance(c.h, ua, F, m == 1, 1e-12)
            ib = T.tfde_cn_step(c.h, us, F, None, un, 1e-12)   # also invalidates the chain
            us, un = un, us
            assert ia.relres <= 1e-12 and ib.relres <= 1e-12
            assert relerr(to_host(ua), to_host(us)) < 1e-10
        # a stale chain (tfde_cn_step ran in between) must not be used: the
        # result still equals the oracle step
        th = (M + 0.5) * c.o.dt
        T.tfde_source_example2(c.h, -math.exp(-th), -math.exp(-th), F)
        ref = to_host(ua).copy()
        T.tfde_cn_advance(c.h, ua, F, False, 1e-12)
        b = o.rhs(c.o, ref, to_host(F))
        tau = o.build_tau(c.o)
        if sym:
            xo, _ = o.pcg(lambda v: o.apply_A(c.o, v), lambda r: o.apply_Pinv(tau, r), b, ref, 1e-14, 1000)
        else:
            xo, _ = o.gmres_left(lambda v: o.apply_A(c.o, v), lambda r: o.apply_Pinv(tau, r), b, ref, 1e-14, 1000,
                                 20, "true")
        assert relerr(to_host(ua), xo) < 1e-10
    finally:
        c.close()
