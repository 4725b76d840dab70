"""GPU parity of TFDE_MIXED on the FFT passes: grids the tensor-core
contraction does not take (an n_a that is not a multiple of 8, n_a > 448,
the 2-D problem) run FP32 inner PCG / GMRES on the FFT-embedded Toeplitz
products and the FFT DST-I, inside FP64 refinement whose residual uses the
FP64 FFT passes.  Everything is checked against the oracle: the FP32 fast
operator and preconditioner to the FP32 rounding level, solutions of the
refined solvers to the oracle's tight PCG / GMRES solutions, a CN trajectory
to the oracle's CN solve, and a grid with n_1 = 480 > 448 (several FFT
lengths: 1024 for the Toeplitz embedding, 2048 for the Bluestein DST of
order 481)."""
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


# ragged grids: n_a not multiples of 8, n + 1 prime on some axes (DST of prime order)
CASES = [
    ((30, 21, 37), (0.3, 0.6, 0.8), (1.0, 2.0, 1.5), (0.5, 2.0, 1.0), 0.05),
    ((12, 16, 16), (0.5,) * 3, (1.0,) * 3, (1.0,) * 3, 0.1),
    ((480, 12, 10), (0.7, 0.4, 0.6), (1.0,) * 3, (1.0,) * 3, 0.05),
]


@pytest.mark.parametrize("case", CASES)
def test_fft_mixed_operators_match_oracle(T, case):
    n, d, kp, km, dt = case
    h = T.tfde_assemble(T.make_params(n, d, kp, km, dt), T.TFDE_MIXED)
    try:
        op = o.Problem(n=n, delta=d, kp=kp, km=km, dt=dt)
        v = inp.uniform_vector(op.shape, 61)
        y = to_dev(np.zeros_like(v))
        # the accurate operator: FP64 FFT passes
        T.tfde_matvec(h, T.TFDE_OP_A, to_dev(v), y)
        assert relerr(to_host(y), o.apply_A(op, v)) < 1e-13
        T.tfde_matvec(h, T.TFDE_OP_RHS, to_dev(v), y)
        assert relerr(to_host(y), o.rhs(op, v, None)) < 1e-13
        # the inner (FP32 FFT) operator and preconditioner: FP32 rounding of
        # the input (2^-24) plus log2(L) butterfly levels of FP32 rounding
        T.tfde_matvec(h, T.TFDE_OP_A | T.TFDE_OP_FAST, to_dev(v), y)
        assert relerr(to_host(y), o.apply_A(op, v)) < 5e-6
        T.tfde_precond(h, to_dev(v), y)
        assert relerr(to_host(y), o.apply_Pinv(o.build_tau(op), v)) < 5e-6
    finally:
        T.tfde_destroy(h)


@pytest.mark.parametrize("case", [((30, 21, 37), (0.3, 0.6, 0.8), (1.0, 1.5, 2.0), (1.0, 1.5, 2.0), 0.1),
                                  ((480, 12, 10), (0.7, 0.4, 0.6), (1.0,) * 3, (1.0,) * 3, 0.05)])
def test_fft_mixed_pcg_matches_oracle(T, case):
    n, d, kp, km, dt = case
    h = T.tfde_assemble(T.make_params(n, d, kp, km, dt), T.TFDE_MIXED)
    try:
        op = o.Problem(n=n, delta=d, kp=kp, km=km, dt=dt)
        b = inp.uniform_vector(op.shape, 52)
        tau = o.build_tau(op)
        xref, _ = o.pcg(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, np.zeros_like(b), 1e-14, 2000)
        x = to_dev(np.zeros_like(b))
        info = T.tfde_pcg(h, to_dev(b), x, 1e-12, 2000)
        assert info.relres <= 1e-12 and info.refine_sweeps >= 1 and info.fallback == 0
        assert relerr(to_host(x), xref) < 1e-10
        # the reported residual is the oracle's residual of the returned x
        xh = to_host(x)
        assert abs(np.linalg.norm(b - o.apply_A(op, xh)) / np.linalg.norm(b) - info.relres) < 1e-13
    finally:
        T.tfde_destroy(h)


@pytest.mark.parametrize("restart", [20, 4])
def test_fft_mixed_pgmres_matches_oracle(T, restart):
    n, d, kp, km, dt = CASES[0]
    h = T.tfde_assemble(T.make_params(n, d, kp, km, dt), T.TFDE_MIXED)
    try:
        op = o.Problem(n=n, delta=d, kp=kp, km=km, dt=dt)
        b = inp.uniform_vector(op.shape, 53)
        tau = o.build_tau(op)
        xref, _ = o.gmres_left(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, np.zeros_like(b),
                               1e-14, 4000, restart=20, criterion="true")
        x = to_dev(np.zeros_like(b))
        info = T.tfde_pgmres(h, to_dev(b), x, restart, 1e-12, 4000)
        assert info.relres <= 1e-12 and info.fallback == 0
        assert relerr(to_host(x), xref) < 1e-10
    finally:
        T.tfde_destroy(h)


def test_fft_mixed_cn_trajectory_matches_oracle(T):
    """Chained CN advance on a ragged non-symmetric grid, 8 steps at a tight
    residual: equal to the oracle's CN solve and to the FP64 path."""
    n, M = (26, 18, 22), 8
    d, kp, km = (0.6, 0.7, 0.8), (1.0, 2.0, 1.0), (2.0, 1.0, 1.0)
    hm = T.tfde_assemble(T.make_params(n, d, kp, km, 1.0 / M), T.TFDE_MIXED)
    hf = T.tfde_assemble(T.make_params(n, d, kp, km, 1.0 / M), T.TFDE_FP64)
    try:
        op = o.Problem(n=n, delta=d, kp=kp, km=km, dt=1.0 / M)
        u0 = o.exact_u(op, 0.0, "exp")
        res = []
        for h in (hm, hf):
            u = to_dev(u0)
            un = to_dev(np.zeros_like(u0))
            F = to_dev(np.zeros_like(u0))
            for m in range(1, M + 1):
                th = (m - 0.5) * op.dt
                T.tfde_source_example2(h, -math.exp(-th), -math.exp(-th), F)
                info = T.tfde_cn_step(h, u, F, None, un, 1e-12)
                assert info.relres <= 1e-12
                u, un = un, u
            res.append(to_host(u))
        r = o.cn_solve(op, u0, M, tol=1e-13, phi="exp")
        assert relerr(res[0], r.u) < 1e-9
        assert relerr(res[0], res[1]) < 1e-9
    finally:
        T.tfde_destroy(hm)
        T.tfde_destroy(hf)


def test_fft_mixed_2d_matches_fp64(T):
    """The 2-D problem (Example 1) with TFDE_MIXED: PCG and PGMRES solutions
    equal the oracle's 2-D solutions."""
    for kp, km in (((1.0, 1.0), (1.0, 1.0)), ((2.0, 0.5), (1.0, 3.0))):
        n, d, dt = (45, 38), (0.4, 0.7), 0.1
        prm = T.make_params((n[0], n[1], 0), (d[0], d[1], 0.5), (kp[0], kp[1], 1.0), (km[0], km[1], 1.0), dt)
        h = T.tfde_assemble(prm, T.TFDE_MIXED)
        try:
            op = o.Problem(n=(n[0], n[1], 1), delta=(d[0], d[1], 0.5), kp=(kp[0], kp[1], 1.0),
                           km=(km[0], km[1], 1.0), dt=dt, dim=2)
            b = inp.uniform_vector(op.shape, 54)
            tau = o.build_tau(op)
            A = lambda v: o.apply_A(op, v)
            Mi = lambda r: o.apply_Pinv(tau, r)
            x = to_dev(np.zeros_like(b))
            if kp == km:
                xref, _ = o.pcg(A, Mi, b, np.zeros_like(b), 1e-14, 2000)
                info = T.tfde_pcg(h, to_dev(b), x, 1e-12, 2000)
            else:
                xref, _ = o.gmres_left(A, Mi, b, np.zeros_like(b), 1e-14, 4000, restart=20, criterion="true")
                info = T.tfde_pgmres(h, to_dev(b), x, 20, 1e-12, 4000)
            assert info.relres <= 1e-12 and info.fallback == 0
            assert relerr(to_host(x), xref) < 1e-10
        finally:
            T.tfde_destroy(h)


def test_fft_mixed_rejects_grids_beyond_the_fft(T):
    with pytest.raises(T.TfdeError) as e:
        T.tfde_assemble(T.make_params((2056, 8, 8), (0.5,) * 3, (1.0,) * 3, (1.0,) * 3, 0.1), T.TFDE_MIXED)
    assert e.value.status == T.TFDE_EUNSUPPORTED
