"""GPU parity of the mixed-precision path (TFDE_MIXED): the split-BF16
tcgen05 contractions against the oracle, and the FP64-refined solvers against
dense / oracle solutions.  Grid sizes are multiples of 8 (the TMA stride rule)
that span several 128-row / 256-line tiles with ragged tails."""
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


def round_bf16(a):
    """Round float64 values to the nearest BF16 (ties to even), via float32."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


SIZES = [
    ((16, 16, 16), (0.5, 0.5, 0.5), (1.0,) * 3, (1.0,) * 3, 1 / 16),
    ((64, 24, 40), (0.3, 0.6, 0.8), (1.0, 2.0, 1.5), (0.5, 2.0, 1.0), 0.05),
    ((136, 8, 16), (0.7, 0.2, 0.9), (1.0,) * 3, (1.0,) * 3, 0.1),
    ((8, 136, 24), (0.4, 0.9, 0.1), (2.0, 1.0, 0.5), (0.5, 1.0, 2.0), 0.2),
    ((24, 16, 264), (0.6, 0.5, 0.35), (1.0,) * 3, (1.0,) * 3, 0.02),
]


@pytest.mark.parametrize("case", SIZES, ids=lambda c: "x".join(map(str, c[0])))
def test_fast_matvec_and_precond(T, case):
    n, d, kp, km, dt = case
    h = T.tfde_assemble(T.make_params(n, d, kp, km, dt), T.TFDE_MIXED)
    try:
        op = o.Problem(n=n, delta=d, kp=kp, km=km, dt=dt)
        v = inp.uniform_vector(op.shape, 41)
        y = to_dev(np.zeros_like(v))
        T.tfde_matvec(h, T.TFDE_OP_A | T.TFDE_OP_FAST, to_dev(v), y)
        assert relerr(to_host(y), o.apply_A(op, v)) < 2e-4
        T.tfde_matvec(h, T.TFDE_OP_RHS | T.TFDE_OP_FAST, to_dev(v), y)
        assert relerr(to_host(y), o.rhs(op, v, None)) < 2e-4
        # accurate (non-fast) operator of a mixed problem is FP64-exact
        T.tfde_matvec(h, T.TFDE_OP_A, to_dev(v), y)
        assert relerr(to_host(y), o.apply_A(op, v)) < 1e-13
        T.tfde_matvec(h, T.TFDE_OP_RHS, to_dev(v), y)
        assert relerr(to_host(y), o.rhs(op, v, None)) < 1e-13
        T.tfde_matvec(h, T.TFDE_OP_STIFF, to_dev(v), y)
        assert relerr(to_host(y), o.stiffness_terms(op, v)) < 1e-13
        # preconditioner: exact tau inverse within the BF16 rounding of S_n ...
        T.tfde_precond(h, to_dev(v), y)
        z = to_host(y)
        tau = o.build_tau(op)
        assert relerr(z, o.apply_Pinv(tau, v)) < 3e-2
        # ... and tight against the same transform with S_n rounded to BF16
        Sb = [round_bf16(S) for S in tau.S]
        zb = o.apply_S_N(Sb, o.apply_S_N(Sb, v) / tau.Lam)
        assert relerr(z, zb) < 2e-4
    finally:
        T.tfde_destroy(h)


@pytest.mark.parametrize("n", [(16, 16, 16), (40, 32, 24)])
def test_mixed_pcg_matches_dense_solution(T, n):
    d, kp = (0.3, 0.6, 0.8), (1.0, 1.5, 2.0)
    h = T.tfde_assemble(T.make_params(n, d, kp, kp, 0.1), T.TFDE_MIXED)
    try:
        op = o.Problem(n=n, delta=d, kp=kp, km=kp, dt=0.1)
        b = inp.uniform_vector(op.shape, 51)
        tau = o.build_tau(op)
        xref, _ = o.pcg(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, np.zeros_like(b), 1e-14, 2000)
        x = to_dev(np.zeros_like(b))
        info = T.tfde_pcg(h, to_dev(b), x, 1e-12, 2000)
        assert info.relres <= 1e-12 and info.refine_sweeps >= 1 and info.fallback == 0
        assert relerr(to_host(x), xref) < 1e-10
    finally:
        T.tfde_destroy(h)


def test_mixed_pcg_long_inner_solves(T):
    """Inner solves longer than the ring of kept search directions (3): the
    solution of the inner PCG is combined from the directions and their
    step lengths, and a window that fills the ring is folded into the FP32
    accumulator before the oldest direction is overwritten.  A stiff, high
    order problem from x0 = 0 at a tight tolerance runs sweeps of four or
    more inner iterations; the result must still match the oracle's
    solution."""
    n, d, kp = (32, 24, 16), (0.9, 0.85, 0.95), (1.0, 2.0, 1.5)
    dt = 1.0
    h = T.tfde_assemble(T.make_params(n, d, kp, kp, dt), T.TFDE_MIXED)
    try:
        op = o.Problem(n=n, delta=d, kp=kp, km=kp, dt=dt)
        b = inp.uniform_vector(op.shape, 57)
        tau = o.build_tau(op)
        xref, _ = o.pcg(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, np.zeros_like(b), 1e-14, 4000)
        x = to_dev(np.zeros_like(b))
        info = T.tfde_pcg(h, to_dev(b), x, 1e-12, 4000)
        assert info.relres <= 1e-12 and info.fallback == 0
        # at least one sweep ran more inner iterations than the ring holds
        assert info.iters > 3 * info.refine_sweeps, (info.iters, info.refine_sweeps)
        assert relerr(to_host(x), xref) < 1e-10
    finally:
        T.tfde_destroy(h)


def test_mixed_cn_step_tight_parity(T):
    """One CN step from the same u^{m-1}: mixed solve to a 1e-12 true residual
    matches the oracle's 1e-14 PCG solution to <= 1e-10 relative error."""
    n = (32, 24, 16)
    d, k = (0.7, 0.7, 0.7), (1.0,) * 3
    h = T.tfde_assemble(T.make_params(n, d, k, k, 0.05), T.TFDE_MIXED)
    try:
        op = o.Problem(n=n, delta=d, kp=k, km=k, dt=0.05)
        u0 = inp.smoothed_uniform(op.shape, 2)
        F = o.source_cell_average(op, 0.025, "exp")
        b = o.rhs(op, u0, F)
        tau = o.build_tau(op)
        xo, _ = o.pcg(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, u0, 1e-14, 2000)
        un = to_dev(np.zeros_like(u0))
        info = T.tfde_cn_step(h, to_dev(u0), to_dev(F), None, un, 1e-12)
        assert info.relres <= 1e-12
        assert relerr(to_host(un), xo) < 1e-10
    finally:
        T.tfde_destroy(h)


def test_mixed_trajectory_n16(T):
    """16^3 symmetric workload, 16 steps at tol 1e-8: every step meets the
    true residual, and the final error against the manufactured solution
    equals the oracle's."""
    n, M = 16, 16
    d, k = (0.5,) * 3, (1.0,) * 3
    h = T.tfde_assemble(T.make_params((n,) * 3, d, k, k, 1.0 / M), T.TFDE_MIXED)
    try:
        op = o.Problem(n=(n,) * 3, delta=d, kp=k, km=k, dt=1.0 / M)
        u = to_dev(o.exact_u(op, 0.0, "exp"))
        un = to_dev(np.zeros(op.shape))
        F = to_dev(np.zeros(op.shape))
        for m in range(1, M + 1):
            th = (m - 0.5) * op.dt
            T.tfde_source_example2(h, -math.exp(-th), -math.exp(-th), F)
            info = T.tfde_cn_step(h, u, F, None, un, 1e-8)
            assert info.relres <= 1e-8
            u, un = un, u
        r = o.cn_solve(op, o.exact_u(op, 0.0, "exp"), M, tol=1e-12, phi="exp")
        assert relerr(to_host(u), r.u) < 1e-6
    finally:
        T.tfde_destroy(h)


def test_accurate_apply_wide_dynamic_range(T):
    """Lines whose entries span many orders of magnitude: the exact-integer
    slice contraction (49-bit fixed point under each row and line maximum) is
    accurate to the FP64 level in norm, relative to |A| |v|."""
    n = (32, 24, 40)
    d, kp, km = (0.35, 0.65, 0.9), (1.0, 2.0, 1.0), (0.5, 1.0, 2.0)
    h = T.tfde_assemble(T.make_params(n, d, kp, km, 0.3), T.TFDE_MIXED)
    try:
        op = o.Problem(n=n, delta=d, kp=kp, km=km, dt=0.3)
        rng = np.random.default_rng(81)
        v = inp.uniform_vector(op.shape, 82) * 10.0 ** rng.uniform(-12, 3, size=op.shape)
        y = to_dev(np.zeros_like(v))
        T.tfde_matvec(h, T.TFDE_OP_A, to_dev(v), y)
        ref = o.apply_A(op, v)
        # |A| |v| elementwise: the same Kronecker terms with absolute-valued factors
        absop = o.Problem(n=n, delta=d, kp=kp, km=km, dt=0.3)
        absop.B = [np.abs(B) for B in absop.B]
        absAv = o.apply_A(absop, np.abs(v))
        assert np.abs(to_host(y) - ref).max() <= 1e-13 * absAv.max()
    finally:
        T.tfde_destroy(h)


def test_mixed_cn_advance_trajectory(T):
    """Chained mixed-precision advance over 8 steps equals FP64 steps at a tight residual."""
    n, M = (24, 16, 32), 8
    d, k = (0.6, 0.7, 0.8), (1.0,) * 3
    hm = T.tfde_assemble(T.make_params(n, d, k, k, 1.0 / M), T.TFDE_MIXED)
    hf = T.tfde_assemble(T.make_params(n, d, k, k, 1.0 / M), T.TFDE_FP64)
    try:
        op = o.Problem(n=n, delta=d, kp=k, km=k, dt=1.0 / M)
        u0 = o.exact_u(op, 0.0, "exp")
        F = to_dev(np.zeros_like(u0))
        um, uf = to_dev(u0), to_dev(u0)
        for m in range(1, M + 1):
            th = (m - 0.5) * op.dt
            T.tfde_source_example2(hm, -math.exp(-th), -math.exp(-th), F)
            im = T.tfde_cn_advance(hm, um, F, m == 1, 1e-12)
            T.tfde_cn_advance(hf, uf, F, m == 1, 1e-13)
            assert im.relres <= 1e-12
        assert relerr(to_host(um), to_host(uf)) < 1e-10
    finally:
        T.tfde_destroy(hm)
        T.tfde_destroy(hf)


@pytest.mark.parametrize("n,restart", [((16, 16, 16), 20), ((40, 32, 24), 20), ((64, 24, 40), 4)])
def test_mixed_pgmres_matches_dense_solution(T, n, restart):
    """Non-symmetric system: FP32 inner GMRES cycles inside FP64 refinement
    reach a 1e-12 true residual without falling back to FP64 cycles, and agree
    with the oracle's GMRES solution driven to 1e-14."""
    d, kp, km = (0.3, 0.6, 0.8), (1.0, 1.5, 2.0), (0.5, 2.0, 1.0)
    h = T.tfde_assemble(T.make_params(n, d, kp, km, 0.1), T.TFDE_MIXED)
    try:
        op = o.Problem(n=n, delta=d, kp=kp, km=km, dt=0.1)
        b = inp.uniform_vector(op.shape, 52)
        tau = o.build_tau(op)
        xref, _ = o.gmres_left(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, np.zeros_like(b),
                               1e-14, 4000, restart=20, criterion="true")
        x = to_dev(np.zeros_like(b))
        info = T.tfde_pgmres(h, to_dev(b), x, restart, 1e-12, 2000)
        assert info.relres <= 1e-12 and info.fallback == 0
        assert info.refine_sweeps >= 1 and info.restarts == info.refine_sweeps
        assert relerr(to_host(x), xref) < 1e-10
    finally:
        T.tfde_destroy(h)


def test_mixed_cn_step_nonsymmetric_tight_parity(T):
    """One non-symmetric CN step (PGMRES) from the same u^{m-1}, mixed path at a
    1e-12 true residual against the oracle's 1e-14 GMRES solution."""
    n = (32, 24, 48)
    d, kp, km = (0.3, 0.6, 0.8), (1.0,) * 3, (0.5,) * 3
    h = T.tfde_assemble(T.make_params(n, d, kp, km, 0.02), T.TFDE_MIXED)
    try:
        op = o.Problem(n=n, delta=d, kp=kp, km=km, dt=0.02)
        u0 = inp.smoothed_uniform(op.shape, 2)
        b = o.rhs(op, u0, None)
        tau = o.build_tau(op)
        xo, _ = o.gmres_left(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, u0, 1e-14, 4000,
                             restart=20, criterion="true")
        un = to_dev(np.zeros_like(u0))
        info = T.tfde_cn_step(h, to_dev(u0), None, None, un, 1e-12)
        assert info.relres <= 1e-12 and info.fallback == 0 and info.restarts >= 1
        assert relerr(to_host(un), xo) < 1e-10
    finally:
        T.tfde_destroy(h)


def test_mixed_nonsymmetric_advance_matches_fp64(T):
    """Chained non-symmetric advance (f = 0, smoothed noise u0) over 6 steps:
    mixed PGMRES equals the all-FP64 PGMRES path at tight residuals."""
    n, M = (48, 40, 32), 6
    d, kp, km = (0.3, 0.6, 0.8), (1.0,) * 3, (0.5,) * 3
    hm = T.tfde_assemble(T.make_params(n, d, kp, km, 1.0 / M), T.TFDE_MIXED)
    hf = T.tfde_assemble(T.make_params(n, d, kp, km, 1.0 / M), T.TFDE_FP64)
    try:
        u0 = inp.smoothed_uniform(tuple(reversed(n)), 2)
        um, uf = to_dev(u0), to_dev(u0)
        for m in range(1, M + 1):
            im = T.tfde_cn_advance(hm, um, None, m == 1, 1e-12)
            T.tfde_cn_advance(hf, uf, None, m == 1, 1e-13)
            assert im.relres <= 1e-12 and im.fallback == 0
        assert relerr(to_host(um), to_host(uf)) < 1e-10
    finally:
        T.tfde_destroy(hm)
        T.tfde_destroy(hf)


def test_mixed_beyond_exact_accumulation_takes_the_fft_passes(T):
    """n_a = 456 > 448 (where the exact-slice residual's FP32 sums would pass
    2^24): TFDE_MIXED runs on the FFT passes instead, and the batched solver,
    whose grouped launches are the tensor-core contraction's, refuses it."""
    prm = T.make_params((456, 8, 8), (0.5,) * 3, (1.0,) * 3, (1.0,) * 3, 0.1)
    h = T.tfde_assemble(prm, T.TFDE_MIXED)
    try:
        op = o.Problem(n=(456, 8, 8), delta=(0.5,) * 3, kp=(1.0,) * 3, km=(1.0,) * 3, dt=0.1)
        v = inp.uniform_vector(op.shape, 62)
        y = to_dev(np.zeros_like(v))
        T.tfde_matvec(h, T.TFDE_OP_A, to_dev(v), y)
        assert relerr(to_host(y), o.apply_A(op, v)) < 1e-13
    finally:
        T.tfde_destroy(h)
    with pytest.raises(T.TfdeError) as e:
        T.tfde_batch_create([prm], 20)
    assert e.value.status == T.TFDE_EUNSUPPORTED


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_extrapolated_guess_same_solution_fewer_iterations(T, prec):
    """Chained advance with the order-2 extrapolated initial guess reaches the
    same trajectory (tight residuals) as the previous-step guess, with fewer
    inner iterations once the history is built."""
    n, M = (32, 24, 40), 10
    d, k = (0.7, 0.7, 0.7), (1.0,) * 3
    p = T.TFDE_MIXED if prec == "mixed" else T.TFDE_FP64
    h0 = T.tfde_assemble(T.make_params(n, d, k, k, 1.0 / M), p)
    h2 = T.tfde_assemble(T.make_params(n, d, k, k, 1.0 / M), p)
    T.tfde_set_guess_order(h2, 2)
    try:
        op = o.Problem(n=n, delta=d, kp=k, km=k, dt=1.0 / M)
        u0 = o.exact_u(op, 0.0, "exp")
        F = to_dev(np.zeros_like(u0))
        ua, ub = to_dev(u0), to_dev(u0)
        it0 = it2 = 0
        for m in range(1, M + 1):
            th = (m - 0.5) * op.dt
            T.tfde_source_example2(h0, -math.exp(-th), -math.exp(-th), F)
            ia = T.tfde_cn_advance(h0, ua, F, m == 1, 1e-12)
            ib = T.tfde_cn_advance(h2, ub, F, m == 1, 1e-12)
            assert ia.relres <= 1e-12 and ib.relres <= 1e-12
            if m > 3:
                it0 += ia.iters
                it2 += ib.iters
        assert relerr(to_host(ua), to_host(ub)) < 1e-10
        assert it2 < it0
    finally:
        T.tfde_destroy(h0)
        T.tfde_destroy(h2)


def test_guess_order_rejects_bad_values(T):
    h = T.tfde_assemble(T.make_params((16, 16, 16), (0.5,) * 3, (1.0,) * 3, (1.0,) * 3, 0.1), T.TFDE_MIXED)
    try:
        for bad in (-1, 4):
            with pytest.raises(T.TfdeError):
                T.tfde_set_guess_order(h, bad)
        T.tfde_set_guess_order(h, 3)
    finally:
        T.tfde_destroy(h)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_mr_corrected_guess_same_solution_fewer_iterations(T, prec):
    """Order 3 (the order-2 extrapolation with its minimal-residual
    correction over the stored A u) reaches the trajectory of the order-2
    guess at tol 1e-8, within the tolerance, with no more inner iterations
    and no more refinement sweeps once the history is built, and strictly
    fewer iterations over the run."""
    n, M = (48, 40, 32), 12
    d, k = (0.7, 0.7, 0.7), (1.0,) * 3
    p = T.TFDE_MIXED if prec == "mixed" else T.TFDE_FP64
    h2 = T.tfde_assemble(T.make_params(n, d, k, k, 0.05), p)
    h3 = T.tfde_assemble(T.make_params(n, d, k, k, 0.05), p)
    T.tfde_set_guess_order(h2, 2)
    T.tfde_set_guess_order(h3, 3)
    try:
        op = o.Problem(n=n, delta=d, kp=k, km=k, dt=0.05)
        u0 = o.exact_u(op, 0.0, "exp")
        F = to_dev(np.zeros_like(u0))
        ua, ub = to_dev(u0), to_dev(u0)
        it2 = it3 = sw2 = sw3 = 0
        for m in range(1, M + 1):
            th = (m - 0.5) * op.dt
            T.tfde_source_example2(h2, -math.exp(-th), -math.exp(-th), F)
            ia = T.tfde_cn_advance(h2, ua, F, m == 1, 1e-8)
            ib = T.tfde_cn_advance(h3, ub, F, m == 1, 1e-8)
            assert ia.relres <= 1e-8 and ib.relres <= 1e-8
            if m > 3:
                it2 += ia.iters
                it3 += ib.iters
                sw2 += ia.refine_sweeps
                sw3 += ib.refine_sweeps
        # both trajectories meet a 1e-8 relative residual at every step (the
        # honest FP64 residual); their difference is bounded by that, not by
        # the guess
        assert relerr(to_host(ua), to_host(ub)) < 1e-5
        assert it3 < it2 and sw3 <= sw2
    finally:
        T.tfde_destroy(h2)
        T.tfde_destroy(h3)


def test_mr_corrected_guess_nonsymmetric(T):
    """The correction minimises the residual norm, so it also serves the
    non-symmetric (PGMRES) path: order 3 against the previous-step guess on a
    chained non-symmetric run, same trajectory at tight residuals."""
    n, M = (32, 24, 40), 8
    d, kp, km = (0.3, 0.6, 0.8), (1.0,) * 3, (0.5,) * 3
    h0 = T.tfde_assemble(T.make_params(n, d, kp, km, 0.02), T.TFDE_MIXED)
    h3 = T.tfde_assemble(T.make_params(n, d, kp, km, 0.02), T.TFDE_MIXED)
    T.tfde_set_guess_order(h3, 3)
    try:
        u0 = inp.smoothed_uniform(tuple(reversed(n)), 5)
        ua, ub = to_dev(u0), to_dev(u0)
        for m in range(1, M + 1):
            ia = T.tfde_cn_advance(h0, ua, None, m == 1, 1e-12)
            ib = T.tfde_cn_advance(h3, ub, None, m == 1, 1e-12)
            assert ia.relres <= 1e-12 and ib.relres <= 1e-12
        assert relerr(to_host(ua), to_host(ub)) < 1e-10
    finally:
        T.tfde_destroy(h0)
        T.tfde_destroy(h3)


@pytest.mark.parametrize("nonsym", [False, True])
def test_six_slice_residual_is_honest(T, nonsym):
    """At tol >= 1e-9 the refinement residual uses 6 digit slices (42 bits).
    The residual the library reports must agree with the oracle's FP64
    residual of the returned solution, and that residual must meet tol."""
    n = (48, 32, 40)
    d = (0.3, 0.6, 0.8)
    kp, km = ((1.0,) * 3, (0.5,) * 3) if nonsym else ((1.0,) * 3, (1.0,) * 3)
    h = T.tfde_assemble(T.make_params(n, d, kp, km, 0.05), T.TFDE_MIXED)
    try:
        op = o.Problem(n=n, delta=d, kp=kp, km=km, dt=0.05)
        b = inp.uniform_vector(op.shape, 61)
        x = to_dev(np.zeros_like(b))
        solve = T.tfde_pgmres if nonsym else T.tfde_pcg
        info = solve(h, to_dev(b), x, 20, 1e-8, 2000) if nonsym else solve(h, to_dev(b), x, 1e-8, 2000)
        xr = to_host(x)
        true_rel = np.linalg.norm(b - o.apply_A(op, xr)) / np.linalg.norm(b)
        assert true_rel <= 1e-8
        assert abs(true_rel - info.relres) <= 1e-11
    finally:
        T.tfde_destroy(h)


def test_device_loop_matches_host_loop(T):
    """The inner PCG's device-side loop (Sec. 3.1 iterations as one graph
    launch per refinement sweep, stop test on the device) runs the same
    kernels in the same order as the host-driven loop: the same iteration
    counts and the same CN steps, at a tight tolerance that takes several
    sweeps and more than one window of the direction ring."""
    import torch
    n = (32, 24, 16)
    d, k, dt = (0.7, 0.7, 0.7), (1.0,) * 3, 0.05
    prm = T.make_params(n, d, k, k, dt)
    ha = T.tfde_assemble(prm, T.TFDE_MIXED)
    hb = T.tfde_assemble(prm, T.TFDE_MIXED)
    try:
        T.tfde_set_device_loop(hb, False)
        u0 = inp.smoothed_uniform(tuple(reversed(n)), 7)
        ua, ub = to_dev(u0), to_dev(u0)
        Fa, Fb = torch.empty_like(ua), torch.empty_like(ub)
        for m in range(3):
            e = math.exp(-(m + 0.5) * dt)
            T.tfde_source_example2(ha, -e, -e, Fa)
            T.tfde_source_example2(hb, -e, -e, Fb)
            ia = T.tfde_cn_advance(ha, ua, Fa, m == 0, 1e-12)
            ib = T.tfde_cn_advance(hb, ub, Fb, m == 0, 1e-12)
            assert ia.iters == ib.iters and ia.refine_sweeps == ib.refine_sweeps
            assert ia.iters > 3 and ia.relres <= 1e-12
            assert relerr(to_host(ua), to_host(ub)) < 1e-14
    finally:
        T.tfde_destroy(ha)
        T.tfde_destroy(hb)


@pytest.mark.parametrize("restart", [20, 4])
def test_gmres_device_loop_matches_host_loop(T, restart):
    """The inner GMRES cycle's device-side loop (Arnoldi steps, Givens
    rotations, stop test and the small triangular solve on the device; Sec.
    3.2) against the host-driven cycle: the same steps and solution, including
    restarts (restart 4) and a tight tolerance."""
    n = (32, 24, 48)
    d, kp, km, dt = (0.3, 0.6, 0.8), (1.0,) * 3, (0.5,) * 3, 0.02
    prm = T.make_params(n, d, kp, km, dt)
    ha = T.tfde_assemble(prm, T.TFDE_MIXED)
    hb = T.tfde_assemble(prm, T.TFDE_MIXED)
    try:
        T.tfde_set_device_loop(hb, False)
        op = o.Problem(n=n, delta=d, kp=kp, km=km, dt=dt)
        u0 = inp.smoothed_uniform(op.shape, 2)
        b = o.rhs(op, u0, None)
        xa, xb = to_dev(u0), to_dev(u0)
        ia = T.tfde_pgmres(ha, to_dev(b), xa, restart, 1e-12, 4000)
        ib = T.tfde_pgmres(hb, to_dev(b), xb, restart, 1e-12, 4000)
        assert ia.iters == ib.iters and ia.restarts == ib.restarts and ia.relres <= 1e-12
        assert relerr(to_host(xa), to_host(xb)) < 1e-13
        tau = o.build_tau(op)
        xo, _ = o.gmres_left(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, u0, 1e-14, 4000,
                             restart=20, criterion="true")
        assert relerr(to_host(xa), xo) < 1e-10
    finally:
        T.tfde_destroy(ha)
        T.tfde_destroy(hb)
