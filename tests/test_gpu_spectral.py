"""The inner solves in the sine-transform eigenbasis (tfde_set_spectral_inner).

S_N is symmetric and orthogonal and diagonalises the tau preconditioner and
the mass operator (Eq. (diag_tau_pre); the mass matrices are tridiagonal
Toeplitz), so PCG with P on A c = r is PCG with the diagonal Lambda on
S_N A S_N (Sec. 3.1), and left-preconditioned GMRES likewise (Sec. 3.2): the
same iterates in exact arithmetic.  The refined solutions of both bases must
match the oracle's, with the same iteration counts up to rounding, and the
eigenbasis must run three tensor-core passes per inner iteration (plus two
sine transforms of three passes per refinement sweep)."""
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


CASES = [
    ((40, 32, 24), (0.3, 0.6, 0.8), (1.0, 1.5, 2.0), 0.1),
    ((64, 24, 136), (0.7, 0.2, 0.9), (2.0, 1.0, 0.5), 0.05),   # ragged 128-row / 256-line tiles
    ((16, 16, 16), (0.5, 0.5, 0.5), (1.0, 1.0, 1.0), 1 / 16),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])))
def test_eigenbasis_and_grid_basis_pcg_match_oracle(T, case):
    n, d, kp, dt = case
    op = o.Problem(n=n, delta=d, kp=kp, km=kp, dt=dt)
    b = inp.uniform_vector(op.shape, 71)
    tau = o.build_tau(op)
    xref, _ = o.pcg(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, np.zeros_like(b), 1e-14, 4000)
    iters = {}
    for spectral in (True, False):
        h = T.tfde_assemble(T.make_params(n, d, kp, kp, dt), T.TFDE_MIXED)
        try:
            T.tfde_set_spectral_inner(h, spectral)
            x = to_dev(np.zeros_like(b))
            info = T.tfde_pcg(h, to_dev(b), x, 1e-12, 4000)
            assert info.relres <= 1e-12 and info.fallback == 0, (spectral, info.relres, info.fallback)
            assert relerr(to_host(x), xref) < 1e-10
            iters[spectral] = (info.iters, info.refine_sweeps)
        finally:
            T.tfde_destroy(h)
    # the same Krylov method: iteration counts agree up to rounding effects
    assert abs(iters[True][0] - iters[False][0]) <= max(2, iters[False][0] // 5), iters


def test_eigenbasis_schedule_three_passes_per_iteration(T):
    """Host-driven loop (every tensor-core launch timed): the split launches of
    one solve are 3 per inner iteration and 6 per refinement sweep (the
    residual into the eigenbasis and the correction back)."""
    n, d, kp, dt = (48, 40, 32), (0.4, 0.5, 0.6), (1.0, 1.0, 1.0), 0.05
    op = o.Problem(n=n, delta=d, kp=kp, km=kp, dt=dt)
    b = inp.uniform_vector(op.shape, 72)
    h = T.tfde_assemble(T.make_params(n, d, kp, kp, dt), T.TFDE_MIXED)
    try:
        T.tfde_set_spectral_inner(h, True)
        T.tfde_stats_reset(time_tc=True)
        x = to_dev(np.zeros_like(b))
        info = T.tfde_pcg(h, to_dev(b), x, 1e-9, 4000)
        st = T.tfde_stats_get()
        T.tfde_stats_reset(time_tc=False)
        assert info.relres <= 1e-9 and info.fallback == 0
        ks = st.kind[T.TFDE_KIND_SPLIT]
        assert ks.launches == 3 * info.iters + 6 * info.refine_sweeps, (ks.launches, info.iters, info.refine_sweeps)
        assert ks.timed == ks.launches and ks.ms > 0
    finally:
        T.tfde_destroy(h)


def test_device_loop_and_host_loop_agree(T):
    """The eigenbasis iterations as one graph launch per sweep (device-side
    stop test) and driven from the host give the same iteration counts and
    solutions (up to the order of the inner products' atomic sums)."""
    n, d, kp, dt = (32, 24, 40), (0.6, 0.5, 0.35), (1.0, 1.0, 1.0), 0.02
    op = o.Problem(n=n, delta=d, kp=kp, km=kp, dt=dt)
    b = inp.uniform_vector(op.shape, 73)
    out = {}
    for dev_loop in (True, False):
        h = T.tfde_assemble(T.make_params(n, d, kp, kp, dt), T.TFDE_MIXED)
        try:
            T.tfde_set_spectral_inner(h, True)
            T.tfde_set_device_loop(h, dev_loop)
            x = to_dev(np.zeros_like(b))
            info = T.tfde_pcg(h, to_dev(b), x, 1e-11, 4000)
            assert info.relres <= 1e-11
            out[dev_loop] = (info.iters, to_host(x))
            launches = T.tfde_device_loop_launches(h)
            assert (launches == info.refine_sweeps) if dev_loop else (launches == 0), (dev_loop, launches)
        finally:
            T.tfde_destroy(h)
    assert out[True][0] == out[False][0]
    assert relerr(out[True][1], out[False][1]) < 1e-10


def test_chained_cn_steps_in_the_eigenbasis_match_oracle(T):
    """Four chained CN steps with the extrapolated guess (order 3) in the
    eigenbasis: each step's solution at a 1e-12 residual against the oracle's
    step from the same u^{m-1}."""
    n, d, kp, dt = (24, 32, 40), (0.7, 0.7, 0.7), (1.0, 1.0, 1.0), 0.05
    op = o.Problem(n=n, delta=d, kp=kp, km=kp, dt=dt)
    h = T.tfde_assemble(T.make_params(n, d, kp, kp, dt), T.TFDE_MIXED)
    try:
        T.tfde_set_spectral_inner(h, True)
        T.tfde_set_guess_order(h, 3)
        u = o.exact_u(op, 0.0, "exp")
        ud = to_dev(u)
        tau = o.build_tau(op)
        for m in range(1, 5):
            th = (m - 0.5) * dt
            F = to_dev(np.zeros_like(u))
            T.tfde_source_example2(h, -math.exp(-th), -math.exp(-th), F)
            u_prev = to_host(ud)
            b = o.rhs(op, u_prev, to_host(F))
            uref, _ = o.pcg(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, u_prev.copy(), 1e-14,
                            4000)
            info = T.tfde_cn_advance(h, ud, F, m == 1, 1e-12)
            assert info.relres <= 1e-12
            assert relerr(to_host(ud), uref) < 1e-10, m
    finally:
        T.tfde_destroy(h)


NONSYM = [
    ((40, 32, 24), (0.3, 0.6, 0.8), (1.0, 1.5, 2.0), (0.5, 2.0, 1.0), 0.1, 20),
    ((64, 24, 136), (0.7, 0.2, 0.9), (2.0, 1.0, 0.5), (1.0, 0.5, 1.5), 0.05, 4),   # short cycles, ragged tiles
]


@pytest.mark.parametrize("case", NONSYM, ids=lambda c: "x".join(map(str, c[0])) + f"_m{c[5]}")
def test_eigenbasis_and_grid_basis_pgmres_match_oracle(T, case):
    """Left-preconditioned GMRES (Sec. 3.2) in both bases: Lambda^{-1} S_N A S_N
    in the eigenbasis is the grid basis's P^{-1} A transformed by S_N, so the
    refined solutions match the oracle's and the Arnoldi step counts agree."""
    n, d, kp, km, dt, restart = case
    op = o.Problem(n=n, delta=d, kp=kp, km=km, dt=dt)
    b = inp.uniform_vector(op.shape, 74)
    tau = o.build_tau(op)
    xref, _ = o.gmres_left(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, np.zeros_like(b), 1e-14,
                           4000, restart=20, criterion="true")
    iters = {}
    for spectral in (True, False):
        for dev_loop in ((True, False) if spectral else (True,)):
            h = T.tfde_assemble(T.make_params(n, d, kp, km, dt), T.TFDE_MIXED)
            try:
                T.tfde_set_spectral_inner(h, spectral)
                T.tfde_set_device_loop(h, dev_loop)
                x = to_dev(np.zeros_like(b))
                info = T.tfde_pgmres(h, to_dev(b), x, restart, 1e-12, 4000)
                assert info.relres <= 1e-12 and info.fallback == 0, (spectral, dev_loop, info.relres)
                launches = T.tfde_device_loop_launches(h)
                assert (launches == info.restarts) if dev_loop else (launches == 0), (spectral, dev_loop, launches)
                assert relerr(to_host(x), xref) < 1e-10
                iters[(spectral, dev_loop)] = info.iters
            finally:
                T.tfde_destroy(h)
    assert iters[(True, True)] == iters[(True, False)], iters
    assert abs(iters[(True, True)] - iters[(False, True)]) <= max(2, iters[(False, True)] // 5), iters


def test_toggle_rejected_where_unavailable(T):
    f64 = T.tfde_assemble(T.make_params((16, 16, 16), (0.5,) * 3, (1.0,) * 3, (1.0,) * 3, 0.1), T.TFDE_FP64)
    fft = T.tfde_assemble(T.make_params((15, 16, 17), (0.5,) * 3, (1.0,) * 3, (1.0,) * 3, 0.1), T.TFDE_MIXED)
    ns = T.tfde_assemble(T.make_params((16, 16, 16), (0.5,) * 3, (1.0,) * 3, (0.5,) * 3, 0.1), T.TFDE_MIXED)
    try:
        for h in (f64, fft):
            with pytest.raises(T.TfdeError) as e:
                T.tfde_set_spectral_inner(h, True)
            assert e.value.status == T.TFDE_EUNSUPPORTED
            T.tfde_set_spectral_inner(h, False)   # accepted, no effect
        T.tfde_set_spectral_inner(ns, True)        # non-symmetric tensor-core problems have it too
        T.tfde_set_spectral_inner(ns, False)
    finally:
        for h in (f64, fft, ns):
            T.tfde_destroy(h)
