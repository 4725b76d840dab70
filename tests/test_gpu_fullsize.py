"""Parity of the mixed path with the oracle at the benchmark sizes.

Per CN step from the same u^{m-1} (Sec. 2, Eq. (CN) and Eq. (linear_sys)),
both sides solve to a tight true FP64 residual, so two correct solvers agree
far below the tolerance: A >= A_N >= 1/8 in the symmetric case (and the
symmetric part of the non-symmetric operator likewise), so
||x_gpu - x_oracle|| <= 8 (||r_gpu|| + ||r_oracle||), i.e. about 1e-11 of
||b|| ~ ||x|| at residuals 1e-12 / 1e-13.  The bar is 1e-10 relative
error.  The oracle (numpy FP64, dense per-axis products) takes 10-40 s per
solve at n = 256 on the host cores."""
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


def oracle_pcg_step(op, u_prev, F, tol=1e-13):
    tau = o.build_tau(op)
    b = o.rhs(op, u_prev, F)
    x, info = o.pcg(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, u_prev, tol, 4000)
    assert info.converged
    return x


def test_c3_n256_symmetric_step_matches_oracle(T):
    """The benchmark workload (n = 256, delta = 0.7, k+ = k- = 1, dt = 1/20,
    exp(-t) manufactured source): one mixed PCG step from the exact initial
    data at a 1e-12 true residual against the oracle's PCG at 1e-13."""
    W = inp.WORKLOADS["n256_sym_exp"]
    n, dt = W["n"], 1.0 / W["M"]
    op = o.Problem(n=(n, n, n), delta=W["delta"], kp=W["kp"], km=W["km"], dt=dt)
    u0 = inp.example2_initial(n)
    F = o.source_cell_average(op, 0.5 * dt, "exp")
    xo = oracle_pcg_step(op, u0, F)
    h = T.tfde_assemble(T.make_params((n, n, n), W["delta"], W["kp"], W["km"], dt), T.TFDE_MIXED)
    try:
        un = to_dev(np.zeros_like(u0))
        info = T.tfde_cn_step(h, to_dev(u0), to_dev(F), None, un, 1e-12)
        assert info.relres <= 1e-12 and info.fallback == 0
        assert relerr(to_host(un), xo) < 1e-10
    finally:
        T.tfde_destroy(h)


def test_c3_n256_chained_advance_matches_oracle(T):
    """The benchmark's call path: tfde_cn_advance chained in place with the
    order-3 extrapolated guess and the device-side source, three steps at a
    1e-12 residual; the third step against the oracle's step from the GPU's
    own u^2 (fed back, as the per-step parity reading prescribes)."""
    import torch
    W = inp.WORKLOADS["n256_sym_exp"]
    n, dt = W["n"], 1.0 / W["M"]
    op = o.Problem(n=(n, n, n), delta=W["delta"], kp=W["kp"], km=W["km"], dt=dt)
    h = T.tfde_assemble(T.make_params((n, n, n), W["delta"], W["kp"], W["km"], dt), T.TFDE_MIXED)
    try:
        T.tfde_set_guess_order(h, 3)
        u = to_dev(inp.example2_initial(n))
        F = torch.empty_like(u)
        prev = None
        for m in range(3):
            e = math.exp(-(m + 0.5) * dt)
            T.tfde_source_example2(h, -e, -e, F)
            if m == 2:
                prev = to_host(u)
            info = T.tfde_cn_advance(h, u, F, m == 0, 1e-12)
            assert info.relres <= 1e-12 and info.fallback == 0
        Fh = o.source_cell_average(op, 2.5 * dt, "exp")
        assert relerr(to_host(F), Fh) < 1e-13
        xo = oracle_pcg_step(op, prev, Fh)
        assert relerr(to_host(u), xo) < 1e-10
    finally:
        T.tfde_destroy(h)


def test_c2_n128_nonsymmetric_step_matches_oracle(T):
    """The non-symmetric workload (n = 128, delta = (0.3, 0.6, 0.8), k+ = 1,
    k- = 0.5, f = 0, smoothed-noise u0 with seed 2, dt = 1/50): one mixed
    PGMRES(20) step at a 1e-12 true residual against the oracle's
    left-preconditioned GMRES(20) at 1e-13."""
    W = inp.WORKLOADS["n128_nonsym"]
    n, dt = W["n"], 1.0 / W["M"]
    op = o.Problem(n=(n, n, n), delta=W["delta"], kp=W["kp"], km=W["km"], dt=dt)
    u0 = inp.smoothed_uniform(op.shape, W["u0_seed"])
    b = o.rhs(op, u0, None)
    tau = o.build_tau(op)
    xo, info = o.gmres_left(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, u0, 1e-13, 4000,
                            restart=20, criterion="true")
    assert info.converged
    h = T.tfde_assemble(T.make_params((n, n, n), W["delta"], W["kp"], W["km"], dt), T.TFDE_MIXED)
    try:
        un = to_dev(np.zeros_like(u0))
        info = T.tfde_cn_step(h, to_dev(u0), None, None, un, 1e-12)
        assert info.relres <= 1e-12 and info.fallback == 0 and info.restarts >= 1
        assert relerr(to_host(un), xo) < 1e-10
    finally:
        T.tfde_destroy(h)
