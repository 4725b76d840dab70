"""Spectral estimates of the preconditioned systems (Sec. 3) by Lanczos on the
GPU (tfde_spectrum): against dense eigensolves of the oracle's explicit
matrices on a small grid (A of Eq. (original_matrix_form), P of Eq.
(pre_definition)), and at the benchmark sizes against the paper's bounds:
Theorem CG_bounded_sprctrum / Lemma prop:eigen_S (symmetric part in
(1/2, 3/2)) and Lemma eigen_Skew (skew radius <= varsigma)."""
import math

import numpy as np
import pytest
from scipy import linalg

from oracle import tfde_oracle as o
import tfde_inputs as inp
from gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2511_21198_gb300 import build
    build.build()
    from paper_2511_21198_gb300 import tfde
    tfde.load()
    return tfde


def dense_spectra(op):
    A = o.dense_A(op)
    P = o.dense_P_from_definition(op)
    w, Q = linalg.eigh(P)
    Ph = Q @ np.diag(w ** -0.5) @ Q.T
    MH = Ph @ (0.5 * (A + A.T)) @ Ph
    MS = Ph @ (0.5 * (A - A.T)) @ Ph
    eh = linalg.eigvalsh(0.5 * (MH + MH.T))
    es = np.abs(linalg.eigvals(MS)).max()
    return eh[0], eh[-1], es


@pytest.mark.parametrize("case", [
    ((4, 5, 3), (0.3, 0.6, 0.8), (1.0, 2.0, 1.5), (0.5, 1.0, 0.5), 0.05),
    ((6, 4, 4), (0.7, 0.7, 0.7), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), 0.05),
])
def test_lanczos_estimates_match_dense_eigensolve(T, case):
    n, d, kp, km, dt = case
    op = o.Problem(n=n, delta=d, kp=kp, km=km, dt=dt)
    lo, hi, rho = dense_spectra(op)
    N = n[0] * n[1] * n[2]
    v0 = to_dev(inp.uniform_vector(op.shape, 9))
    info = T.tfde_spectrum(T.make_params(n, d, kp, km, dt), N, v0)
    assert abs(info.sym_min - lo) <= 1e-7 and abs(info.sym_max - hi) <= 1e-7
    assert abs(info.skew_rho - rho) <= 1e-6 * max(rho, 1.0)
    vs = max(1.5 * math.tan(0.5 * math.pi * d[a]) * abs(kp[a] - km[a]) / (kp[a] + km[a]) for a in range(3))
    assert info.varsigma == pytest.approx(vs, rel=1e-14)
    assert info.omega == pytest.approx(math.sqrt((2 + 4 * vs * vs) / (3 + 4 * vs * vs)), rel=1e-14)


def test_benchmark_sizes_inside_the_paper_bounds(T):
    """n = 256 symmetric (the benchmark) and n = 128 non-symmetric: 40
    Lanczos steps; the Ritz values of the symmetric part stay in (1/2, 3/2)
    and the skew radius below varsigma, the grid-independent constants."""
    W = inp.WORKLOADS["n256_sym_exp"]
    n = W["n"]
    v0 = to_dev(inp.uniform_vector((n, n, n), 10))
    s = T.tfde_spectrum(T.make_params((n, n, n), W["delta"], W["kp"], W["km"], 1.0 / W["M"]), 40, v0)
    assert 0.5 < s.sym_min < s.sym_max < 1.5 and s.skew_rho == 0.0
    W = inp.WORKLOADS["n128_nonsym"]
    n = W["n"]
    v0 = to_dev(inp.uniform_vector((n, n, n), 11))
    s = T.tfde_spectrum(T.make_params((n, n, n), W["delta"], W["kp"], W["km"], 1.0 / W["M"]), 40, v0)
    assert 0.5 < s.sym_min < s.sym_max < 1.5
    assert 0.0 < s.skew_rho <= s.varsigma
    assert math.sqrt(2.0 / 3.0) <= s.omega < 1.0
