"""tfde_cn_advance_host: the chained CN step (Eq. (CN)) with the state copied
from and to host buffers, the copies overlapping the step's own work.  The
host output must equal the device-only advance of the same steps (up to the
order of atomic inner-product sums), and the device state must hold exactly
what was copied out."""
import math

import numpy as np
import pytest
import torch

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
    ("mixed_sym_order3", (24, 32, 40), (0.7, 0.6, 0.5), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), "MIXED", 3),
    ("mixed_nonsym", (32, 24, 16), (0.3, 0.6, 0.8), (1.0, 1.5, 0.5), (0.5, 1.0, 2.0), "MIXED", 0),
    ("fp64_sym", (16, 16, 24), (0.5, 0.5, 0.5), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), "FP64", 2),
    # over 2^20 points: the input arrives in eight pieces and the right-hand-side
    # and guess pass runs range by range as they come in
    ("mixed_sym_order3_pieces", (96, 104, 112), (0.7, 0.7, 0.7), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), "MIXED", 3),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_host_buffer_steps_match_device_steps(T, case):
    _, n, d, kp, km, prec, order = case
    dt = 0.05
    steps = 5
    op = o.Problem(n=n, delta=d, kp=kp, km=km, dt=dt)
    u0 = o.exact_u(op, 0.0, "exp") if kp == km else inp.smoothed_uniform(tuple(reversed(n)), 5)
    precision = T.TFDE_MIXED if prec == "MIXED" else T.TFDE_FP64
    hd = T.tfde_assemble(T.make_params(n, d, kp, km, dt), precision)
    hh = T.tfde_assemble(T.make_params(n, d, kp, km, dt), precision)
    try:
        for h in (hd, hh):
            T.tfde_set_guess_order(h, order)
        ud = to_dev(u0)
        uh = to_dev(np.zeros_like(u0))
        hin = torch.from_numpy(np.ascontiguousarray(u0)).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        for m in range(1, steps + 1):
            th = (m - 0.5) * dt
            F = to_dev(np.zeros_like(u0))
            T.tfde_source_example2(hd, -math.exp(-th), -math.exp(-th), F)
            a = T.tfde_cn_advance(hd, ud, F, m == 1, 1e-11)
            b = T.tfde_cn_advance_host(hh, hin, hout, uh, F, m == 1, 1e-11)
            torch.cuda.synchronize()
            assert a.relres <= 1e-11 and b.relres <= 1e-11, (m, a.relres, b.relres)
            assert np.array_equal(hout.numpy(), to_host(uh)), m          # the copy is the device state
            assert relerr(hout.numpy(), to_host(ud)) < 1e-12, m          # and the device-only step's result
            if m % 2:
                hin, hout = hout, hin                                     # separate buffers
            else:
                hin.copy_(hout)                                           # in place: output aliases input
                hout = hin
    finally:
        T.tfde_destroy(hd)
        T.tfde_destroy(hh)


def test_host_buffer_arguments_checked(T):
    n = (16, 16, 16)
    h = T.tfde_assemble(T.make_params(n, (0.5,) * 3, (1.0,) * 3, (1.0,) * 3, 0.1), T.TFDE_MIXED)
    try:
        u = to_dev(np.zeros(tuple(reversed(n))))
        host = torch.zeros(tuple(reversed(n)), dtype=torch.float64).pin_memory()
        for hin, hout in ((u, host), (host, u)):
            with pytest.raises(T.TfdeError) as e:
                T.tfde_cn_advance_host(h, hin, hout, u, None, True, 1e-8)
            assert e.value.status == T.TFDE_EINVAL
        info = T.tfde_cn_advance_host(h, host, host, u, None, True, 1e-8)   # zero data: done at once
        assert info.iters == 0 and float(host.abs().max()) == 0.0
    finally:
        T.tfde_destroy(h)
