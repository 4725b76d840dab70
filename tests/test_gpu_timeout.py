"""The bounded device-side waits of the tensor-core kernels (Sec. 3.1 solves
run on them): a wait that nothing satisfies gives up after its limit, reports
TFDE_ETIMEOUT, releases the kernel's tensor memory, and leaves the device
usable for the next tensor-core call.  The wait is made to run out on an
mbarrier that nothing arrives on; no copy or MMA is in flight, so nothing can
fault."""
import numpy as np
import pytest

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


def test_bounded_wait_runs_out_and_device_stays_usable(T):
    import time
    for limit in (50_000, 2_000_000):   # 50 us and 2 ms; the second call also re-allocates tensor memory
        t0 = time.perf_counter()
        st, freed = T.tfde_selftest_wait(limit)
        assert st == T.TFDE_ETIMEOUT and freed == 1, (st, T.tfde_last_error())
        assert time.perf_counter() - t0 < 5.0
    # the next tensor-core work on the same context runs normally
    n = (16, 16, 16)
    h = T.tfde_assemble(T.make_params(n, (0.5, 0.5, 0.5), (1.0,) * 3, (1.0,) * 3, 0.1), T.TFDE_MIXED)
    h64 = T.tfde_assemble(T.make_params(n, (0.5, 0.5, 0.5), (1.0,) * 3, (1.0,) * 3, 0.1), T.TFDE_FP64)
    try:
        v = inp.uniform_vector((16, 16, 16), 71)
        y = to_dev(np.zeros_like(v))
        y64 = to_dev(np.zeros_like(v))
        T.tfde_matvec(h, T.TFDE_OP_A | T.TFDE_OP_FAST, to_dev(v), y)
        T.tfde_matvec(h64, T.TFDE_OP_A, to_dev(v), y64)
        assert relerr(to_host(y), to_host(y64)) < 1e-4
    finally:
        T.tfde_destroy(h)
        T.tfde_destroy(h64)


def test_selftest_rejects_limits_out_of_range(T):
    for bad in (0, 999, 3_000_000_000):
        st, _ = T.tfde_selftest_wait(bad)
        assert st == T.TFDE_EINVAL
