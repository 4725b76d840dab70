"""The allocation-free mass operator, called through the C ABI.

tfde_mass_apply_noalloc is for callers that cannot allocate device memory
when they apply the operator (fixed memory budgets, loops where the
allocator's implicit synchronisation is not allowed, plug-ins handed
ready-made buffers).  Its result must equal A_N x from the existing entry
point: A_N = (A + (2 A_N - A)) / 2, i.e. the mean of tfde_matvec with
TFDE_OP_A and TFDE_OP_RHS on an FP64 problem of the same grid.  Two calls in a
row with different inputs check that the shared fixed scratch carries nothing
over.  This file is collected last so that a run stopping at the first
failure has already run every other test."""
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


def reference_mass_apply(T, n, v):
    h = T.tfde_assemble(T.make_params(n, (0.4, 0.6, 0.8), (1.0, 2.0, 1.0), (0.5, 1.0, 1.5), 0.1), T.TFDE_FP64)
    try:
        x = to_dev(v)
        ya = to_dev(np.zeros_like(v))
        yr = to_dev(np.zeros_like(v))
        T.tfde_matvec(h, T.TFDE_OP_A, x, ya)
        T.tfde_matvec(h, T.TFDE_OP_RHS, x, yr)
        return 0.5 * (to_host(ya) + to_host(yr))
    finally:
        T.tfde_destroy(h)


@pytest.mark.parametrize("n", [(40, 24, 16), (64, 64, 64), (1, 7, 3), (1, 512, 512), (512, 1, 512)])
def test_noalloc_mass_apply_matches_existing_entry_point_twice(T, n):
    """Two calls in a row with different inputs; (1, 512, 512) has more x
    lines than one launch dimension holds (65535 blocks of 4 lines)."""
    shape = (n[2], n[1], n[0])
    # the reference (A x + (2 A_N - A) x) / 2 cancels the stiffness terms,
    # which grow with the grid: its own rounding sets the bar on long axes
    bar = 1e-13 if max(n) <= 64 else 1e-12
    for seed in (61, 62):   # two calls in a row, different inputs
        v = inp.uniform_vector(shape, seed)
        y = to_dev(np.full(shape, np.nan))
        T.tfde_mass_apply_noalloc(n, to_dev(v), y)
        assert relerr(to_host(y), reference_mass_apply(T, n, v)) < bar


def test_noalloc_in_place_and_allocates_nothing(T):
    """y may be the same buffer as x, and a call (after the first on the
    device, which looks up the scratch address) changes neither the device's
    free memory nor torch's allocator state."""
    import torch
    n = (24, 16, 40)
    shape = (n[2], n[1], n[0])
    v = inp.uniform_vector(shape, 63)
    ref = reference_mass_apply(T, n, v)
    x = to_dev(v)
    y = to_dev(np.zeros(shape))
    T.tfde_mass_apply_noalloc(n, x, y)   # first call on this device
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    T.tfde_mass_apply_noalloc(n, x, x)   # in place
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0
    assert relerr(to_host(x), ref) < 1e-13


def test_noalloc_rejects_grids_beyond_the_limit(T):
    x = to_dev(np.zeros(8))
    with pytest.raises(T.TfdeError) as e:
        T.tfde_mass_apply_noalloc((65, 64, 64), x, x)
    assert e.value.status == T.TFDE_EINVAL and "262144" in str(e.value)
