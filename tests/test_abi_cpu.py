"""CPU-only checks of the C-ABI library: it builds, loads, exports every
symbol include/tfde.h declares, and its host-side assembly (generator
coefficients, eigenvalue arrays, eta) agrees with the oracle.  No GPU work."""
import os
import re

import numpy as np
import pytest

from oracle import tfde_oracle as o

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_21198_gb300 import build
    build.build()
    from paper_2511_21198_gb300 import tfde
    return tfde


def declared_symbols():
    out = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            out |= set(re.findall(r"\b(tfde_[a-z0-9_]+)\s*\(", txt))
    return out


def test_every_declared_symbol_is_exported(lib):
    import ctypes
    so = ctypes.CDLL(lib.LIB_PATH)
    syms = declared_symbols()
    assert len(syms) >= 12
    for s in sorted(syms):
        assert hasattr(so, s), s
    assert set(lib.EXPORTS) <= syms


def test_version(lib):
    assert "sm_103a" in lib.tfde_version()


@pytest.mark.parametrize("d", [0.05, 0.3, 0.5, 0.7, 0.95])
@pytest.mark.parametrize("n", [1, 2, 3, 17, 256, 1000])
def test_host_coefficients_match_oracle(lib, d, n):
    p = lib.make_params((n, 5, 7), (d, 0.5, 0.5), (1.0, 2.0, 1.0), (0.5, 2.0, 1.0), 0.05)
    q, lt, lm, eta = lib.tfde_host_coefficients(p, 0)
    qo = o.q_coefficients(d, n)
    np.testing.assert_allclose(q, qo, rtol=5e-15, atol=0)
    np.testing.assert_allclose(lt, o.tau_eigenvalues(qo, n), rtol=1e-13, atol=1e-15 * max(1.0, abs(qo[1])))
    np.testing.assert_allclose(lm, o.mass_eigenvalues(n), rtol=2e-16, atol=2e-16)
    assert eta == pytest.approx(o.eta(d, 1.0 / (n + 1), 0.05), rel=1e-15)


@pytest.mark.parametrize("bad", [dict(delta=(1.5, 0.5, 0.5)), dict(delta=(0.0, 0.5, 0.5)),
                                 dict(n=(0, 4, 4)), dict(kp=(-1.0, 1.0, 1.0)), dict(dt=0.0)])
def test_host_validation(lib, bad):
    args = dict(n=(4, 4, 4), delta=(0.5, 0.5, 0.5), kp=(1.0, 1.0, 1.0), km=(1.0, 1.0, 1.0), dt=0.1)
    args.update(bad)
    p = lib.make_params(**args)
    with pytest.raises(lib.TfdeError) as e:
        lib.tfde_host_coefficients(p, 0)
    assert e.value.status == lib.TFDE_EINVAL


def test_tune_table_round_trip_on_the_host(lib, tmp_path):
    """The autotuner's table is host state: entries set, read back, replaced
    per launch class, rejected when out of range, cached as JSON per GPU
    name and applied again (no GPU work)."""
    lib.load()
    lib.tfde_tune_clear()
    e1 = dict(grouped=0, kmajor=1, out_mode=3, stage_bytes=49152, n=256, tiles=512, grid=128, stages=3,
              us=15.5, us_default=16.25)
    e2 = dict(grouped=1, kmajor=0, out_mode=1, stage_bytes=98304, n=0, tiles=1024, grid=152, stages=2,
              us=60.0, us_default=60.0)
    lib.tfde_tune_set([e1, e2])
    got = lib.tfde_tune_get()
    assert got == [e1, e2]
    lib.tfde_tune_set([dict(e1, grid=144, stages=4)])          # same class: replaced, not added
    got = lib.tfde_tune_get()
    assert len(got) == 2 and got[0]["grid"] == 144 and got[0]["stages"] == 4
    with pytest.raises(lib.TfdeError) as e:
        lib.tfde_tune_set([dict(e2, stages=3)])                # 3 x 96 KB exceeds the 192 KB ring
    assert e.value.status == lib.TFDE_EINVAL
    path = str(tmp_path / "tuning.json")
    lib.save_tuning(path, "GPU A")
    lib.tfde_tune_clear()
    assert lib.tfde_tune_get() == []
    assert lib.load_tuning(path, "GPU B") == 0
    assert lib.load_tuning(path, "GPU A") == 2
    assert lib.tfde_tune_get() == got
    lib.tfde_tune_clear()
