"""The autotuner of the tensor-core contraction's launch parameters on the
GPU: tfde_tune / tfde_batch_tune fill the table with measured choices,
solves with the tuned launches still match the oracle, and a table cached as
JSON is applied by a fresh process."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import tfde_oracle as o
import tfde_inputs as inp
from gpu_helpers import relerr, to_dev, to_host

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def T():
    from paper_2511_21198_gb300 import build
    build.build()
    from paper_2511_21198_gb300 import tfde
    tfde.load()
    return tfde


def gpu_name():
    import torch
    return torch.cuda.get_device_name(0)


def test_tune_problem_and_solve_matches_oracle(T):
    n, d, kp = (64, 48, 40), (0.3, 0.6, 0.8), (1.0, 1.5, 2.0)
    T.tfde_tune_clear()
    h = T.tfde_assemble(T.make_params(n, d, kp, kp, 0.1), T.TFDE_MIXED)
    try:
        op = o.Problem(n=n, delta=d, kp=kp, km=kp, dt=0.1)
        b = inp.uniform_vector(op.shape, 71)
        x0 = to_dev(np.zeros_like(b))
        T.tfde_pcg(h, to_dev(b), x0, 1e-12, 2000)        # builds the device-loop graph with the defaults
        T.tfde_tune(h, 5)
        table = T.tfde_tune_get()
        # the operator's two grouped pairs and its z pass, the preconditioner's passes
        assert len(table) >= 5
        import torch
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        for e in table:
            assert 1 <= e["grid"] <= min(sms, e["tiles"]) and 2 <= e["stages"] <= 4
            assert e["us"] > 0 and e["us"] <= e["us_default"] * 1.0001
        tau = o.build_tau(op)
        xref, _ = o.pcg(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, np.zeros_like(b), 1e-14, 2000)
        x = to_dev(np.zeros_like(b))
        info = T.tfde_pcg(h, to_dev(b), x, 1e-12, 2000)   # recaptured with the tuned launches
        assert info.relres <= 1e-12 and info.fallback == 0
        assert relerr(to_host(x), xref) < 1e-10
    finally:
        T.tfde_destroy(h)
        T.tfde_tune_clear()


def test_tune_batch_then_advance_converges(T):
    prm = [T.make_params((32, 24, 16), (0.5, 0.6, 0.7), (1.0, 2.0, 1.0), (0.5, 1.0, 2.0), 0.1),
           T.make_params((16, 16, 48), (0.3, 0.4, 0.5), (1.0,) * 3, (1.0,) * 3, 0.1),
           T.make_params((40, 8, 24), (0.8, 0.2, 0.6), (2.0, 1.0, 1.0), (1.0, 1.0, 0.5), 0.1)]
    T.tfde_tune_clear()
    B = T.tfde_batch_create(prm, 20)
    try:
        T.tfde_batch_tune(B, 3)
        table = T.tfde_tune_get()
        assert table and all(e["grouped"] == 1 for e in table)
        us = [to_dev(inp.smoothed_uniform(tuple(p.n)[::-1], 5 + i)) for i, p in enumerate(prm)]
        infos = T.tfde_batch_cn_advance(B, us, None, True, 1e-10)
        assert all(i.relres <= 1e-10 for i in infos)
    finally:
        T.tfde_batch_destroy(B)
        T.tfde_tune_clear()


def test_cached_table_applies_in_a_fresh_process(T, tmp_path):
    n = (48, 40, 32)
    T.tfde_tune_clear()
    h = T.tfde_assemble(T.make_params(n, (0.5,) * 3, (1.0,) * 3, (1.0,) * 3, 0.1), T.TFDE_MIXED)
    try:
        T.tfde_tune(h, 3)
    finally:
        T.tfde_destroy(h)
    table = T.tfde_tune_get()
    path = str(tmp_path / "tuning.json")
    T.save_tuning(path, gpu_name())
    T.tfde_tune_clear()
    code = (
        "import json, sys, numpy as np, torch\n"
        "from paper_2511_21198_gb300 import tfde as T\n"
        "T.load()\n"
        f"k = T.load_tuning({path!r}, torch.cuda.get_device_name(0))\n"
        f"h = T.tfde_assemble(T.make_params({n!r}, (0.5,) * 3, (1.0,) * 3, (1.0,) * 3, 0.1), T.TFDE_MIXED)\n"
        "b = torch.rand(" + f"{n[2]}, {n[1]}, {n[0]}" + ", dtype=torch.float64, device='cuda')\n"
        "x = torch.zeros_like(b)\n"
        "info = T.tfde_pcg(h, b, x, 1e-12, 2000)\n"
        "T.tfde_destroy(h)\n"
        "print(json.dumps({'applied': k, 'table': T.tfde_tune_get(), 'relres': info.relres}))\n")
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["applied"] == len(table) and out["table"] == table
    assert out["relres"] <= 1e-12
