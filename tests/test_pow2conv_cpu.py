"""Integer FP64 <-> FP32 conversions with a power-of-two scale (the inner
solver's residual scale and the correction's scale back): bit-identical to
IEEE round-to-nearest-even conversions of the scaled values, on random,
tie and subnormal-range inputs.  The same header the CUDA kernels include is
compiled for the host."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2511_21198_gb300", "csrc")


def test_pow2_conversions_match_ieee(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "pow2conv_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "native", "pow2conv_check.cpp"),
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    f = out.stdout.split()
    assert out.returncode == 0, out.stdout + out.stderr
    assert int(f[1]) > 3_000_000 and int(f[2]) == 0
    assert int(f[4]) > 3_000_000 and int(f[5]) == 0
    assert f[7] == "1"
