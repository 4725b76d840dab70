"""Builds libtfde.so in-tree: every csrc/*.cu compiled for sm_103a in
parallel, then linked into paper_2511_21198_gb300/_lib/libtfde.so.

An object is reused only when a stamp beside it records the SHA-256 of its
source, of every header, of the compiler flags, of the nvcc version and of
the host machine type it was built on: a copy of the tree moved to another
machine, or any edited file, recompiles (file times are not trusted).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import platform
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libtfde.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
          "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def nvcc_path() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found (CUDA toolkit required to build libtfde)")
    return p


def _headers_digest() -> str:
    hs = sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                + glob.glob(os.path.join(ROOT, "include", "*.h")))
    h = hashlib.sha256()
    for f in hs:
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()


_NVCC_VERSION = None


def _nvcc_version() -> str:
    global _NVCC_VERSION
    if _NVCC_VERSION is None:
        r = subprocess.run([nvcc_path(), "--version"], capture_output=True, text=True)
        _NVCC_VERSION = r.stdout.strip().splitlines()[-1] if r.returncode == 0 and r.stdout.strip() else "?"
    return _NVCC_VERSION


def _unit_digest(src: str, headers: str, extra: list[str]) -> str:
    h = hashlib.sha256()
    h.update(open(src, "rb").read())
    h.update(headers.encode())
    h.update(" ".join([*ARCH, *CFLAGS, *extra]).encode())
    h.update(_nvcc_version().encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def _compile(src: str, obj: str, extra: list[str]) -> None:
    cmd = [nvcc_path(), *ARCH, *CFLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    """Compile the translation units whose stamp does not match and relink;
    returns the library path."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    extra = list(extra_flags or [])
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = _headers_digest()
    jobs = []
    objs = []
    digests = {}
    for s in srcs:
        o = os.path.join(BUILD_DIR, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        d = _unit_digest(s, headers, extra)
        digests[o] = d
        stamp = o + ".sha256"
        fresh = (os.path.exists(o) and os.path.exists(stamp) and open(stamp).read().strip() == d)
        if force or not fresh:
            jobs.append((s, o))
    if jobs:
        for _, o in jobs:   # a failed compile must not leave a matching stamp behind
            if os.path.exists(o + ".sha256"):
                os.remove(o + ".sha256")
        with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            futs = [ex.submit(_compile, s, o, extra) for s, o in jobs]
            for f in futs:
                f.result()
        for _, o in jobs:
            with open(o + ".sha256", "w") as f:
                f.write(digests[o])
    link_stamp = LIB_PATH + ".sha256"
    link_digest = hashlib.sha256("".join(digests[o] for o in objs).encode()).hexdigest()
    linked = os.path.exists(LIB_PATH) and os.path.exists(link_stamp) and open(link_stamp).read().strip() == link_digest
    if jobs or force or not linked:
        if os.path.exists(link_stamp):
            os.remove(link_stamp)
        cmd = [nvcc_path(), *ARCH, "-shared", "-o", LIB_PATH, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link of libtfde.so failed:\n" + r.stderr)
        with open(link_stamp, "w") as f:
            f.write(link_digest)
    if verbose:
        print(f"built {LIB_PATH} ({len(jobs)} units recompiled, {len(srcs) - len(jobs)} reused by source hash)")
    return LIB_PATH


if __name__ == "__main__":
    build(verbose=True)
