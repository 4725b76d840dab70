"""Seeded synthetic inputs shared by the oracle-side tests and the GPU-side tests
and bench.  Holds none of the method's arithmetic: only random draws, a
binomial smoothing filter for initial data, and workload parameter tables.

Every generator takes an explicit seed and returns host float64 numpy arrays
(or plain Python values), so both sides see identical bits.
"""
from __future__ import annotations

import numpy as np


def smoothed_uniform(shape, seed: int, passes: int = 4) -> np.ndarray:
    """uniform(0,1) noise on a (n3, n2, n1) grid, smoothed by `passes`
    applications per axis of the binomial filter [1, 2, 1] / 4 with zero
    exterior, then scaled so that max |u| = 1."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, size=shape)
    for _ in range(passes):
        for ax in range(3):
            pad = [(0, 0)] * 3
            pad[ax] = (1, 1)
            up = np.pad(u, pad)
            sl = [slice(None)] * 3
            lo, mid, hi = list(sl), list(sl), list(sl)
            lo[ax] = slice(0, -2)
            mid[ax] = slice(1, -1)
            hi[ax] = slice(2, None)
            u = 0.25 * up[tuple(lo)] + 0.5 * up[tuple(mid)] + 0.25 * up[tuple(hi)]
    return u / np.abs(u).max()


def uniform_vector(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Plain seeded uniform(lo, hi) grid function (for operator parity tests)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


def batched_instances(count: int = 64, seed: int = 4, sizes=(32, 48, 64, 96, 128)):
    """Parameters of the uneven batched workload: n ~ uniform over `sizes`,
    delta_i ~ U(0.1, 0.9) and k_{i,+-} ~ U(0.5, 2) per axis."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.choice(sizes))
        out.append(dict(n=(n, n, n),
                        delta=tuple(float(v) for v in rng.uniform(0.1, 0.9, 3)),
                        kp=tuple(float(v) for v in rng.uniform(0.5, 2.0, 3)),
                        km=tuple(float(v) for v in rng.uniform(0.5, 2.0, 3))))
    return out


# The five workloads of the benchmark table (grid size per axis n, so that
# h = 1/(n+1); T = 1 and dt = 1/M).
WORKLOADS = {
    "n16_sym_exp": dict(n=16, delta=(0.5, 0.5, 0.5), kp=(1.0,) * 3, km=(1.0,) * 3, M=16,
                        source="exp", tol=1e-8),
    "n128_nonsym": dict(n=128, delta=(0.3, 0.6, 0.8), kp=(1.0,) * 3, km=(0.5,) * 3, M=50,
                        source=None, u0_seed=2, tol=1e-8),
    "n256_sym_exp": dict(n=256, delta=(0.7, 0.7, 0.7), kp=(1.0,) * 3, km=(1.0,) * 3, M=20,
                         source="exp", tol=1e-8),
}


def example2_initial(n, phi0: float = 1.0) -> np.ndarray:
    """Nodal values phi0 * P(x) P(y) P(z), P(s) = s^2 (1-s)^2, at the interior
    nodes s_p = p/(n_a+1) of (0,1)^3: the initial data of the manufactured
    workloads (problem data, shape (n3, n2, n1))."""
    if isinstance(n, int):
        n = (n, n, n)
    ax = [np.arange(1, m + 1, dtype=np.float64) / (m + 1) for m in n]
    Px, Py, Pz = (a * a * (1.0 - a) ** 2 for a in ax)
    return phi0 * Pz[:, None, None] * Py[None, :, None] * Px[None, None, :]
