"""CPU oracle of the warm-start network (test infrastructure only: imported by
tests/, __graft_entry__.smoke() and bench.py's CPU baseline, never by the
product path).

The network is not part of the paper; it is the learned initial guess of the
CN solves.  It maps, per grid point, the input channels
    (u^m, dt F^{m+1/2}, c_1, ..., c_9)
(u and dt F scaled by 1/s, s = max |u^m|; nine problem coefficients as
constant planes -- the caller's choice; the package passes delta_1..3 and
the logarithms of the per-axis stiffness scales eta_a k+_a, eta_a k-_a)
to Delta / s, Delta = u^{m+1} - u^m, through four 3x3x3 convolutions with
zero padding ("same" size) and ReLU between them.

Everything is written from the definition, in float64:

  conv:   y[o, p] = b[o] + sum_i sum_{t in {-1,0,1}^3} W[o, i, t + 1] x[i, p + t]
          (x = 0 outside the grid; p = (z, y, x) with x fastest)
  dx:     dx[i, p] = sum_o sum_t W[o, i, t + 1] dy[o, p - t]
  dW:     dW[o, i, t + 1] = sum_p dy[o, p] x[i, p + t]
  db:     db[o] = sum_p dy[o, p]
  ReLU:   a = max(z, 0), dz = da * [z > 0]
  loss:   L = mean over points of (out - target)^2 (one output channel)

Arrays: activations (C, n3, n2, n1); weights (Cout, Cin, 3, 3, 3) indexed
[o, i, dz + 1, dy + 1, dx + 1]; bias (Cout,).

Parity is pinned in tests/test_oracle_cnn.py against a library correlation
(scipy.ndimage.correlate), closed-form shifts, the adjoint identity and
central finite differences.
"""
from __future__ import annotations

import itertools

import numpy as np

TAPS = list(itertools.product((-1, 0, 1), repeat=3))  # (dz, dy, dx), dx fastest


def shifted(x: np.ndarray, t) -> np.ndarray:
    """s[..., p] = x[..., p + t] with zero fill outside the grid (last three axes)."""
    dz, dy, dx = t
    out = np.zeros_like(x)
    n3, n2, n1 = x.shape[-3:]

    def rng(d, n):
        # destination range [a, b) such that a + d, b - 1 + d stay inside [0, n)
        return max(0, -d), min(n, n - d)

    z0, z1 = rng(dz, n3)
    y0, y1 = rng(dy, n2)
    x0, x1 = rng(dx, n1)
    out[..., z0:z1, y0:y1, x0:x1] = x[..., z0 + dz:z1 + dz, y0 + dy:y1 + dy, x0 + dx:x1 + dx]
    return out


def conv3d(x: np.ndarray, W: np.ndarray, b: np.ndarray | None = None) -> np.ndarray:
    """y[o, p] = b[o] + sum_i sum_t W[o, i, t+1] x[i, p + t]."""
    cout, cin = W.shape[:2]
    y = np.zeros((cout,) + x.shape[1:])
    for t in TAPS:
        xs = shifted(x, t)
        w = W[:, :, t[0] + 1, t[1] + 1, t[2] + 1]
        for o in range(cout):
            for i in range(cin):
                y[o] += w[o, i] * xs[i]
    if b is not None:
        y += b[:, None, None, None]
    return y


def conv3d_backward(x: np.ndarray, W: np.ndarray, dy: np.ndarray):
    """Gradients of sum(dy * conv3d(x, W, b)) with respect to x, W and b."""
    cout, cin = W.shape[:2]
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for t in TAPS:
        w = W[:, :, t[0] + 1, t[1] + 1, t[2] + 1]
        neg = (-t[0], -t[1], -t[2])
        dys = shifted(dy, neg)          # dy[o, p - t]
        xs = shifted(x, t)              # x[i, p + t]
        for o in range(cout):
            for i in range(cin):
                dx[i] += w[o, i] * dys[o]
                dW[o, i, t[0] + 1, t[1] + 1, t[2] + 1] = np.sum(dy[o] * xs[i])
    db = dy.reshape(cout, -1).sum(axis=1)
    return dx, dW, db


def forward(params, x: np.ndarray):
    """params = [(W1, b1), ..., (W4, b4)]; ReLU after every layer but the last.
    Returns (output, list of layer inputs, list of pre-activations)."""
    inputs, pre = [], []
    a = x
    for k, (W, b) in enumerate(params):
        inputs.append(a)
        z = conv3d(a, W, b)
        pre.append(z)
        a = np.maximum(z, 0.0) if k + 1 < len(params) else z
    return a, inputs, pre


def loss_and_grads(params, x: np.ndarray, target: np.ndarray):
    """L = mean((out - target)^2) over the points of the single output channel,
    and dL/d(W_k, b_k) by the chain rule through the layers."""
    out, inputs, pre = forward(params, x)
    npts = out.size
    diff = out - target
    L = float(np.sum(diff * diff) / npts)
    g = 2.0 * diff / npts
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        if k + 1 < len(params):
            g = g * (pre[k] > 0.0)
        dx, dW, db = conv3d_backward(inputs[k], params[k][0], g)
        grads[k] = (dW, db)
        g = dx
    return L, grads


def input_channels(u: np.ndarray, dtF: np.ndarray | None, c1, c2, c3, u1: np.ndarray | None = None,
                   u2: np.ndarray | None = None) -> tuple[np.ndarray, float]:
    """The input channels of one sample and its scale s = max |u| (1 for
    u = 0): u / s, dtF / s, the constants c1 + c2 + c3 (three each), and with
    a time history u1 = u^{m-1} (and u2 = u^{m-2}) the first and second
    differences (u - u1) / s and (u - 2 u1 + u2) / s (13 channels)."""
    s = float(np.abs(u).max())
    if s == 0.0:
        s = 1.0
    ch = [u / s, (dtF / s) if dtF is not None else np.zeros_like(u)]
    for v in list(c1) + list(c2) + list(c3):
        ch.append(np.full_like(u, float(v)))
    if u1 is not None:
        ch.append((u - u1) / s)
        ch.append((u - 2.0 * u1 + u2) / s if u2 is not None else np.zeros_like(u))
    return np.stack(ch), s


def extrapolation_base(u: np.ndarray, u1: np.ndarray | None = None, u2: np.ndarray | None = None) -> np.ndarray:
    """What the network's output corrects: u, or the polynomial extrapolation
    in time through the history (2u - u1 with one level, 3u - 3u1 + u2 with
    two: the interpolating polynomial of degree 1 / 2 evaluated one step on)."""
    if u1 is None:
        return u
    if u2 is None:
        return 2.0 * u - u1
    return 3.0 * u - 3.0 * u1 + u2


def adam_step(p: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, step: int, lr: float,
              b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update in place (Kingma & Ba, Algorithm 1), step counted from 1."""
    m *= b1
    m += (1.0 - b1) * g
    v *= b2
    v += (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    p -= lr * mh / (np.sqrt(vh) + eps)
