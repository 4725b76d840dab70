"""Learned initial guess of the CN solves: host-side driver of the warm-start
network whose forward pass, gradients and Adam updates run in libtfde's
kernels (tfde_cnn_* in include/tfde.h).

The network sees, per grid point, (u^m / s, dt F^{m+1/2} / s), nine
coefficients as constant planes and the first and second time differences
(u^m - u^{m-1}) / s, (u^m - 2u^{m-1} + u^{m-2}) / s, s = max |u^m|, and
predicts the correction (u^{m+1} - x_e) / s to the order-2 extrapolation in
time x_e = 3u^m - 3u^{m-1} + u^{m-2} (without a history: to u^m).  The coefficients are delta_1..3 and the logarithms of
the per-axis stiffness scales eta_a k+_a and eta_a k-_a (eta_a = dt /
(2 Gamma(delta_a + 1) h_a^{2 - delta_a}), Eq. (linear_sys)): with q_k
depending on delta alone, these nine numbers fix the discrete operator at any
resolution, so a network trained on one grid applies to finer ones.  Training samples are consecutive time
levels of trajectories that the solver itself computes (tfde_cn_advance);
inference proposes x0 = x_e + s * net(...) to tfde_cn_advance_guess, which
starts from the least-residual point between u^m and x0 (the previous-step
guess whenever x0's FP64 residual is not smaller).

Parameter layout (flat float32, tfde.CNN_PARAMS values): per layer l = 0..3,
W_l[co][ci][tap] (16 x 16 x 27, tap = (dz+1) 9 + (dy+1) 3 + (dx+1)) then
b_l[co] (16); layer 0 reads channels 0..12, layer 3 writes channel 0.
"""
from __future__ import annotations

import math

import numpy as np

from . import tfde as T

CH = 16
NTAP = 27
WSZ = CH * CH * NTAP
PSZ = WSZ + CH
IN_CH = 13   # u, dt F, nine coefficients, two time differences
HIDDEN = 16
CHANNELS = [IN_CH, HIDDEN, HIDDEN, HIDDEN, 1]


def init_params(seed: int, last_scale: float = 0.1) -> np.ndarray:
    """He-normal weights for the real channels (zero elsewhere), zero biases;
    the last layer scaled down so that the untrained guess is close to u^m."""
    rng = np.random.default_rng(seed)
    flat = np.zeros(T.CNN_PARAMS, dtype=np.float32)
    for l, (cin, cout) in enumerate(zip(CHANNELS[:-1], CHANNELS[1:])):
        W = rng.standard_normal((cout, cin, NTAP)) * math.sqrt(2.0 / (NTAP * cin))
        if l == len(CHANNELS) - 2:
            W *= last_scale
        blk = flat[l * PSZ:l * PSZ + WSZ].reshape(CH, CH, NTAP)
        blk[:cout, :cin, :] = W
    return flat


def flat_to_layers(flat: np.ndarray):
    """[(W (cout, cin, 3, 3, 3), b (cout,)), ...] in the layout of the CPU oracle."""
    out = []
    for l, (cin, cout) in enumerate(zip(CHANNELS[:-1], CHANNELS[1:])):
        blk = np.asarray(flat[l * PSZ:l * PSZ + WSZ], dtype=np.float64).reshape(CH, CH, NTAP)
        W = blk[:cout, :cin, :].reshape(cout, cin, 3, 3, 3).copy()
        b = np.asarray(flat[l * PSZ + WSZ:l * PSZ + WSZ + cout], dtype=np.float64).copy()
        out.append((W, b))
    return out


def layers_to_flat(layers) -> np.ndarray:
    flat = np.zeros(T.CNN_PARAMS, dtype=np.float32)
    for l, (W, b) in enumerate(layers):
        cout, cin = W.shape[:2]
        blk = flat[l * PSZ:l * PSZ + WSZ].reshape(CH, CH, NTAP)
        blk[:cout, :cin, :] = W.reshape(cout, cin, NTAP)
        flat[l * PSZ + WSZ:l * PSZ + WSZ + cout] = b
    return flat


def coefficients(params) -> list:
    """(delta_a, log(eta_a k+_a), log(eta_a k-_a)), a = 1..3, of a problem's tfde_params."""
    eta = [T.tfde_host_coefficients(params, a)[3] for a in range(3)]
    return ([float(params.delta[a]) for a in range(3)] + [math.log(eta[a] * params.kp[a]) for a in range(3)]
            + [math.log(eta[a] * params.km[a]) for a in range(3)])


def random_problem(rng):
    """delta ~ U(0.1, 0.9), k+- ~ U(0.5, 2) per axis."""
    return (tuple(rng.uniform(0.1, 0.9, 3)), tuple(rng.uniform(0.5, 2.0, 3)), tuple(rng.uniform(0.5, 2.0, 3)))


def generate_trajectories(n: int, seeds, steps: int, dt, with_source: bool, tol: float = 1e-10,
                          stream=None, device=None):
    """One trajectory per seed: random coefficients, smoothed-noise u0 (seed),
    `steps` chained CN steps of the mixed solver; dt is a number or a list of
    candidates drawn per trajectory.  Returns a list of
    (coef, [u^0 .. u^steps] (device tensors), [dt F^{m+1/2}] or None)."""
    import torch

    import tfde_inputs as inp

    out = []
    for seed in seeds:
        rng = np.random.default_rng(1000 + seed)
        delta, kp, km = random_problem(rng)
        step = float(rng.choice(dt)) if isinstance(dt, (list, tuple)) else float(dt)
        prm = T.make_params((n, n, n), delta, kp, km, step)
        h = T.tfde_assemble(prm, T.TFDE_MIXED, stream)
        try:
            u = torch.from_numpy(inp.smoothed_uniform((n, n, n), seed)).to(device)
            us = [u.clone()]
            Fs = [] if with_source else None
            F = torch.zeros_like(u)
            for m in range(steps):
                th = (m + 0.5) * step
                if with_source:
                    # manufactured-solution source of Example 2 with time factor exp(-t)
                    T.tfde_source_example2(h, -math.exp(-th), -math.exp(-th), F, stream)
                    dtF = torch.empty_like(u)
                    T.tfde_source_example2(h, -step * math.exp(-th), -step * math.exp(-th), dtF, stream)
                    Fs.append(dtF)
                T.tfde_cn_advance(h, u, F if with_source else None, m == 0, tol, stream)
                us.append(u.clone())
            out.append((coefficients(prm), us, Fs))
        finally:
            T.tfde_destroy(h)
    return out


def train(net: int, data, adam_steps: int, batch: int, lr: float, seed: int, stream=None, history: bool = True):
    """Adam on mini-batches of samples (u^m, dt F, coef) -> u^{m+1}, with the
    two previous levels as history when `history` (samples from m = 2 on);
    returns the mean sample loss of every Adam step."""
    samples = []
    for coef, us, Fs in data:
        for m in range(2 if history else 0, len(us) - 1):
            samples.append((coef, us[m], us[m - 1] if history else None, us[m - 2] if history else None,
                            None if Fs is None else Fs[m], us[m + 1]))
    rng = np.random.default_rng(seed)
    hist = []
    for step in range(adam_steps):
        idx = rng.choice(len(samples), size=min(batch, len(samples)), replace=False)
        tot = 0.0
        for i in idx:
            coef, u, u1, u2, dtF, un = samples[i]
            tot += T.tfde_cnn_accumulate_hist(net, u, u1, u2, dtF, coef, un, stream)
        T.tfde_cnn_adam_step(net, lr, stream)
        hist.append(tot / len(idx))
    return hist
