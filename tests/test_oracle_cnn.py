"""Pins of the warm-start network's CPU oracle (no GPU): a library
correlation, closed-form shifts, the adjoint identity and central finite
differences, chosen so that a transposed tap, a flipped sign, a dropped term
or a wrong channel index each fail one of them."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import cnn_oracle as C


def rand_params(rng, chans):
    out = []
    for cin, cout in zip(chans[:-1], chans[1:]):
        W = rng.standard_normal((cout, cin, 3, 3, 3)) / np.sqrt(27 * cin)
        b = 0.1 * rng.standard_normal(cout)
        out.append((W, b))
    return out


def test_single_channel_equals_library_correlation():
    """One input and one output channel: y = correlate(x, w) with zero
    padding, as scipy.ndimage.correlate computes it."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 5, 6, 7))
    W = rng.standard_normal((1, 1, 3, 3, 3))
    y = C.conv3d(x, W)
    ref = ndimage.correlate(x[0], W[0, 0], mode="constant", cval=0.0)
    assert np.allclose(y[0], ref, rtol=0, atol=1e-12)


def test_multichannel_is_sum_of_library_correlations():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 4, 5, 6))
    W = rng.standard_normal((2, 3, 3, 3, 3))
    b = rng.standard_normal(2)
    y = C.conv3d(x, W, b)
    for o in range(2):
        ref = b[o] + sum(ndimage.correlate(x[i], W[o, i], mode="constant", cval=0.0) for i in range(3))
        assert np.allclose(y[o], ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("t", [(0, 0, 1), (0, 1, 0), (1, 0, 0), (-1, 1, -1)])
def test_delta_kernel_is_a_shift(t):
    """W = e_t on channel (0 <- 1): y_0[p] = x_1[p + t] (0 outside), y_1 = 0."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 4, 4, 5))
    W = np.zeros((2, 2, 3, 3, 3))
    W[0, 1, t[0] + 1, t[1] + 1, t[2] + 1] = 1.0
    y = C.conv3d(x, W)
    n3, n2, n1 = x.shape[1:]
    for z in range(n3):
        for yy in range(n2):
            for xx in range(n1):
                q = (z + t[0], yy + t[1], xx + t[2])
                inside = 0 <= q[0] < n3 and 0 <= q[1] < n2 and 0 <= q[2] < n1
                assert y[0, z, yy, xx] == (x[1][q] if inside else 0.0)
    assert not y[1].any()


def test_adjoint_identity_pins_input_gradient():
    """<conv(x), y> = <x, conv^T(y)>: the input gradient of the backward pass
    is the adjoint of the forward convolution."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal((3, 4, 5, 6))
    W = rng.standard_normal((2, 3, 3, 3, 3))
    dy = rng.standard_normal((2, 4, 5, 6))
    dx, _, db = C.conv3d_backward(x, W, dy)
    assert np.isclose(np.sum(C.conv3d(x, W) * dy), np.sum(x * dx), rtol=1e-12)
    assert np.allclose(db, dy.reshape(2, -1).sum(axis=1))


def test_weight_gradient_by_central_differences():
    """sum(dy * conv(x, W)) is linear in W: central differences are exact up to
    rounding, entry by entry."""
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2, 3, 4, 3))
    W = rng.standard_normal((2, 2, 3, 3, 3))
    dy = rng.standard_normal((2, 3, 4, 3))
    _, dW, _ = C.conv3d_backward(x, W, dy)
    h = 1e-3
    for idx in [(0, 0, 0, 0, 0), (1, 0, 2, 1, 0), (0, 1, 1, 1, 1), (1, 1, 0, 2, 2), (0, 1, 2, 0, 1)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += h
        Wm[idx] -= h
        fd = (np.sum(dy * C.conv3d(x, Wp)) - np.sum(dy * C.conv3d(x, Wm))) / (2 * h)
        assert np.isclose(dW[idx], fd, rtol=1e-9, atol=1e-9)


def test_network_gradient_by_central_differences():
    """Four layers with ReLU, MSE loss: backpropagated gradients match central
    differences of the loss on a tiny grid."""
    rng = np.random.default_rng(6)
    params = rand_params(rng, [3, 4, 4, 4, 1])
    x = rng.standard_normal((3, 3, 4, 4))
    target = rng.standard_normal((1, 3, 4, 4))
    L, grads = C.loss_and_grads(params, x, target)
    h = 1e-6
    for k in range(4):
        W, b = params[k]
        for idx in [(0, 0, 1, 1, 1), (0, W.shape[1] - 1, 2, 0, 1)]:
            W[idx] += h
            Lp, _ = C.loss_and_grads(params, x, target)
            W[idx] -= 2 * h
            Lm, _ = C.loss_and_grads(params, x, target)
            W[idx] += h
            assert np.isclose(grads[k][0][idx], (Lp - Lm) / (2 * h), rtol=1e-5, atol=1e-9)
        b[0] += h
        Lp, _ = C.loss_and_grads(params, x, target)
        b[0] -= 2 * h
        Lm, _ = C.loss_and_grads(params, x, target)
        b[0] += h
        assert np.isclose(grads[k][1][0], (Lp - Lm) / (2 * h), rtol=1e-5, atol=1e-9)


def test_adam_first_step_moves_by_learning_rate():
    """Adam's first bias-corrected step is lr * g / (|g| + eps): a move of
    about lr against the sign of every gradient entry."""
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    C.adam_step(p, g, m, v, 1, 0.01)
    assert np.allclose(p, [1.0 - 0.01, -2.0 + 0.01, 0.5 - 0.01 * 1e-3 / (1e-3 + 1e-8)], rtol=1e-12)


def test_adam_three_steps_against_unrolled_moment_averages():
    """Three Adam steps with a different gradient each step, against the
    unrolled form of the moments (Kingma & Ba, Sec. 3: m_t = (1 - b1)
    sum_i b1^(t-i) g_i, likewise v_t with g_i^2 and b2), evaluated in exact
    rational arithmetic with b1 = 1/2, b2 = 3/4 and eps = 0: a wrong decay,
    bias-correction exponent or moment update from step 2 on fails."""
    from fractions import Fraction as Fr
    b1, b2, lr = 0.5, 0.75, 0.125
    gs = [np.array([0.5, -2.0, 1.0]), np.array([-1.0, 4.0, 1.0]), np.array([0.25, 1.0, -3.0])]
    p = np.array([1.0, -1.0, 0.0])
    m, v = np.zeros(3), np.zeros(3)
    expect = [Fr(1), Fr(-1), Fr(0)]
    for t in range(1, 4):
        C.adam_step(p, gs[t - 1], m, v, t, lr, b1=b1, b2=b2, eps=0.0)
        for e in range(3):
            mt = sum((1 - Fr(1, 2)) * Fr(1, 2) ** (t - i) * Fr(gs[i - 1][e]) for i in range(1, t + 1))
            vt = sum((1 - Fr(3, 4)) * Fr(3, 4) ** (t - i) * Fr(gs[i - 1][e]) ** 2 for i in range(1, t + 1))
            mh = mt / (1 - Fr(1, 2) ** t)
            vh = vt / (1 - Fr(3, 4) ** t)
            expect[e] -= Fr(lr) * mh / Fr(float(np.sqrt(float(vh))))
        np.testing.assert_allclose(p, [float(x) for x in expect], rtol=1e-14, atol=1e-15)


def test_adam_constant_gradient_moves_lr_per_step():
    """With the same gradient at every step the bias-corrected moments equal
    g and g^2 exactly, so every step moves each weight by lr * g / (|g| + eps)."""
    g = np.array([0.3, -4.0, 2.0])
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 6):
        C.adam_step(p, g, m, v, t, 0.01)
    np.testing.assert_allclose(p, -5 * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_input_channels_layout():
    u = np.arange(24, dtype=float).reshape(2, 3, 4) - 5.0
    ch, s = C.input_channels(u, 2 * u, (0.1, 0.2, 0.3), (1, 2, 3), (4, 5, 6))
    assert s == 18.0 and ch.shape == (11, 2, 3, 4)
    assert np.allclose(ch[0], u / 18.0) and np.allclose(ch[1], 2 * u / 18.0)
    assert np.allclose(ch[2:11, 0, 0, 0], [0.1, 0.2, 0.3, 1, 2, 3, 4, 5, 6])


def test_history_channels_and_extrapolation_base():
    """The history channels are the first and second time differences, and
    the base is the interpolating polynomial through the last levels
    evaluated one step ahead: exact for data quadratic (linear) in time."""
    t = np.arange(4.0)
    rng = np.random.default_rng(0)
    a, b, c = (rng.standard_normal((2, 3, 2)) for _ in range(3))
    lev = [a + b * tt + c * tt * tt for tt in t]        # u^{m-2}, u^{m-1}, u^m, u^{m+1}
    np.testing.assert_allclose(C.extrapolation_base(lev[2], lev[1], lev[0]), lev[3], rtol=1e-12, atol=1e-12)
    lin = [a + b * tt for tt in t]
    np.testing.assert_allclose(C.extrapolation_base(lin[2], lin[1]), lin[3], rtol=1e-12, atol=1e-12)
    ch, s = C.input_channels(lev[2], None, (0.1,) * 3, (1,) * 3, (2,) * 3, lev[1], lev[0])
    assert ch.shape[0] == 13
    np.testing.assert_allclose(ch[11] * s, lev[2] - lev[1])
    np.testing.assert_allclose(ch[12] * s, 2 * c)   # second difference of a quadratic: 2c (unit steps)
