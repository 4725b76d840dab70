"""GPU parity of the warm-start network (tfde_cnn_*): the tensor-core
convolutions, the backward pass and the Adam update against the CPU oracle,
and the guard that keeps the previous-step guess when the proposed one is not
better (tfde_cn_advance_guess)."""
import numpy as np
import pytest

from oracle import cnn_oracle as C
from oracle import tfde_oracle as o
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


@pytest.fixture(scope="module")
def W():
    from paper_2511_21198_gb300 import warmstart
    return warmstart


def bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_forward(layers, x):
    """The oracle's forward pass with the storage precision of the kernels:
    BF16 inputs, weights and hidden activations, exact accumulation."""
    a = bf16(x)
    for k, (Wt, b) in enumerate(layers):
        z = C.conv3d(a, bf16(Wt), b.astype(np.float32).astype(np.float64))
        a = bf16(np.maximum(z, 0.0)) if k + 1 < len(layers) else z
    return a


def pad_channels(x, cin):
    """Zero channels up to the network's input width (the history channels of
    a call without a history)."""
    if x.shape[0] >= cin:
        return x
    return np.concatenate([x, np.zeros((cin - x.shape[0],) + x.shape[1:])])


def random_net(W, seed):
    flat = W.init_params(seed, last_scale=1.0)
    rng = np.random.default_rng(seed + 1)
    for l in range(4):
        cout = W.CHANNELS[l + 1]
        flat[l * W.PSZ + W.WSZ:l * W.PSZ + W.WSZ + cout] = 0.05 * rng.standard_normal(cout)
    return flat


@pytest.mark.parametrize("n", [(10, 7, 5), (33, 4, 6)])
def test_forward_matches_oracle(T, W, n):
    """x0 - u = s * net(...) on grids whose 128-slot tiles span several lines
    and planes with ragged ends."""
    flat = random_net(W, 3)
    net = T.tfde_cnn_create(n)
    try:
        T.tfde_cnn_set_params(net, flat)
        shape = tuple(reversed(n))
        u = inp.uniform_vector(shape, 5) - 0.3
        dtF = 0.1 * inp.uniform_vector(shape, 6)
        coef = [0.3, 0.6, 0.8, 1.0, 1.5, 0.7, 0.5, 2.0, 1.2]
        x0 = to_dev(np.zeros(shape))
        T.tfde_cnn_predict(net, to_dev(u), to_dev(dtF), coef, x0)
        x, s = C.input_channels(u, dtF, coef[0:3], coef[3:6], coef[6:9])
        ref = bf16_forward(W.flat_to_layers(flat), pad_channels(x, W.CHANNELS[0]))[0]
        got = (to_host(x0) - u) / s
        assert relerr(got, ref) < 1e-2
        assert np.abs(got - ref).max() <= 3e-2 * np.abs(ref).max()
    finally:
        T.tfde_cnn_destroy(net)


def test_forward_with_history_matches_oracle(T, W):
    """The history channels (first and second time differences) and the
    extrapolation base: x0 = (3u - 3u1 + u2) + s * net(...) against the
    oracle's forward pass on the BF16 storage of the 13 input channels."""
    n = (10, 7, 5)
    flat = random_net(W, 4)
    net = T.tfde_cnn_create(n)
    try:
        T.tfde_cnn_set_params(net, flat)
        shape = tuple(reversed(n))
        u = inp.uniform_vector(shape, 5) - 0.3
        u1 = u - 0.05 * inp.uniform_vector(shape, 7)
        u2 = u1 - 0.04 * inp.uniform_vector(shape, 8)
        coef = [0.3, 0.6, 0.8, 1.0, 1.5, 0.7, 0.5, 2.0, 1.2]
        x0 = to_dev(np.zeros(shape))
        T.tfde_cnn_predict_hist(net, to_dev(u), to_dev(u1), to_dev(u2), None, coef, x0)
        x, s = C.input_channels(u, None, coef[0:3], coef[3:6], coef[6:9], u1, u2)
        ref = bf16_forward(W.flat_to_layers(flat), x)[0]
        got = (to_host(x0) - C.extrapolation_base(u, u1, u2)) / s
        assert relerr(got, ref) < 1e-2
        assert np.abs(got - ref).max() <= 3e-2 * np.abs(ref).max()
    finally:
        T.tfde_cnn_destroy(net)


def bf16_backward(layers, x, target):
    """The oracle's backpropagation (conv3d / conv3d_backward) with the storage
    precision of the kernels: BF16 inputs, weights and hidden activations,
    the output gradient 2 (out - target) / N and every back-propagated
    pre-activation gradient rounded to BF16 (the ReLU mask taken from the
    stored activation), sums exact.  Returns (loss, [(dW, db)] per layer)."""
    Wb = [bf16(Wt) for Wt, _ in layers]
    bb = [b.astype(np.float32).astype(np.float64) for _, b in layers]
    acts = [bf16(x)]
    for k in range(len(layers)):
        z = C.conv3d(acts[-1], Wb[k], bb[k])
        acts.append(bf16(np.maximum(z, 0.0)) if k + 1 < len(layers) else z)
    out = acts[-1]
    npts = out[0].size
    diff = out - target
    L = float(np.sum(diff * diff) / npts)
    g = bf16(2.0 * diff / npts)
    grads = [None] * len(layers)
    for k in range(len(layers) - 1, -1, -1):
        dx, dW, db = C.conv3d_backward(acts[k], Wb[k], g)
        grads[k] = (dW, db)
        if k > 0:
            g = bf16(dx * (acts[k] > 0.0))
    return L, grads


def test_gradients_match_oracle(T, W):
    """One accumulated sample: loss and the gradient of every layer against the
    oracle's backpropagation taken with the kernels' BF16 storage of inputs,
    weights, activations and back-propagated gradients, element by element
    (a wrong tap, channel or sign moves its entries by far more than the
    FP32 accumulation and rare BF16 rounding-boundary differences)."""
    n = (12, 9, 6)
    flat = random_net(W, 7)
    net = T.tfde_cnn_create(n)
    try:
        T.tfde_cnn_set_params(net, flat)
        shape = tuple(reversed(n))
        u = inp.uniform_vector(shape, 8) - 0.5
        un = u + 0.05 * (inp.uniform_vector(shape, 9) - 0.5)
        coef = [0.5, 0.5, 0.5, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0]
        loss = T.tfde_cnn_accumulate(net, to_dev(u), None, coef, to_dev(un))
        g = W.flat_to_layers(T.tfde_cnn_get_grads(net))
        x, s = C.input_channels(u, None, coef[0:3], coef[3:6], coef[6:9])
        L, ref = bf16_backward(W.flat_to_layers(flat), pad_channels(x, W.CHANNELS[0]), (un - u)[None] / s)
        assert abs(loss - L) <= 1e-4 * L
        for k in range(4):
            for got, want in ((g[k][0], ref[k][0]), (g[k][1], ref[k][1])):
                scale = np.abs(want).max()
                assert scale > 0
                assert np.abs(got - want).max() <= 2e-3 * scale, (k, np.abs(got - want).max() / scale)
                assert relerr(got, want) < 2e-3
    finally:
        T.tfde_cnn_destroy(net)


def test_adam_step_matches_oracle(T, W):
    """Two accumulated samples then one Adam step: the parameters move as the
    oracle's Adam with the averaged gradient."""
    n = (8, 8, 8)
    flat = random_net(W, 11)
    net = T.tfde_cnn_create(n)
    try:
        T.tfde_cnn_set_params(net, flat)
        shape = tuple(reversed(n))
        coef = [0.4, 0.5, 0.6, 1.0, 1.0, 1.0, 0.8, 0.8, 0.8]
        for sd in (1, 2):
            u = inp.uniform_vector(shape, 20 + sd)
            T.tfde_cnn_accumulate(net, to_dev(u), None, coef, to_dev(1.01 * u))
        g = T.tfde_cnn_get_grads(net).astype(np.float64) / 2.0
        T.tfde_cnn_adam_step(net, 1e-3)
        got = T.tfde_cnn_get_params(net).astype(np.float64)
        want = flat.astype(np.float64).copy()
        C.adam_step(want, g, np.zeros_like(want), np.zeros_like(want), 1, 1e-3)
        assert np.abs(got - want).max() <= 1e-6
        assert not T.tfde_cnn_get_grads(net).any()
    finally:
        T.tfde_cnn_destroy(net)


def test_training_reduces_loss(T, W):
    """Adam on trajectories the solver generates (n = 16) lowers the loss."""
    import torch
    data = W.generate_trajectories(16, [100, 101, 102], 4, 0.01, with_source=True, device="cuda")
    net = T.tfde_cnn_create((16, 16, 16))
    try:
        T.tfde_cnn_set_params(net, W.init_params(0))
        hist = W.train(net, data, 80, 4, 3e-3, 0)
        assert np.mean(hist[-10:]) < 0.5 * np.mean(hist[:5])
    finally:
        T.tfde_cnn_destroy(net)
        torch.cuda.synchronize()


def test_advance_guess_keeps_better_start(T):
    """tfde_cn_advance_guess: the start is the least-residual point of the
    line from u^{m-1} towards the guess, so a poor guess never starts worse
    than u^{m-1} and the step equals tfde_cn_advance; the converged solution
    as guess is taken and needs (almost) no iterations."""
    n = (24, 16, 32)
    d, kp, km = (0.3, 0.6, 0.8), (1.0,) * 3, (0.5,) * 3
    prm = T.make_params(n, d, kp, km, 0.02)
    ha = T.tfde_assemble(prm, T.TFDE_MIXED)
    hb = T.tfde_assemble(prm, T.TFDE_MIXED)
    try:
        u0 = inp.smoothed_uniform(tuple(reversed(n)), 2)
        ua, ub = to_dev(u0), to_dev(u0)
        ia = T.tfde_cn_advance(ha, ua, None, True, 1e-12)
        worse = to_dev(u0 + 0.5)
        ib, used = T.tfde_cn_advance_guess(hb, ub, None, worse, True, 1e-12)
        assert ib.relres0 <= ia.relres0 * (1 + 1e-12)
        assert relerr(to_host(ub), to_host(ua)) < 1e-10
        # next step: the exact solution as guess
        op = o.Problem(n=n, delta=d, kp=kp, km=km, dt=0.02)
        b = o.rhs(op, to_host(ua), None)
        tau = o.build_tau(op)
        xo, _ = o.gmres_left(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, to_host(ua), 1e-14,
                             4000, restart=20, criterion="true")
        ic, used = T.tfde_cn_advance_guess(hb, ub, None, to_dev(xo), False, 1e-10)
        assert used and ic.iters <= 1 and ic.relres <= 1e-10
        assert relerr(to_host(ub), xo) < 1e-9
    finally:
        T.tfde_destroy(ha)
        T.tfde_destroy(hb)


def test_advance_guess_blend_starts_at_least_residual_point(T):
    """A guess that overshoots the next solution and carries a perturbation
    gives an intermediate blend coefficient: the start u + c (x0 - u) with
    c = <r, A d> / ||A d||^2 (d = x0 - u, r = b - A u).  Its initial relative
    residual, recomputed from the FP64 GPU operator of Eq. (linear_sys), must
    equal the step's relres0, and the guess must count as used."""
    n = (24, 16, 32)
    d, kp, km = (0.3, 0.6, 0.8), (1.0,) * 3, (0.5,) * 3
    prm = T.make_params(n, d, kp, km, 0.02)
    h = T.tfde_assemble(prm, T.TFDE_MIXED)
    h64 = T.tfde_assemble(prm, T.TFDE_FP64)
    try:
        shape = tuple(reversed(n))
        u = to_dev(inp.smoothed_uniform(shape, 3))
        T.tfde_cn_advance(h, u, None, True, 1e-12)          # chain established, u = u^1
        u1 = to_host(u)
        xn = to_dev(np.zeros(shape))
        T.tfde_cn_step(h64, to_dev(u1), None, None, xn, 1e-13)   # the next solution
        x_next = to_host(xn)
        # overshoot the step by 1.5 (alone: least residual at c = 2/3) plus a
        # smooth perturbation, so that the best start is an interior point
        dx = x_next - u1
        guess = u1 + 1.5 * dx + 0.05 * np.abs(dx).max() * (inp.smoothed_uniform(shape, 4) - 0.5)

        def A64(v, op=T.TFDE_OP_A):
            y = to_dev(np.zeros(shape))
            T.tfde_matvec(h64, op, to_dev(v), y)
            return to_host(y)
        b = A64(u1, T.TFDE_OP_RHS)
        r = b - A64(u1)
        Ad = A64(guess - u1)
        c = float(np.sum(r * Ad) / np.sum(Ad * Ad))
        assert 0.3 < c < 0.95, c
        rel0 = float(np.linalg.norm(r - c * Ad) / np.linalg.norm(b))
        info, used = T.tfde_cn_advance_guess(h, u, None, to_dev(guess), False, 1e-10)
        assert used == 1
        assert abs(info.relres0 - rel0) <= 1e-6 * rel0, (info.relres0, rel0)
        assert info.relres <= 1e-10
        assert relerr(to_host(u), x_next) < 1e-8
    finally:
        T.tfde_destroy(h)
        T.tfde_destroy(h64)


def test_trained_network_gain_is_measured_and_harmless(T, W):
    """What the trained network gains over the method without it: a network
    trained on the solver's own trajectories (n = 16, with the time history)
    proposes the starts of 10 CN steps at n = 24; the same steps from the
    previous-step guess.  Both runs reach the same solutions (the FP64
    residual test decides), the network's blended starts never have a larger
    residual than u^m, and the iteration counts of both are recorded.  On
    this problem class the network does not save iterations: its BF16
    correction is rough at the grid scale, which the stiffness terms amplify
    in the residual (the measured averages are printed)."""
    import torch
    data = W.generate_trajectories(16, list(range(100, 116)), 6, [0.01, 0.02], with_source=False, device="cuda")
    net = T.tfde_cnn_create((16, 16, 16))
    try:
        T.tfde_cnn_set_params(net, W.init_params(0))
        W.train(net, data, 150, 4, 3e-3, 0)
        params = T.tfde_cnn_get_params(net)
    finally:
        T.tfde_cnn_destroy(net)
    n, dt = (24, 24, 24), 0.02
    prm = T.make_params(n, (0.3, 0.6, 0.8), (1.0,) * 3, (0.5,) * 3, dt)
    coef = W.coefficients(prm)
    ne = T.tfde_cnn_create(n)
    ha = T.tfde_assemble(prm, T.TFDE_MIXED)
    hb = T.tfde_assemble(prm, T.TFDE_MIXED)
    try:
        T.tfde_cnn_set_params(ne, params)
        u0 = to_dev(inp.smoothed_uniform(tuple(reversed(n)), 5))
        ua, ub = u0.clone(), u0.clone()
        T.tfde_cn_advance(ha, ua, None, True, 1e-10)
        T.tfde_cn_advance(hb, ub, None, True, 1e-10)
        hist = [u0.clone()]
        x0 = torch.empty_like(ub)
        ia = ib = 0
        for m in range(10):
            a = T.tfde_cn_advance(ha, ua, None, False, 1e-10)
            T.tfde_cnn_predict_hist(ne, ub, hist[-1], hist[-2] if len(hist) > 1 else None, None, coef, x0)
            prev = ub.clone()
            b, used = T.tfde_cn_advance_guess(hb, ub, None, x0, False, 1e-10)
            hist = [hist[-1], prev]
            assert b.relres0 <= a.relres0 * (1 + 1e-6)   # never a worse start than u^m
            assert a.relres <= 1e-10 and b.relres <= 1e-10
            assert relerr(to_host(ub), to_host(ua)) < 1e-8
            ia += a.iters
            ib += b.iters
        print(f"iterations per step: previous-step guess {ia / 10:.2f}, network {ib / 10:.2f}")
        assert ib <= ia + 30   # the guard bounds the harm to a few iterations per step
    finally:
        T.tfde_cnn_destroy(ne)
        T.tfde_destroy(ha)
        T.tfde_destroy(hb)
