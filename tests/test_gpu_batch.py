"""GPU parity of the batched solve (tfde_batch_*): problems of uneven size and
coefficients advanced together in lock step must give, problem by problem,
the same CN trajectory as the single-problem solvers (and the oracle)."""
import numpy as np
import pytest

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


def small_batch(count, seed, sizes=(8, 16, 24, 32, 40)):
    """Uneven problems in the recipe of the batched workload, on small grids:
    every axis size drawn separately, delta ~ U(0.1, 0.9), k+- ~ U(0.5, 2)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = tuple(int(v) for v in rng.choice(sizes, 3))
        out.append(dict(n=n, delta=tuple(rng.uniform(0.1, 0.9, 3)), kp=tuple(rng.uniform(0.5, 2.0, 3)),
                        km=tuple(rng.uniform(0.5, 2.0, 3))))
    return out


def test_batch_first_step_matches_oracle(T):
    """One batched step from smoothed-noise data equals, for every problem,
    the oracle's left-preconditioned GMRES solution of its CN system."""
    probs = small_batch(4, 11, sizes=(8, 16, 24))
    dt = 0.1
    params = [T.make_params(p["n"], p["delta"], p["kp"], p["km"], dt) for p in probs]
    B = T.tfde_batch_create(params, 20)
    try:
        u0 = [inp.smoothed_uniform(tuple(reversed(p["n"])), 20 + i) for i, p in enumerate(probs)]
        us = [to_dev(u) for u in u0]
        infos = T.tfde_batch_cn_advance(B, us, None, True, 1e-12)
        for i, p in enumerate(probs):
            op = o.Problem(n=p["n"], delta=p["delta"], kp=p["kp"], km=p["km"], dt=dt)
            b = o.rhs(op, u0[i], None)
            tau = o.build_tau(op)
            xo, _ = o.gmres_left(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, u0[i], 1e-14, 4000,
                                 restart=20, criterion="true")
            assert infos[i].relres <= 1e-12 and infos[i].fallback == 0
            assert relerr(to_host(us[i]), xo) < 1e-10
    finally:
        T.tfde_batch_destroy(B)


def test_batch_trajectory_matches_single_problem_fp64(T):
    """Six uneven problems (one symmetric), 5 chained steps with sources on
    two of them: the batched trajectories equal the all-FP64 single-problem
    advance at tight residuals."""
    probs = small_batch(6, 12)
    probs[2]["km"] = probs[2]["kp"]          # a symmetric one rides along
    dt = 0.05
    params = [T.make_params(p["n"], p["delta"], p["kp"], p["km"], dt) for p in probs]
    B = T.tfde_batch_create(params, 20)
    singles = [T.tfde_assemble(pp, T.TFDE_FP64) for pp in params]
    try:
        u0 = [inp.smoothed_uniform(tuple(reversed(p["n"])), 30 + i) for i, p in enumerate(probs)]
        ub = [to_dev(u) for u in u0]
        us = [to_dev(u) for u in u0]
        Fs = [None] * len(probs)
        Fs[1] = to_dev(inp.uniform_vector(tuple(reversed(probs[1]["n"])), 7))
        Fs[4] = to_dev(inp.uniform_vector(tuple(reversed(probs[4]["n"])), 8))
        for m in range(5):
            infos = T.tfde_batch_cn_advance(B, ub, Fs, m == 0, 1e-12)
            for i in range(len(probs)):
                T.tfde_cn_advance(singles[i], us[i], Fs[i], m == 0, 1e-13)
                assert infos[i].relres <= 1e-12
        for i in range(len(probs)):
            assert relerr(to_host(ub[i]), to_host(us[i])) < 1e-10
    finally:
        T.tfde_batch_destroy(B)
        for h in singles:
            T.tfde_destroy(h)


def test_batch_large_uneven_sizes(T):
    """Sizes of the batched workload (32..128 per axis, tiles with ragged
    tails in both the row and the line direction) at the metric tolerance."""
    probs = inp.batched_instances(count=5, seed=4)
    dt = 0.1
    params = [T.make_params(p["n"], p["delta"], p["kp"], p["km"], dt) for p in probs]
    B = T.tfde_batch_create(params, 20)
    singles = [T.tfde_assemble(pp, T.TFDE_FP64) for pp in params]
    try:
        u0 = [inp.smoothed_uniform(tuple(reversed(p["n"])), 40 + i) for i, p in enumerate(probs)]
        ub = [to_dev(u) for u in u0]
        us = [to_dev(u) for u in u0]
        for m in range(2):
            infos = T.tfde_batch_cn_advance(B, ub, None, m == 0, 1e-10)
            for i in range(len(probs)):
                T.tfde_cn_advance(singles[i], us[i], None, m == 0, 1e-13)
                assert infos[i].relres <= 1e-10 and infos[i].fallback == 0
        for i in range(len(probs)):
            # both solutions within their residual bounds of the exact one
            assert relerr(to_host(ub[i]), to_host(us[i])) < 1e-8
    finally:
        T.tfde_batch_destroy(B)
        for h in singles:
            T.tfde_destroy(h)


def test_batch_guess_order_same_trajectory(T):
    """Batched chained steps with the corrected extrapolated guess (order 3)
    reach the trajectories of the previous-step guess at tight residuals, in
    fewer iterations once the history is built."""
    probs = small_batch(5, 13, sizes=(16, 24, 32))
    dt = 0.05
    params = [T.make_params(p["n"], p["delta"], p["kp"], p["km"], dt) for p in probs]
    B0 = T.tfde_batch_create(params, 20)
    B3 = T.tfde_batch_create(params, 20)
    T.tfde_batch_set_guess_order(B3, 3)
    try:
        u0 = [inp.smoothed_uniform(tuple(reversed(p["n"])), 40 + i) for i, p in enumerate(probs)]
        ua = [to_dev(u) for u in u0]
        ub = [to_dev(u) for u in u0]
        it0 = it3 = 0
        for m in range(8):
            ia = T.tfde_batch_cn_advance(B0, ua, None, m == 0, 1e-12)
            ib = T.tfde_batch_cn_advance(B3, ub, None, m == 0, 1e-12)
            assert all(i.relres <= 1e-12 for i in ia) and all(i.relres <= 1e-12 for i in ib)
            if m >= 3:
                it0 += sum(i.iters for i in ia)
                it3 += sum(i.iters for i in ib)
        for a, b in zip(ua, ub):
            assert relerr(to_host(a), to_host(b)) < 1e-10
        assert it3 < it0
        # once every problem has two history levels and its mass term, the
        # right-hand sides and guesses run grouped (order 0 never does)
        assert T.tfde_batch_grouped_prepares(B3) >= 3 and T.tfde_batch_grouped_prepares(B0) == 0
        with pytest.raises(T.TfdeError):
            T.tfde_batch_set_guess_order(B3, 4)
    finally:
        T.tfde_batch_destroy(B0)
        T.tfde_batch_destroy(B3)


def test_batch_argument_errors(T):
    good = T.make_params((16, 16, 16), (0.5,) * 3, (1.0,) * 3, (0.5,) * 3, 0.1)
    with pytest.raises(T.TfdeError) as e:
        T.tfde_batch_create([], 20)
    assert e.value.status == T.TFDE_EINVAL
    with pytest.raises(T.TfdeError) as e:
        T.tfde_batch_create([good, T.make_params((12, 16, 16), (0.5,) * 3, (1.0,) * 3, (1.0,) * 3, 0.1)], 20)
    assert e.value.status == T.TFDE_EUNSUPPORTED
    B = T.tfde_batch_create([good, good], 20)
    try:
        assert T.load().tfde_batch_count(B) == 2
        u = to_dev(np.zeros((16, 16, 16)))
        with pytest.raises(T.TfdeError) as e:
            T.tfde_batch_cn_advance(B, [u, u], None, True, 1e-8)
        assert e.value.status == T.TFDE_EINVAL
        # zero data: every problem converges at once with a zero solution
        v = to_dev(np.zeros((16, 16, 16)))
        infos = T.tfde_batch_cn_advance(B, [u, v], None, True, 1e-8)
        assert all(i.iters == 0 for i in infos)
        assert float(np.abs(to_host(u)).max()) == 0.0
    finally:
        T.tfde_batch_destroy(B)


@pytest.mark.parametrize("spectral", [True, False], ids=["eigenbasis", "grid"])
def test_batch_both_bases_match_oracle(T, spectral):
    """The batched GMRES cycles in the sine-transform eigenbasis (grouped
    Lambda^{-1} S_N A S_N passes, one forward and one backward transform per
    cycle; the default) and in the grid basis: one step of five uneven
    problems (ragged tiles, a short restart) against the oracle's solutions."""
    probs = small_batch(5, 13, sizes=(8, 16, 24, 40, 136))
    dt = 0.05
    params = [T.make_params(p["n"], p["delta"], p["kp"], p["km"], dt) for p in probs]
    B = T.tfde_batch_create(params, 6)
    try:
        T.tfde_batch_set_spectral_inner(B, spectral)
        u0 = [inp.smoothed_uniform(tuple(reversed(p["n"])), 40 + i) for i, p in enumerate(probs)]
        us = [to_dev(u) for u in u0]
        infos = T.tfde_batch_cn_advance(B, us, None, True, 1e-12)
        for i, p in enumerate(probs):
            op = o.Problem(n=p["n"], delta=p["delta"], kp=p["kp"], km=p["km"], dt=dt)
            b = o.rhs(op, u0[i], None)
            tau = o.build_tau(op)
            xo, _ = o.gmres_left(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, u0[i], 1e-14, 4000,
                                 restart=20, criterion="true")
            assert infos[i].relres <= 1e-12 and infos[i].fallback == 0, (i, infos[i].relres)
            assert relerr(to_host(us[i]), xo) < 1e-10, i
    finally:
        T.tfde_batch_destroy(B)


def test_batch_graph_cycle_and_host_loop_agree(T):
    """The batched eigenbasis cycle as one graph launch per cycle (step index,
    Givens updates and loop condition on the device) and driven step by step
    from the host (the path taken while every tensor-core launch is timed)
    give the same iteration counts and solutions, both matching the oracle."""
    probs = small_batch(4, 17, sizes=(8, 16, 24, 32))
    dt = 0.1
    params = [T.make_params(p["n"], p["delta"], p["kp"], p["km"], dt) for p in probs]
    u0 = [inp.smoothed_uniform(tuple(reversed(p["n"])), 60 + i) for i, p in enumerate(probs)]
    runs = {}
    for timed in (False, True):
        B = T.tfde_batch_create(params, 8)
        try:
            T.tfde_stats_reset(time_tc=timed)
            us = [to_dev(u) for u in u0]
            infos = T.tfde_batch_cn_advance(B, us, None, True, 1e-12)
            runs[timed] = ([i.iters for i in infos], [to_host(u) for u in us])
            graph_cycles = T.tfde_batch_graph_cycles(B)
            assert (graph_cycles == 0) if timed else (graph_cycles > 0), (timed, graph_cycles)
        finally:
            T.tfde_stats_reset(time_tc=False)
            T.tfde_batch_destroy(B)
    assert runs[False][0] == runs[True][0]
    for i, p in enumerate(probs):
        op = o.Problem(n=p["n"], delta=p["delta"], kp=p["kp"], km=p["km"], dt=dt)
        b = o.rhs(op, u0[i], None)
        tau = o.build_tau(op)
        xo, _ = o.gmres_left(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, u0[i], 1e-14, 4000,
                             restart=20, criterion="true")
        assert relerr(runs[False][1][i], xo) < 1e-10 and relerr(runs[True][1][i], xo) < 1e-10, i


def symmetric_batch(count, seed, sizes):
    """Uneven symmetric problems (k+ = k- on every axis, drawn per axis)."""
    probs = small_batch(count, seed, sizes=sizes)
    for p in probs:
        p["km"] = p["kp"]
    return probs


def oracle_step(p, u0, dt):
    """The oracle's CN solution from u0: PCG (Sec. 3.1) when the problem is
    symmetric, left-preconditioned GMRES (Sec. 3.2) otherwise."""
    op = o.Problem(n=p["n"], delta=p["delta"], kp=p["kp"], km=p["km"], dt=dt)
    b = o.rhs(op, u0, None)
    tau = o.build_tau(op)
    if tuple(p["kp"]) == tuple(p["km"]):
        x, _ = o.pcg(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, u0.copy(), 1e-14, 4000)
    else:
        x, _ = o.gmres_left(lambda v: o.apply_A(op, v), lambda r: o.apply_Pinv(tau, r), b, u0, 1e-14, 4000,
                            restart=20, criterion="true")
    return x


def test_batch_symmetric_problems_take_pcg(T):
    """Five uneven symmetric problems (ragged tiles): one batched step runs
    their inner solves as the lock-step PCG (no GMRES cycle at all) and each
    solution equals the oracle's PCG solution of its CN system."""
    probs = symmetric_batch(5, 19, sizes=(8, 16, 24, 40, 136))
    dt = 0.05
    params = [T.make_params(p["n"], p["delta"], p["kp"], p["km"], dt) for p in probs]
    B = T.tfde_batch_create(params, 20)
    try:
        u0 = [inp.smoothed_uniform(tuple(reversed(p["n"])), 70 + i) for i, p in enumerate(probs)]
        us = [to_dev(u) for u in u0]
        infos = T.tfde_batch_cn_advance(B, us, None, True, 1e-12)
        sweeps = sum(i.refine_sweeps for i in infos)
        assert T.tfde_batch_pcg_solves(B) == sweeps > 0
        assert T.tfde_batch_graph_cycles(B) == 0
        for i, p in enumerate(probs):
            assert infos[i].relres <= 1e-12 and infos[i].fallback == 0, (i, infos[i].relres)
            assert relerr(to_host(us[i]), oracle_step(p, u0[i], dt)) < 1e-10, i
    finally:
        T.tfde_batch_destroy(B)


def test_batch_mixed_symmetry_pcg_and_gmres(T):
    """Three symmetric and three non-symmetric problems in one batch: the
    symmetric ones take the batched PCG, the others the batched GMRES cycles,
    in the same refinement sweeps; every solution matches the oracle's."""
    sym = symmetric_batch(3, 23, sizes=(8, 16, 24, 32))
    nonsym = small_batch(3, 29, sizes=(8, 16, 24, 32))
    probs = [sym[0], nonsym[0], sym[1], nonsym[1], sym[2], nonsym[2]]
    dt = 0.1
    params = [T.make_params(p["n"], p["delta"], p["kp"], p["km"], dt) for p in probs]
    B = T.tfde_batch_create(params, 20)
    try:
        u0 = [inp.smoothed_uniform(tuple(reversed(p["n"])), 80 + i) for i, p in enumerate(probs)]
        us = [to_dev(u) for u in u0]
        infos = T.tfde_batch_cn_advance(B, us, None, True, 1e-12)
        assert T.tfde_batch_pcg_solves(B) == sum(infos[i].refine_sweeps for i in (0, 2, 4))
        assert T.tfde_batch_graph_cycles(B) > 0
        for i, p in enumerate(probs):
            assert infos[i].relres <= 1e-12 and infos[i].fallback == 0, (i, infos[i].relres)
            assert relerr(to_host(us[i]), oracle_step(p, u0[i], dt)) < 1e-10, i
    finally:
        T.tfde_batch_destroy(B)


def test_batch_symmetric_pcg_chained_steps_and_toggle(T):
    """Four chained steps of a symmetric batch with the batched PCG, and the
    same steps with it switched off (every problem through GMRES): both
    trajectories equal the single-problem mixed path's at tight residuals,
    and only the first run uses the PCG."""
    probs = symmetric_batch(4, 31, sizes=(16, 24, 32, 48))
    dt = 0.05
    params = [T.make_params(p["n"], p["delta"], p["kp"], p["km"], dt) for p in probs]
    u0 = [inp.smoothed_uniform(tuple(reversed(p["n"])), 90 + i) for i, p in enumerate(probs)]
    singles = [T.tfde_assemble(pp, T.TFDE_MIXED) for pp in params]
    try:
        ref = [to_dev(u) for u in u0]
        for m in range(4):
            for i in range(len(probs)):
                assert T.tfde_cn_advance(singles[i], ref[i], None, m == 0, 1e-12).relres <= 1e-12
        for pcg in (True, False):
            B = T.tfde_batch_create(params, 20)
            try:
                T.tfde_batch_set_symmetric_pcg(B, pcg)
                ub = [to_dev(u) for u in u0]
                for m in range(4):
                    infos = T.tfde_batch_cn_advance(B, ub, None, m == 0, 1e-12)
                    assert all(i.relres <= 1e-12 and i.fallback == 0 for i in infos), m
                assert (T.tfde_batch_pcg_solves(B) > 0) if pcg else (T.tfde_batch_pcg_solves(B) == 0)
                assert (T.tfde_batch_graph_cycles(B) == 0) if pcg else (T.tfde_batch_graph_cycles(B) > 0)
                for i in range(len(probs)):
                    assert relerr(to_host(ub[i]), to_host(ref[i])) < 1e-10, (pcg, i)
            finally:
                T.tfde_batch_destroy(B)
        with pytest.raises(T.TfdeError) as e:
            T.tfde_batch_set_symmetric_pcg(0, True)
        assert e.value.status == T.TFDE_EINVAL
    finally:
        for h in singles:
            T.tfde_destroy(h)


def test_batch_pcg_graph_and_host_loop_agree(T):
    """The batched PCG iterations as one graph launch per sweep (iteration
    index, stop tests and loop condition on the device) and driven from the
    host (while every tensor-core launch is timed): the same iteration counts
    and, up to the order of the atomic inner-product sums, the same
    solutions, both matching the oracle's PCG."""
    probs = symmetric_batch(4, 37, sizes=(8, 16, 24, 32))
    dt = 0.1
    params = [T.make_params(p["n"], p["delta"], p["kp"], p["km"], dt) for p in probs]
    u0 = [inp.smoothed_uniform(tuple(reversed(p["n"])), 100 + i) for i, p in enumerate(probs)]
    runs = {}
    for timed in (False, True):
        B = T.tfde_batch_create(params, 20)
        try:
            T.tfde_stats_reset(time_tc=timed)
            us = [to_dev(u) for u in u0]
            infos = T.tfde_batch_cn_advance(B, us, None, True, 1e-12)
            runs[timed] = ([i.iters for i in infos], [to_host(u) for u in us])
            launches = T.tfde_batch_pcg_graph_launches(B)
            sweeps = max(i.refine_sweeps for i in infos)
            assert (launches == 0) if timed else (launches == sweeps > 0), (timed, launches, sweeps)
        finally:
            T.tfde_stats_reset(time_tc=False)
            T.tfde_batch_destroy(B)
    assert runs[False][0] == runs[True][0]
    for i, p in enumerate(probs):
        xo = oracle_step(p, u0[i], dt)
        assert relerr(runs[False][1][i], xo) < 1e-10 and relerr(runs[True][1][i], xo) < 1e-10, i


def test_batch_extreme_axis_lengths_match_oracle(T):
    """Axes of 448 points (the largest the tensor-core path takes: four row
    halves per tile in the grouped exact contraction, the longest lines in
    the grouped slicing) beside axes of 8, along every axis, symmetric and
    non-symmetric problems in one batch: one step each against the oracle."""
    probs = [
        dict(n=(448, 8, 16), delta=(0.7, 0.3, 0.5), kp=(1.0, 1.0, 1.0), km=(1.0, 1.0, 1.0)),
        dict(n=(16, 448, 8), delta=(0.4, 0.8, 0.6), kp=(1.5, 0.5, 1.0), km=(0.5, 1.5, 2.0)),
        dict(n=(8, 16, 448), delta=(0.2, 0.6, 0.9), kp=(1.0, 2.0, 0.7), km=(1.0, 2.0, 0.7)),
        dict(n=(8, 8, 8), delta=(0.5, 0.5, 0.5), kp=(1.0, 0.6, 1.2), km=(0.8, 1.1, 0.9)),
    ]
    dt = 0.05
    params = [T.make_params(p["n"], p["delta"], p["kp"], p["km"], dt) for p in probs]
    B = T.tfde_batch_create(params, 20)
    try:
        u0 = [inp.smoothed_uniform(tuple(reversed(p["n"])), 110 + i) for i, p in enumerate(probs)]
        us = [to_dev(u) for u in u0]
        infos = T.tfde_batch_cn_advance(B, us, None, True, 1e-12)
        assert T.tfde_batch_pcg_solves(B) > 0 and T.tfde_batch_graph_cycles(B) > 0
        for i, p in enumerate(probs):
            assert infos[i].relres <= 1e-12 and infos[i].fallback == 0, (i, infos[i].relres)
            assert relerr(to_host(us[i]), oracle_step(p, u0[i], dt)) < 1e-10, i
    finally:
        T.tfde_batch_destroy(B)


def test_batch_grouped_prepare_matches_single_problem_steps(T):
    """Six chained steps with the order-3 guess and a source on one problem:
    the batch (whose right-hand sides and guesses run grouped once the
    history is built) and the single-problem mixed path reach the same
    trajectories at tight residuals."""
    probs = small_batch(4, 41, sizes=(16, 24, 32))
    probs[1]["km"] = probs[1]["kp"]
    dt = 0.05
    params = [T.make_params(p["n"], p["delta"], p["kp"], p["km"], dt) for p in probs]
    B = T.tfde_batch_create(params, 20)
    singles = [T.tfde_assemble(pp, T.TFDE_MIXED) for pp in params]
    try:
        T.tfde_batch_set_guess_order(B, 3)
        for h in singles:
            T.tfde_set_guess_order(h, 3)
        u0 = [inp.smoothed_uniform(tuple(reversed(p["n"])), 120 + i) for i, p in enumerate(probs)]
        ub = [to_dev(u) for u in u0]
        us = [to_dev(u) for u in u0]
        Fs = [None] * len(probs)
        Fs[2] = to_dev(inp.uniform_vector(tuple(reversed(probs[2]["n"])), 9))
        for m in range(6):
            infos = T.tfde_batch_cn_advance(B, ub, Fs, m == 0, 1e-12)
            for i in range(len(probs)):
                assert T.tfde_cn_advance(singles[i], us[i], Fs[i], m == 0, 1e-12).relres <= 1e-12
                assert infos[i].relres <= 1e-12 and infos[i].fallback == 0, (m, i)
        assert T.tfde_batch_grouped_prepares(B) >= 2
        for i in range(len(probs)):
            assert relerr(to_host(ub[i]), to_host(us[i])) < 1e-10, i
    finally:
        T.tfde_batch_destroy(B)
        for h in singles:
            T.tfde_destroy(h)
