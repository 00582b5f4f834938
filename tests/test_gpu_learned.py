"""The learned stepper end to end: training on plain-stepper trajectories, the
guarded advance and its fallback, and what the network gains (or loses)
against the plain stepper."""
import numpy as np
import pytest

import oracle
import paper_2105_09671_gb300 as ac
from paper_2105_09671_gb300 import _lib as L

pytestmark = pytest.mark.gpu


def _stream():
    import torch
    return torch.cuda.Stream()


def _held_out_jumps(ndim, n, steps, count, seed):
    """(inputs, targets) of `count` jumps of the FP64 oracle on n^ndim grids:
    states of random and tanh-sphere trajectories at several ages, each
    advanced by `steps` Euler steps; rounded to FP32 like the training data."""
    h = 1.0 / n
    eps, dt = 4.0 * h, 0.1 * h * h
    shape = (n,) * ndim
    rng = np.random.default_rng(seed)
    xs, ys = [], []
    for b in range(count):
        if b % 2 == 0:
            phi = oracle.init_random(shape, seed=seed + b)
        else:
            phi = oracle.init_sphere(shape, h, float(rng.uniform(0.1, 0.4)), eps)
        phi = oracle.step(phi, h, eps, dt, steps * int(rng.integers(0, 20)))
        x = phi.astype(np.float32).astype(np.float64)
        xs.append(x.astype(np.float32))
        ys.append(oracle.step(x, h, eps, dt, steps).astype(np.float32))
    return np.stack(xs), np.stack(ys)


@pytest.mark.parametrize("ndim,n,pool,iters,drop", [(2, 64, 16, 400, 0.1), (3, 16, 8, 300, 0.75)])
def test_training_on_plain_trajectories_lowers_the_held_out_loss(ndim, n, pool, iters, drop):
    # The training loss itself spikes whenever a fresh trajectory (fast
    # spinodal growth) enters the pool, so the test measures the loss on a
    # fixed held-out set of oracle jumps before (the identity jump of the
    # initial weights) and after training.  Measured on GB300: 2D 2.9e-3 ->
    # 1.6e-4, 3D (16^3, where eps = 4 h is a quarter of the box) 0.116 -> 0.064.
    import torch
    s = _stream()
    steps = 16
    x, y = _held_out_jumps(ndim, n, steps, 8, seed=900 + ndim)
    xd = torch.from_numpy(x).cuda()
    yd = torch.from_numpy(y).cuda()
    nz = n if ndim == 3 else 1
    scale = steps * 0.1 / 16.0  # steps dt / eps^2 with dt = 0.1 h^2, eps = 4 h
    net = L.ac_net_create(ndim, s.cuda_stream)
    try:
        torch.cuda.synchronize()
        before, _ = L.ac_net_loss_grads(net, xd.data_ptr(), yd.data_ptr(), len(x), n, n, nz, scale)
        cfg = L.AcTrainConfig(n=n, eps_cells=4.0, pool=pool, trajectory_jumps=40, iterations=iters,
                              steps_per_jump=steps, lr=1e-3, lr_final=1e-5, seed=3)
        hist, used = L.ac_net_train(net, cfg)
        after, _ = L.ac_net_loss_grads(net, xd.data_ptr(), yd.data_ptr(), len(x), n, n, nz, scale)
    finally:
        L.ac_net_destroy(net)
    print(f"\n{ndim}D held-out loss: identity {before:.3e}, trained {after:.3e}")
    assert used >= pool
    assert np.all(np.isfinite(hist))
    assert np.isfinite(after) and after < drop * before


def test_rejected_jumps_fall_back_to_the_plain_stepper_exactly():
    import torch
    s = _stream()
    n = 128
    h = 1.0 / n
    net = L.ac_net_create(2, s.cuda_stream)
    cnt = L.ac_net_param_count(2)
    # a broken network: huge weights make every jump violate max |phi| <= 1.001
    L.ac_net_set_params(net, np.full(cnt, 50.0, dtype=np.float32))
    sim = ac.Simulation((n, n), h, 4 * h, 0.1 * h * h, dtype="f32", stream=s)
    ref = ac.Simulation((n, n), h, 4 * h, 0.1 * h * h, dtype="f32", stream=s)
    try:
        sim.init_random(seed=5)
        ref.init_random(seed=5)
        guard = L.AcGuard(16, 1e-6, 1.001, 0.0)
        fb = L.ac_learned_advance(sim.ctx, net, 10, guard)
        ref.step(160)
        assert fb == 10
        assert np.array_equal(sim.to_numpy(), ref.to_numpy())
    finally:
        sim.close()
        ref.close()
        L.ac_net_destroy(net)


def test_identity_network_is_rejected_by_the_residual_check():
    # the initial network is the identity jump; on an evolving state its
    # residual against one 16 dt Euler estimate is 16 dt |RHS|, so a tight
    # residual threshold rejects it and the plain stepper runs instead
    s = _stream()
    n = 96
    h = 1.0 / n
    net = L.ac_net_create(2, s.cuda_stream)
    sim = ac.Simulation((n, n), h, 4 * h, 0.1 * h * h, dtype="f32", stream=s)
    try:
        sim.init_sphere(r0=0.3)
        fb = L.ac_learned_advance(sim.ctx, net, 4, L.AcGuard(16, 1e-6, 1.001, 1e-9))
        assert fb == 4
        phi0 = oracle.init_sphere((n, n), h, 0.3, 4 * h).astype(np.float32).astype(np.float64)
        out = sim.to_numpy().astype(np.float64)
        np.testing.assert_allclose(out, oracle.step(phi0, h, 4 * h, 0.1 * h * h, 64), rtol=0, atol=1e-5)
    finally:
        sim.close()
        L.ac_net_destroy(net)


def test_jump_residual_of_the_plain_stepper():
    # the guard's residual of a true 16-step jump is small for a smooth
    # circle and much larger for a random state (spinodal growth)
    import torch
    s = _stream()
    n = 128
    h = 1.0 / n
    vals = {}
    for init in ("sphere", "random"):
        a = ac.Simulation((n, n), h, 4 * h, 0.1 * h * h, dtype="f32", stream=s)
        b = ac.Simulation((n, n), h, 4 * h, 0.1 * h * h, dtype="f32", stream=s)
        try:
            if init == "sphere":
                a.init_sphere(r0=0.3)
                b.init_sphere(r0=0.3)
            else:
                a.init_random(seed=1)
                b.init_random(seed=1)
            b.step(16)
            mabs, res = L.ac_jump_residual(a.ctx, b._buf.data_ptr(), 16)
            vals[init] = res
            assert mabs <= 1.0 + 1e-6
        finally:
            a.close()
            b.close()
    assert 0 < vals["sphere"] < vals["random"]


@pytest.mark.parametrize("shape", [(128, 128), (200, 130), (40, 40), (24, 24, 24), (64, 48, 40)])
def test_spot_check_reproduces_the_plain_stepper(shape):
    # the spot check recomputes the plain stepper's 16-step result on boxes;
    # for a jump made by the plain stepper itself it must find no difference
    # at all (same FP32 arithmetic), whether the boxes sit inside the grid,
    # touch its faces, or cover it (40^2, 24^3: boxes clipped to the grid)
    s = _stream()
    n = max(shape)
    h = 1.0 / n
    a = ac.Simulation(shape, h, 4 * h, 0.1 * h * h, dtype="f32", stream=s)
    b = ac.Simulation(shape, h, 4 * h, 0.1 * h * h, dtype="f32", stream=s)
    try:
        a.init_random(seed=3)
        b.init_random(seed=3)
        b.step(16)
        for seed in (7, 8):
            mx, rel, cells = L.ac_jump_spot_check(a.ctx, b._buf.data_ptr(), 16, 0, 0, seed)
            assert mx == 0.0 and rel == 0.0
            assert cells > 0
        if shape in ((40, 40), (24, 24, 24)):
            # every default box (64 in 2D, 16 in 3D) clips to the whole grid
            assert cells == np.prod(shape) * (64 if len(shape) == 2 else 16)
    finally:
        a.close()
        b.close()


def test_spot_check_measures_planted_errors():
    import torch
    s = _stream()
    n = 40  # boxes of 32 + 2 * 16 cells clip to the whole 40^2 grid: every cell is checked
    h = 1.0 / n
    a = ac.Simulation((n, n), h, 4 * h, 0.1 * h * h, dtype="f32", stream=s)
    b = ac.Simulation((n, n), h, 4 * h, 0.1 * h * h, dtype="f32", stream=s)
    try:
        a.init_sphere(r0=0.3)
        b.init_sphere(r0=0.3)
        b.step(16)
        with torch.cuda.stream(s):
            ref = b.phi.clone()
            b.phi.mul_(1.0 + 1e-3)  # a uniform relative error of 1e-3
        mx, rel, _ = L.ac_jump_spot_check(a.ctx, b._buf.data_ptr(), 16, 1, 0, 1)
        assert abs(rel - 1e-3) <= 1e-6
        with torch.cuda.stream(s):
            b.phi.copy_(ref)
            b.phi[n - 1, 0] += 0.5  # one wrong cell in a corner of the domain
        mx, rel, _ = L.ac_jump_spot_check(a.ctx, b._buf.data_ptr(), 16, 1, 0, 1)
        assert mx == pytest.approx(0.5, abs=1e-6)
        assert rel > 0
    finally:
        a.close()
        b.close()


def _trained_net(s):
    net = L.ac_net_create(2, s.cuda_stream)
    cfg = L.AcTrainConfig(n=64, eps_cells=4.0, pool=16, trajectory_jumps=40, iterations=600,
                          steps_per_jump=16, lr=1e-3, lr_final=1e-5, seed=11)
    L.ac_net_train(net, cfg)
    return net


def test_calibration_sets_the_residual_threshold():
    s = _stream()
    net = _trained_net(s)
    try:
        cal = L.AcTrainConfig(n=64, eps_cells=4.0, pool=16, trajectory_jumps=40, iterations=1,
                              steps_per_jump=16, lr=1e-3, lr_final=1e-5, seed=12345)
        guard = L.AcGuard(16, 1e-6, 1.001, 0.0, 0.0, 0, 0, 99)
        rep = L.ac_net_calibrate_guard(net, cal, 2.0, guard)
        print(f"\ncalibration: {rep}")
        assert rep["states"] == 16
        assert rep["plain_residual_max"] > 0
        assert guard.residual_tol == pytest.approx(2.0 * rep["plain_residual_max"], rel=1e-12)
        assert 0 < rep["net_rel_err_median"] <= rep["net_rel_err_max"]
        # on 64^2 the spot check's boxes cover the whole grid: its estimate is
        # the whole-field error (up to the order of the sums)
        assert rep["spot_rel_err_max"] == pytest.approx(rep["net_rel_err_max"], rel=1e-9)
    finally:
        L.ac_net_destroy(net)


@pytest.mark.parametrize("init", ["circle", "random"])
def test_guarded_learned_stepper_meets_the_target_or_falls_back(init):
    """A trained network advances a 128^2 field by 40 guarded jumps (640
    steps); the guard's spot check allows each jump a relative error of
    1e-3 / 40 against the plain stepper (the final target over the jumps),
    so the result must be within 1e-3 relative L2 of the FP64 oracle,
    whether the jumps are accepted or fall back.  Measured on GB300 with
    this small network: every jump is rejected on both states (its
    per-jump errors are ~1e-3 on the circle and up to ~0.6 on the random
    state), the result is the plain stepper's (~2e-7 from the oracle), and
    the hybrid is slower than the plain stepper.  Without the spot check
    the random state's error grows to ~1.5: the guard is what keeps it."""
    import time
    import torch
    s = _stream()
    net = _trained_net(s)
    n, jumps = 128, 40
    h = 1.0 / n
    target = 1e-3
    try:
        cal = L.AcTrainConfig(n=64, eps_cells=4.0, pool=16, trajectory_jumps=40, iterations=1,
                              steps_per_jump=16, lr=1e-3, lr_final=1e-5, seed=12345)
        guard = L.AcGuard(16, 1e-6, 1.001, 0.0, target / jumps, 0, 0, 99)
        L.ac_net_calibrate_guard(net, cal, 2.0, guard)
        assert guard.residual_tol > 0
        phi0 = (oracle.init_sphere((n, n), h, 0.3, 4 * h) if init == "circle"
                else oracle.init_random((n, n), seed=5))
        ref = oracle.step(phi0.astype(np.float32).astype(np.float64), h, 4 * h, 0.1 * h * h, 16 * jumps)
        res = {}
        for mode in ("learned", "unguarded", "plain"):
            sim = ac.Simulation((n, n), h, 4 * h, 0.1 * h * h, dtype="f32", stream=s)
            try:
                sim.load(phi0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rep = None
                if mode == "learned":
                    _, rep = L.ac_learned_advance(sim.ctx, net, jumps, guard, with_report=True)
                elif mode == "unguarded":
                    _, rep = L.ac_learned_advance(sim.ctx, net, jumps, L.AcGuard(16, 1e30, 1e30, 0.0),
                                                  with_report=True)
                else:
                    sim.step(16 * jumps)
                s.synchronize()
                dt = time.perf_counter() - t0
                out = sim.to_numpy().astype(np.float64)
            finally:
                sim.close()
            res[mode] = (dt, rep, float(np.linalg.norm(out - ref) / np.linalg.norm(ref)))
        rl = res["learned"][1]
        print(f"\n{init}: learned {res['learned'][0]*1e3:.2f} ms, {rl['fallbacks']}/{jumps} fallbacks "
              f"(spot {rl['rejected_spot']}, energy {rl['rejected_energy']}, max {rl['rejected_max_abs']}, "
              f"residual {rl['rejected_residual']}), largest spot error {rl['max_spot_rel']:.2e}, "
              f"rel-L2 {res['learned'][2]:.2e}; unguarded rel-L2 {res['unguarded'][2]:.2e}; "
              f"plain {res['plain'][0]*1e3:.2f} ms, rel-L2 {res['plain'][2]:.2e}")
        assert res["plain"][2] <= 1e-5
        assert res["learned"][2] <= target
        assert rl["jumps"] == jumps
    finally:
        L.ac_net_destroy(net)
