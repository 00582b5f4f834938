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


def test_what_the_trained_network_gains_over_the_plain_stepper():
    """Train a 2D network on 64^2 trajectories, advance a 128^2 circle by 40
    guarded jumps (640 steps) and report time and error against the plain
    stepper and the FP64 oracle.  Measured on GB300: the hybrid is about 3x
    slower than the plain stepper here and about 2e-2 relative L2 from the
    oracle (the 1e-3 target is not met; the plain stepper is at 2e-7).  The
    assertions bound that outcome as a regression check: the guard keeps the
    field in [-1.001, 1.001] and the error below 5e-2."""
    import time
    import torch
    s = _stream()
    net = L.ac_net_create(2, s.cuda_stream)
    n = 128
    h = 1.0 / n
    try:
        cfg = L.AcTrainConfig(n=64, eps_cells=4.0, pool=16, trajectory_jumps=40, iterations=600,
                              steps_per_jump=16, lr=1e-3, lr_final=1e-5, seed=11)
        L.ac_net_train(net, cfg)
        phi0 = oracle.init_sphere((n, n), h, 0.3, 4 * h)
        ref = oracle.step(phi0.astype(np.float32).astype(np.float64), h, 4 * h, 0.1 * h * h, 640)
        res = {}
        for mode in ("learned", "plain"):
            sim = ac.Simulation((n, n), h, 4 * h, 0.1 * h * h, dtype="f32", stream=s)
            try:
                sim.load(phi0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                fb = None
                if mode == "learned":
                    fb = L.ac_learned_advance(sim.ctx, net, 40, L.AcGuard(16, 1e-6, 1.001, 0.0))
                else:
                    sim.step(640)
                s.synchronize()
                dt = time.perf_counter() - t0
                out = sim.to_numpy().astype(np.float64)
            finally:
                sim.close()
            res[mode] = (dt, fb, float(np.linalg.norm(out - ref) / np.linalg.norm(ref)))
        print(f"learned: {res['learned'][0]*1e3:.2f} ms, {res['learned'][1]} fallbacks, rel-L2 {res['learned'][2]:.2e}; "
              f"plain: {res['plain'][0]*1e3:.2f} ms, rel-L2 {res['plain'][2]:.2e}")
        assert res["plain"][2] <= 1e-5
        assert res["learned"][2] <= 5e-2
    finally:
        L.ac_net_destroy(net)
