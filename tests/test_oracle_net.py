"""Pins of the learned-stepper oracle (oracle/net.py) against facts outside it:
brute-force loops, the paper's pad + second-difference-filter statement of the
Laplacian (checked against the independently pinned stencil oracle), central
finite differences, GELU identities and Adam's first-step closed form."""
import math

import numpy as np
import pytest

import oracle
from oracle import net


def _brute_conv(x, w, b, ndim):
    B = x.shape[0]
    sp = x.shape[1:1 + ndim]
    out = np.zeros((B,) + sp + (w.shape[2],))
    for bi in range(B):
        for p in np.ndindex(*sp):
            for t, off in enumerate(net.taps(ndim)):
                q = tuple(min(max(p[a] + off[a], 0), sp[a] - 1) for a in range(ndim))
                for ci in range(w.shape[1]):
                    for co in range(w.shape[2]):
                        out[(bi,) + p + (co,)] += x[(bi,) + q + (ci,)] * w[t, ci, co]
            out[(bi,) + p] += b
    return out


@pytest.mark.parametrize("ndim,shape", [(2, (3, 3)), (2, (2, 5)), (3, (3, 2, 2))])
def test_conv_matches_brute_force(ndim, shape):
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2,) + shape + (2,))
    w = rng.normal(size=(3 ** ndim, 2, 3))
    b = rng.normal(size=3)
    np.testing.assert_allclose(net.conv(x, w, b, ndim), _brute_conv(x, w, b, ndim), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("shape", [(9, 13), (5, 6, 7)])
def test_replicate_pad_with_second_difference_filter_is_the_laplacian(shape):
    # Section 2.2: replication padding + the 2nd-order differencing filter give
    # dt * Lap_h phi.  With eps huge the reaction vanishes, so one oracle step
    # is phi + (dt/h^2) * (neighbour sum - 2d phi).
    ndim = len(shape)
    h, dt = 1.0 / max(shape), 0.1 / max(shape) ** 2
    phi = np.random.default_rng(1).uniform(-1, 1, size=shape)
    w = np.zeros((3 ** ndim, 1, 1))
    for t, off in enumerate(net.taps(ndim)):
        if sum(abs(o) for o in off) == 1:
            w[t] = 1.0
        elif all(o == 0 for o in off):
            w[t] = -2.0 * ndim
    lap = net.conv(phi[None, ..., None], w, np.zeros(1), ndim)[0, ..., 0]
    stepped = oracle.step(phi, h, 1e9, dt, 1)
    np.testing.assert_allclose(stepped - phi, dt / (h * h) * lap, rtol=0, atol=1e-14)


def test_gelu_identities():
    x = np.linspace(-6, 6, 241)
    assert net.gelu(np.array(0.0)) == 0.0
    np.testing.assert_allclose(net.gelu(x) - net.gelu(-x), x, atol=1e-15)
    assert net.gelu(np.array(30.0)) == pytest.approx(30.0, rel=1e-15)
    d = 1e-6
    fd = (net.gelu(x + d) - net.gelu(x - d)) / (2 * d)
    np.testing.assert_allclose(net.gelu_grad(x), fd, rtol=1e-7, atol=1e-9)
    # tanh form of GELU: gelu(1) = 0.5 (1 + tanh(sqrt(2/pi) * 1.044715))
    assert float(net.gelu(np.array(1.0))) == pytest.approx(
        0.5 * (1 + math.tanh(math.sqrt(2 / math.pi) * 1.044715)), rel=1e-15)


@pytest.mark.parametrize("ndim,shape", [(2, (5, 4)), (3, (3, 3, 2))])
def test_gradients_match_finite_differences(ndim, shape):
    rng = np.random.default_rng(2)
    params = net.init_params(ndim, seed=3, channels=3)
    # give the last layer non-zero weights so every gradient path is exercised
    params[-1] = (rng.normal(0, 0.3, size=params[-1][0].shape), rng.normal(0, 0.1, size=1))
    phi = rng.uniform(-1, 1, size=(2,) + shape)
    target = rng.uniform(-1, 1, size=(2,) + shape)
    scale = 0.1
    _, grads = net.loss_and_grads(params, phi, target, scale, ndim)
    d = 1e-6
    for li in range(net.LAYERS):
        for j in range(2):
            p = params[li][j]
            g = grads[li][j]
            for idx in list(np.ndindex(*p.shape))[:: max(1, p.size // 7)]:
                def loss_at(v):
                    q = [list(pp) for pp in params]
                    arr = q[li][j].copy()
                    arr[idx] = v
                    q[li][j] = arr
                    return net.loss_and_grads([tuple(a) for a in q], phi, target, scale, ndim)[0]
                fd = (loss_at(p[idx] + d) - loss_at(p[idx] - d)) / (2 * d)
                assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-9), (li, j, idx)


def test_zero_last_layer_is_the_identity_jump():
    params = net.init_params(2, seed=0)
    phi = np.random.default_rng(4).uniform(-1, 1, size=(1, 8, 8))
    np.testing.assert_array_equal(net.forward(params, phi, 0.1, 2), phi)


def test_adam_first_step_moves_by_lr_times_sign():
    # with m0 = v0 = 0, bias correction makes the first step lr * g / (|g| + eps)
    params = [(np.array([1.0, -2.0, 3.0]), np.array([0.5]))]
    grads = [(np.array([0.3, -4.0, 1e-3]), np.array([-2.0]))]
    st = net.new_adam_state()
    new = net.adam_step(params, grads, st, lr=0.01)
    # eps = 1e-8 shifts the step by at most lr * eps / |g| = 1e-7
    np.testing.assert_allclose(new[0][0], [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01], rtol=0, atol=2e-7)
    np.testing.assert_allclose(new[0][1], [0.5 + 0.01], atol=1e-8)
