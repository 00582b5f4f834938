"""The learned stepper's GPU network (tcgen05 convolutions, BF16 activations,
FP32 accumulation) against the FP64 oracle of oracle/net.py."""
import numpy as np
import pytest

from oracle import net as onet
from paper_2105_09671_gb300 import _lib as L

pytestmark = pytest.mark.gpu

# BF16 activations (8-bit mantissa) through five layers: the network output
# and the gradients agree with FP64 to about 1 % relative L2.
TOL_OUT = 3e-2
TOL_GRAD = 6e-2

# Per-element bounds.  Every layer rounds its activations and its 32 -> 32
# weights to BF16 (relative error <= 2^-9 each, round to nearest) and sums
# in FP32.  A cell's output is a sum of many such rounded products whose
# errors are independent, so its error is about 2^-9 times the RMS size of
# the terms, times sqrt(2 * 6) for the roundings of six layers: ~1.7 * 2^-8
# of the output's RMS, and some 4 sigma of that over 10^4 cells.  Where the
# output is near zero (terms cancelling) the RMS part of the bound covers it:
#   |gpu - oracle| <= C * 2^-8 * (|oracle| + RMS(oracle))
# with C_OUT = 8 for the jump increment.  A wrong tap or a wrong replicated
# boundary cell changes a cell by O(RMS), i.e. a ratio near 0.5, far above
# 8 * 2^-8 = 0.031.
# Weight gradients dW[t][ci][co] = sum_p a[p+t][ci] g[p][co] multiply the
# forward activations (error up to C_OUT * 2^-8 of their RMS) by the
# backward signal, which carries the loss residual's share of the forward
# error and, per layer, the BF16 roundings of the data gradient, of the
# pre-activation inside gelu' and of the transposed weights: about
# 5 * 2^-8 relative per product term.  With random data the terms of a sum
# have random signs, so a gradient entry keeps that relative error (it does
# not average down against the entry's own size), and the largest of ~10^4
# entries sits near 4 sigma, ~20 * 2^-8 of the layer's RMS: C_GRAD = 32.  A
# wrong tap or a wrong replicate-padding adjoint shows on the grids made of
# boundary cells only (3 x 1, 1 x 130, 2 x 2 x 2) as errors of the order of
# the entries themselves, C > 100.
C_OUT = 8.0
C_GRAD = 32.0


def _elementwise_ratio(got, ref):
    """max |got - ref| / (2^-8 (|ref| + RMS(ref))): the C the bound needs."""
    rms = float(np.sqrt(np.mean(ref * ref)))
    return float(np.max(np.abs(got - ref) / (2.0 ** -8 * (np.abs(ref) + rms + 1e-300))))


def _params(ndim, seed):
    p = onet.init_params(ndim, seed=seed)
    rng = np.random.default_rng(seed + 1)
    p[-1] = (rng.normal(0, 0.05, size=p[-1][0].shape), rng.normal(0, 0.01, size=1))
    # non-zero biases everywhere so every bias gradient is exercised
    p = [(w, b + rng.normal(0, 0.05, size=b.shape)) for w, b in p]
    return p


def _flat(params):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])


def _unflat(vec, like):
    out, off = [], 0
    for w, b in like:
        nw, nb = w.size, b.size
        out.append((vec[off:off + nw].reshape(w.shape), vec[off + nw:off + nw + nb]))
        off += nw + nb
    return out


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-30))


CASES = [(2, (2, 17, 200)), (2, (1, 64, 64)), (2, (1, 3, 1)), (2, (1, 1, 130)), (3, (1, 5, 9, 130)),
         (3, (2, 4, 4, 4)), (3, (1, 2, 2, 2))]


def _shape_args(ndim, shape):
    if ndim == 2:
        b, ny, nx = shape
        return b, nx, ny, 1
    b, nz, ny, nx = shape
    return b, nx, ny, nz


@pytest.mark.parametrize("ndim,shape", CASES)
def test_forward_matches_oracle(ndim, shape):
    import torch
    params = _params(ndim, seed=3)
    rng = np.random.default_rng(5)
    phi = rng.uniform(-1, 1, size=shape)
    scale = 0.1
    ref = onet.forward(params, phi, scale, ndim)
    s = torch.cuda.current_stream().cuda_stream
    h = L.ac_net_create(ndim, s)
    try:
        L.ac_net_set_params(h, _flat(params))
        d_phi = torch.tensor(phi, dtype=torch.float32, device="cuda")
        d_out = torch.full_like(d_phi, float("nan"))
        L.ac_net_forward(h, d_phi.data_ptr(), d_out.data_ptr(), *_shape_args(ndim, shape), scale)
        torch.cuda.synchronize()
        out = d_out.cpu().numpy().astype(np.float64)
    finally:
        L.ac_net_destroy(h)
    phi32 = phi.astype(np.float32).astype(np.float64)
    # compare the learned increments (output minus input) / scale
    inc_gpu, inc_ref = (out - phi32) / scale, (ref - phi) / scale
    assert _rel(inc_gpu, inc_ref) <= TOL_OUT
    # and cell by cell, so that one wrong tap or boundary cell cannot hide
    ratio = _elementwise_ratio(inc_gpu, inc_ref)
    print(f"\nforward {ndim}D {shape}: per-element C = {ratio:.2f} (bound {C_OUT})")
    assert ratio <= C_OUT


@pytest.mark.parametrize("ndim,shape", CASES)
def test_loss_and_gradients_match_oracle(ndim, shape):
    import torch
    params = _params(ndim, seed=7)
    rng = np.random.default_rng(9)
    phi = rng.uniform(-1, 1, size=shape)
    target = phi + 0.1 * rng.uniform(-1, 1, size=shape)
    scale = 0.1
    loss_ref, grads_ref = onet.loss_and_grads(params, phi, target, scale, ndim)
    s = torch.cuda.current_stream().cuda_stream
    h = L.ac_net_create(ndim, s)
    try:
        L.ac_net_set_params(h, _flat(params))
        d_phi = torch.tensor(phi, dtype=torch.float32, device="cuda")
        d_tgt = torch.tensor(target, dtype=torch.float32, device="cuda")
        loss, g = L.ac_net_loss_grads(h, d_phi.data_ptr(), d_tgt.data_ptr(), *_shape_args(ndim, shape),
                                      scale, want_grads=True)
    finally:
        L.ac_net_destroy(h)
    assert loss == pytest.approx(loss_ref, rel=TOL_OUT)
    got = _unflat(g.astype(np.float64), params)
    ratios = {}
    for li, ((gw, gb), (rw, rb)) in enumerate(zip(got, grads_ref)):
        assert _rel(gw, rw) <= TOL_GRAD, f"layer {li} weights"
        assert _rel(gb, rb) <= TOL_GRAD, f"layer {li} bias"
        ratios[f"w{li}"] = _elementwise_ratio(gw, rw)
        ratios[f"b{li}"] = _elementwise_ratio(gb, rb)
    print(f"\ngradients {ndim}D {shape}: per-element C " +
          " ".join(f"{k}={v:.2f}" for k, v in ratios.items()) + f" (bound {C_GRAD})")
    bad = {k: v for k, v in ratios.items() if v > C_GRAD}
    assert not bad, f"per-element bound exceeded: {bad}"


def test_adam_training_lowers_the_loss():
    import torch
    ndim, shape = 2, (4, 32, 160)
    rng = np.random.default_rng(0)
    phi = rng.uniform(-1, 1, size=shape)
    target = phi + 0.05 * np.tanh(phi)  # a smooth pointwise map to learn
    s = torch.cuda.current_stream().cuda_stream
    h = L.ac_net_create(ndim, s)
    try:
        L.ac_net_set_params(h, _flat(onet.init_params(ndim, seed=1)))
        d_phi = torch.tensor(phi, dtype=torch.float32, device="cuda")
        d_tgt = torch.tensor(target, dtype=torch.float32, device="cuda")
        losses = [L.ac_net_train_step(h, d_phi.data_ptr(), d_tgt.data_ptr(), *_shape_args(ndim, shape),
                                      0.1, 2e-3) for _ in range(60)]
    finally:
        L.ac_net_destroy(h)
    assert losses[-1] < 0.2 * losses[0]
