"""FP64 oracle of the learned stepper: a small convolutional network that
jumps 16 explicit Euler steps at once, and its training step.

TEST INFRASTRUCTURE ONLY (imported by the tests and the benchmark's CPU leg,
never by the product path).  The network is not in the paper: Section 2.2
expresses one Euler step as replicate padding + a fixed second-difference
convolution + pointwise terms; here the same building block (replicate
padding + 3x3 / 3x3x3 convolution) is stacked with learned filters.

Definition (2D; 3D replaces 3x3 by 3x3x3):
    x0 = phi[..., None]                               (one channel)
    z1 = conv(x0, W1) + b1,   a1 = gelu(z1)           (1 -> C)
    zl = conv(a_{l-1}, Wl) + bl, al = gelu(zl)        (C -> C, l = 2..5)
    z6 = conv(a5, W6) + b6                            (C -> 1)
    phi_hat = phi + s * z6[..., 0]                    (residual jump)
conv(x, W)[p, co] = sum_t sum_ci x[clamp(p + t), ci] W[t, ci, co], the index
clamped to the grid (replicate padding, the zero-Neumann ghost of Section 2);
gelu(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) (the tanh form);
s = 16 dt / eps^2 is a fixed output scale.
Loss: mean over cells of (phi_hat - phi_target)^2 / s^2.
Optimiser: Adam (Kingma & Ba 2015) with bias correction.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

C = 32          # hidden channels
LAYERS = 6


def taps(ndim: int):
    """Offsets of the 3^d stencil taps, in the order the weights use."""
    return list(itertools.product((-1, 0, 1), repeat=ndim))


def _shift(x: np.ndarray, off, ndim: int) -> np.ndarray:
    """x[clamp(p + off)] for every spatial position p (replicate padding).
    x: [B, *spatial, ch]."""
    idx = []
    for ax in range(ndim):
        n = x.shape[1 + ax]
        idx.append(np.clip(np.arange(n) + off[ax], 0, n - 1))
    out = x
    for ax in range(ndim):
        out = np.take(out, idx[ax], axis=1 + ax)
    return out


def conv(x: np.ndarray, w: np.ndarray, b: np.ndarray, ndim: int) -> np.ndarray:
    """Replicate-padded 3^d convolution.  x [B,*S,ci], w [T,ci,co], b [co]."""
    out = np.zeros(x.shape[:-1] + (w.shape[2],))
    for t, off in enumerate(taps(ndim)):
        out += _shift(x, off, ndim) @ w[t]
    return out + b


def conv_grads(x: np.ndarray, w: np.ndarray, gy: np.ndarray, ndim: int):
    """Gradients of sum(gy * conv(x, w, b)) wrt x, w and b."""
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    sp = x.shape[1:1 + ndim]
    for t, off in enumerate(taps(ndim)):
        xs = _shift(x, off, ndim)
        gw[t] = np.tensordot(xs, gy, axes=(list(range(ndim + 1)), list(range(ndim + 1))))
        # adjoint of the clamped gather: scatter-add gy @ w[t]^T to clamp(p + off)
        contrib = gy @ w[t].T
        idx = [np.clip(np.arange(n) + off[ax], 0, n - 1) for ax, n in enumerate(sp)]
        grid = np.meshgrid(*idx, indexing="ij")
        flat = np.ravel_multi_index(grid, sp).ravel()
        for bidx in range(x.shape[0]):
            g = gx[bidx].reshape(-1, x.shape[-1])
            np.add.at(g, flat, contrib[bidx].reshape(-1, contrib.shape[-1]))
    gb = gy.sum(axis=tuple(range(ndim + 1)))
    return gx, gw, gb


_K = math.sqrt(2.0 / math.pi)


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(_K * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    u = _K * (x + 0.044715 * x ** 3)
    t = np.tanh(u)
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * _K * (1.0 + 3 * 0.044715 * x * x)


def init_params(ndim: int, seed: int = 0, channels: int = C):
    """He-style initial weights; the last layer starts at zero (identity jump)."""
    rng = np.random.default_rng(seed)
    T = 3 ** ndim
    shapes = [(T, 1, channels)] + [(T, channels, channels)] * 4 + [(T, channels, 1)]
    params = []
    for li, sh in enumerate(shapes):
        fan_in = sh[0] * sh[1]
        w = rng.normal(0.0, math.sqrt(2.0 / fan_in), size=sh) if li < 5 else np.zeros(sh)
        params.append((w, np.zeros(sh[2])))
    return params


def forward(params, phi: np.ndarray, scale: float, ndim: int, keep: bool = False):
    """phi [B, *S] -> phi_hat [B, *S]; with keep=True also the pre-activations."""
    x = phi[..., None]
    zs, acts = [], [x]
    for li, (w, b) in enumerate(params):
        z = conv(acts[-1], w, b, ndim)
        zs.append(z)
        if li < LAYERS - 1:
            acts.append(gelu(z))
    out = phi + scale * zs[-1][..., 0]
    if keep:
        return out, zs, acts
    return out


def loss_and_grads(params, phi: np.ndarray, target: np.ndarray, scale: float, ndim: int):
    """MSE of the scaled jump error and its gradient wrt every parameter."""
    out, zs, acts = forward(params, phi, scale, ndim, keep=True)
    n = phi.size
    r = (out - target) / scale
    loss = float(np.mean(r * r))
    g = (2.0 / n) * r[..., None]            # d loss / d z6 (since out = phi + scale z6)
    grads = [None] * LAYERS
    for li in range(LAYERS - 1, -1, -1):
        w, _ = params[li]
        gx, gw, gb = conv_grads(acts[li], w, g, ndim)
        grads[li] = (gw, gb)
        if li > 0:
            g = gx * gelu_grad(zs[li - 1])
    return loss, grads


def adam_step(params, grads, state, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state = dict(t, m, v)."""
    state["t"] += 1
    t = state["t"]
    new = []
    for i, ((w, b), (gw, gb)) in enumerate(zip(params, grads)):
        out = []
        for j, (p, g) in enumerate(((w, gw), (b, gb))):
            key = (i, j)
            m = state["m"].get(key, np.zeros_like(p))
            v = state["v"].get(key, np.zeros_like(p))
            m = beta1 * m + (1 - beta1) * g
            v = beta2 * v + (1 - beta2) * g * g
            state["m"][key], state["v"][key] = m, v
            mh = m / (1 - beta1 ** t)
            vh = v / (1 - beta2 ** t)
            out.append(p - lr * mh / (np.sqrt(vh) + eps))
        new.append(tuple(out))
    return new


def new_adam_state():
    return {"t": 0, "m": {}, "v": {}}
