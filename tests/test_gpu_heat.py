"""The heat equation (eps = +inf: no reaction term) through the same CUDA
kernels: every schedule against the oracle, and against the exact discrete
decay of a Neumann cosine mode."""
import math

import numpy as np
import pytest

import oracle
import paper_2105_09671_gb300 as ac

from gpu_util import NP, assert_parity, schedules

pytestmark = pytest.mark.gpu


def _mode(shape, ks):
    axes = [np.cos(np.pi * k * (np.arange(n) + 0.5) / n) for n, k in zip(shape, ks)]
    out = axes[0]
    for a in axes[1:]:
        out = np.multiply.outer(out, a)
    return out


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(37, 70), (9, 20, 33)])
def test_heat_every_schedule_matches_oracle(shape, dtype):
    h = 1.0 / max(shape)
    dt = 0.1 * h * h
    rng = np.random.default_rng(sum(shape))
    phi0 = rng.uniform(-1, 1, size=shape)
    n = 37
    ref = oracle.step(phi0.astype(NP[dtype]).astype(np.float64), h, math.inf, dt, n)
    for variant, k, tile in schedules(len(shape), dtype):
        sim = ac.Simulation(shape, h, math.inf, dt, dtype=dtype)
        try:
            sim.load(phi0)
            sim.set_schedule(variant, k)
            sim.set_tile(tile)
            sim.step(n)
            assert sim.status() == ac.AC_OK
            out = sim.to_numpy().astype(np.float64)
        finally:
            sim.close()
        assert_parity(out, ref, dtype, f"heat {shape} v{variant} k{k} t{tile}")


@pytest.mark.parametrize("shape,ks", [((64, 96), (3, 7)), ((16, 24, 32), (2, 5, 1))])
def test_heat_mode_decays_exactly_on_gpu(shape, ks):
    h = 1.0 / max(shape)
    dt = 0.1 * h * h
    n = 200
    phi0 = _mode(shape, ks)
    lam = -4.0 * sum(math.sin(math.pi * k / (2 * N)) ** 2 for N, k in zip(shape, ks))
    expect = phi0 * (1.0 + (dt / (h * h)) * lam) ** n
    sim = ac.Simulation(shape, h, math.inf, dt, dtype="f64")
    try:
        sim.load(phi0)
        e0 = sim.energy()
        sim.step(n)
        out = sim.to_numpy()
        e1 = sim.energy()
    finally:
        sim.close()
    np.testing.assert_allclose(out, expect, rtol=0, atol=1e-12)
    # the energy is the Dirichlet energy, decreasing under diffusion
    assert 0 < e1 < e0
    assert e0 == pytest.approx(oracle.energy(phi0, h, math.inf), rel=1e-12)
