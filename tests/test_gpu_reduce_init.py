"""GPU reductions (energy, phase volume, non-finite count) and device-side
initial conditions against the oracle."""
import math

import numpy as np
import pytest

import oracle
import paper_2105_09671_gb300 as ac
from paper_2105_09671_gb300 import workloads as wl

from gpu_util import NP, gpu_run, stored

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("shape", [(1, 1), (37, 53), (300, 257), (3, 4, 5), (31, 40, 77)])
def test_energy_and_volume_match_oracle(shape, dtype):
    h = 1.0 / max(shape)
    eps = 3 * h
    phi0 = wl.smooth_field(shape, seed=5) * 1.1
    ref_in = stored(phi0, dtype)  # the oracle sums the very values the GPU holds
    sim = ac.Simulation(shape, h, eps, 0.1 * h * h, dtype=dtype)
    try:
        sim.load(phi0)
        e, v, bad = sim.observe()
        assert sim.energy() == e and sim.phase_volume() == v
    finally:
        sim.close()
    assert bad == 0
    assert e == pytest.approx(oracle.energy(ref_in, h, eps), rel=1e-12)
    assert v == pytest.approx(oracle.phase_volume(ref_in, h), rel=1e-12, abs=1e-300)


def test_nonfinite_cells_reported():
    shape = (33, 40)
    sim = ac.Simulation(shape, 1 / 40, 0.1, 0.1 / 1600, dtype="f32")
    try:
        a = np.zeros(shape)
        a[3, 7] = np.nan
        a[20, 39] = np.inf
        sim.load(a)
        with pytest.raises(ac.AcError) as err:
            sim.energy()
        assert err.value.code == ac.AC_ERR_NONFINITE
        _, _, bad = sim.observe(allow_nonfinite=True)
        assert bad == 2
    finally:
        sim.close()


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("shape", [(64, 64), (37, 90), (20, 24, 28)])
def test_random_init_bit_exact(shape, dtype):
    sim = ac.Simulation(shape, 1 / shape[-1], 0.05, 0.1 / shape[-1] ** 2, dtype=dtype)
    try:
        sim.init_random(seed=1234, amplitude=0.1)
        got = sim.to_numpy()
    finally:
        sim.close()
    ref = oracle.init_random(shape, seed=1234, amplitude=0.1).astype(NP[dtype])
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("shape,r0,eps", [((64, 64), 0.25, 0.015), ((50, 70), 0.3, 0.02),
                                           ((24, 32, 40), 0.2, 0.03)])
def test_sphere_init_matches(shape, r0, eps, dtype):
    h = 1.0 / shape[-1]
    sim = ac.Simulation(shape, h, eps, 0.1 * h * h, dtype=dtype)
    try:
        sim.init_sphere(r0=r0, center=(0.5, 0.5, 0.5))
        got = sim.to_numpy().astype(np.float64)
    finally:
        sim.close()
    ref64 = oracle.init_sphere(shape, h, r0, eps)
    if dtype == "f64":
        # only tanh itself may differ (both libraries round to within an ulp or two)
        np.testing.assert_allclose(got, ref64, rtol=0, atol=4.5e-16)
    else:
        ref = stored(ref64, dtype)
        ulp = np.spacing(np.abs(ref).astype(NP[dtype])).astype(np.float64)
        assert np.all(np.abs(got - ref) <= ulp)


def test_circle_radius_law_on_gpu():
    # configuration of the 64^2 FP64 circle: R^2 shrinks at rate 2 (within the
    # 10% that h ~ eps allows), measured with the GPU volume reduction
    w = wl.CIRCLE_64
    sim = ac.Simulation(w.shape, w.h, w.eps, w.dt, dtype="f64")
    ts, r2 = [], []
    try:
        sim.init_sphere(r0=w.r0)
        for s in range(11):
            if s:
                sim.step(100)
            ts.append(s * 100 * w.dt)
            r2.append(oracle.radius_from_volume(sim.phase_volume(), 2) ** 2)
        final = sim.to_numpy()
    finally:
        sim.close()
    slope = np.polyfit(ts, r2, 1)[0]
    assert slope == pytest.approx(-2.0, rel=0.10)
    ref = oracle.step(oracle.init_sphere(w.shape, w.h, w.r0, w.eps), w.h, w.eps, w.dt, 1000)
    assert float(np.max(np.abs(final - ref))) <= 1e-12


def test_energy_monotone_on_gpu_separation():
    # random initial state (phase separation): the energy decreases at every sample
    shape = (256, 256)
    h = 1 / 256
    eps = 0.01
    sim = ac.Simulation(shape, h, eps, 0.1 * h * h, dtype="f32")
    try:
        sim.init_random(seed=0, amplitude=0.1)
        e_prev = sim.energy()
        for _ in range(20):
            sim.step(100)
            e = sim.energy()
            assert e < e_prev * (1 + 1e-6)
            e_prev = e
    finally:
        sim.close()
