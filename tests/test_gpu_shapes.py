"""The further initial shapes of Section 3.1 (dumbbell, star, torus) on the
GPU, and the experiment of Table 3: Err of Eq. (ERReq), the RMS difference
to the FP64 oracle averaged over every time step, for each of the paper's
runs in 2D and 3D."""
import math

import numpy as np
import pytest

import oracle
import paper_2105_09671_gb300 as ac
from oracle import shapes as S
from paper_2105_09671_gb300 import workloads as wl

from gpu_util import NP, assert_parity, schedules

pytestmark = pytest.mark.gpu


def oracle_init(kind, shape, h, lower, eps, params=(), seed=0):
    if kind == "dumbbell":
        return S.on_grid(S.dumbbell, shape, h, lower, r0=params[0], eps=eps)
    if kind == "star":
        return S.on_grid(S.star, shape, h, lower, eps=eps)
    if kind == "torus":
        return S.on_grid(S.torus, shape, h, lower, r1=params[0], r2=params[1], eps=eps)
    if kind == "sphere":
        return oracle.init_sphere(shape, h, params[0], eps, lower=lower)
    return oracle.init_random(shape, seed=seed)


def gpu_init(sim, kind, lower, params=(), seed=0):
    if kind == "dumbbell":
        sim.init_shape("dumbbell", lower, r0=params[0])
    elif kind == "star":
        sim.init_shape("star", lower)
    elif kind == "torus":
        sim.init_shape("torus", lower, r1=params[0], r2=params[1])
    elif kind == "sphere":
        sim.init_sphere(params[0], lower=lower)
    else:
        sim.init_random(seed)


# small versions of the paper's domains: (kind, shape, h, lower, params)
SMALL = [
    ("dumbbell", (50, 100), 1 / 50, (0.0, 0.0, 0.0), (0.2,)),
    ("dumbbell", (20, 20, 40), 1 / 20, (0.0, 0.0, 0.0), (0.25,)),
    ("star", (64, 64), 1 / 64, (0.0, 0.0, 0.0), ()),
    ("star", (40, 40, 40), 0.05, (-1.0, -1.0, -1.0), ()),
    ("torus", (64, 64), 1 / 64, (0.0, 0.0, 0.0), (0.4, 0.3)),
    ("torus", (40, 40, 40), 0.05, (-1.0, -1.0, -1.0), (0.3, 0.3)),
    ("torus", (30, 44, 36), 0.05, (-1.0, -1.1, -0.9), (0.5, 0.2)),
]
IDS = [f"{k}{len(s)}d-{'x'.join(map(str, s))}" for k, s, *_ in SMALL]


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("case", SMALL, ids=IDS)
def test_device_init_matches_oracle(case, dtype):
    kind, shape, h, lower, params = case
    eps = oracle.eps_m(h, 10)
    ref = oracle_init(kind, shape, h, lower, eps, params)
    sim = ac.Simulation(shape, h, eps, 0.1 * h * h, dtype=dtype)
    try:
        gpu_init(sim, kind, lower, params)
        out = sim.to_numpy().astype(np.float64)
    finally:
        sim.close()
    stored = ref.astype(NP[dtype]).astype(np.float64)
    if dtype == "f64":
        # CUDA's and the host's FP64 tanh / atan / cos differ by an ulp or two
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-13)
    else:
        # one rounding of nearly equal FP64 values: equal but for rare ties
        ulp = 2.5e-7 if dtype == "f32" else 1e-3
        np.testing.assert_allclose(out, stored, rtol=0, atol=ulp)
        assert np.mean(out == stored) > 0.999


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("case", SMALL, ids=IDS)
def test_shapes_step_parity_every_schedule(case, dtype):
    kind, shape, h, lower, params = case
    eps = oracle.eps_m(h, 10)
    dt = 0.1 * h * h
    n = 60
    ref0 = oracle_init(kind, shape, h, lower, eps, params)
    ref = oracle.step(ref0.astype(NP[dtype]).astype(np.float64), h, eps, dt, n)
    for variant, k, tile in schedules(len(shape), dtype):
        sim = ac.Simulation(shape, h, eps, dt, dtype=dtype)
        try:
            gpu_init(sim, kind, lower, params)
            sim.set_schedule(variant, k)
            sim.set_tile(tile)
            sim.step(n)
            assert sim.status() == ac.AC_OK
            out = sim.to_numpy().astype(np.float64)
        finally:
            sim.close()
        assert_parity(out, ref, dtype, f"{kind} {shape} v{variant} k{k} t{tile}")


# Table 3 of the paper (its GPU FP32 PyTorch code against its CPU NumPy code),
# for context next to ours.
PAPER_TABLE3 = {
    "separation2d": 1.75e-6, "dumbbell2d": 7.03e-7, "circle2d": 5.51e-7, "star2d": 6.55e-7,
    "torus2d": 7.52e-7, "separation3d": 3.01e-6, "dumbbell3d": 1.20e-6, "sphere3d": 1.11e-6,
    "star3d": 1.56e-6, "torus3d": 1.91e-6,
}


@pytest.mark.parametrize("case", wl.PAPER_CASES, ids=[c.name for c in wl.PAPER_CASES])
def test_table3_err_against_the_oracle(case):
    """Err (Eq. ERReq) of the FP64 and FP32 stepper against the FP64 oracle
    over every step of the paper's run; the FP32 path starts from the FP32
    rounding of the same state."""
    eps = oracle.eps_m(case.h, case.m)
    cpu64 = oracle_init(case.kind, case.shape, case.h, case.lower, eps, case.params, case.seed)
    cpu32 = cpu64.astype(np.float32).astype(np.float64)
    sims = {d: ac.Simulation(case.shape, case.h, eps, case.dt, dtype=d) for d in ("f64", "f32")}
    acc = {"f64": 0.0, "f32": 0.0}
    try:
        for d, sim in sims.items():
            gpu_init(sim, case.kind, case.lower, case.params, case.seed)
        # the device initial states are the oracle's (to the init tolerance)
        np.testing.assert_allclose(sims["f64"].to_numpy(), cpu64, rtol=0, atol=1e-13)
        for _ in range(case.steps):
            cpu64 = oracle.step(cpu64, case.h, eps, case.dt, 1)
            cpu32 = oracle.step(cpu32, case.h, eps, case.dt, 1)
            for d, sim in sims.items():
                sim.step(1)
                ref = cpu64 if d == "f64" else cpu32
                diff = sim.to_numpy().astype(np.float64) - ref
                acc[d] += math.sqrt(float(np.mean(diff * diff)))
        for sim in sims.values():
            assert sim.status() == ac.AC_OK
    finally:
        for sim in sims.values():
            sim.close()
    err = {d: acc[d] / case.steps for d in acc}
    print(f"\nTable 3 {case.name}: {case.shape} x {case.steps} steps, eps_{case.m:g}: "
          f"Err FP64 {err['f64']:.2e}, FP32 {err['f32']:.2e} (paper's GPU FP32: "
          f"{PAPER_TABLE3[case.name]:.2e})")
    assert err["f64"] <= 1e-13
    assert err["f32"] <= 1e-6
