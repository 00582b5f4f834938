"""Whole runs of the two large configurations against the FP64 oracle:

- 2D phase separation, 4096^2, random state 0.1 U[-1, 1), 5000 steps: the
  FP64 and FP32 steppers (default schedules) against the oracle at the end,
  and the discrete energy every 100 steps, which the scheme must not raise;
- 3D sphere at 256^3, 2000 steps: FP32 and FP16 storage against the oracle.

The oracle runs multithreaded on the host (8.4e10 and 3.4e10 cell-updates)."""
import numpy as np
import pytest

import oracle
import paper_2105_09671_gb300 as ac
from paper_2105_09671_gb300 import workloads as wl

from gpu_util import TOL_MAXABS, TOL_RELL2_F16S, rel_l2

pytestmark = pytest.mark.gpu


def test_separation_4096_full_run():
    w = wl.SEPARATION_4096
    phi0 = oracle.init_random(w.shape, seed=w.seed)
    ref = oracle.step(phi0, w.h, w.eps, w.dt, w.steps)
    ref32 = oracle.step(phi0.astype(np.float32).astype(np.float64), w.h, w.eps, w.dt, w.steps)
    outs, energies = {}, {}
    for dtype in ("f64", "f32"):
        sim = ac.Simulation(w.shape, w.h, w.eps, w.dt, dtype=dtype)
        try:
            sim.init_random(seed=w.seed)
            es = [sim.energy()]
            for _ in range(w.steps // 100):
                sim.step(100)
                es.append(sim.energy())
            assert sim.status() == ac.AC_OK
            outs[dtype] = sim.to_numpy().astype(np.float64)
            energies[dtype] = np.array(es)
        finally:
            sim.close()
    err64 = float(np.max(np.abs(outs["f64"] - ref)))
    err32 = float(np.max(np.abs(outs["f32"] - ref32)))
    print(f"\n4096^2 x {w.steps}: FP64 max-abs {err64:.2e}, FP32 max-abs {err32:.2e}, "
          f"FP32 vs FP64 rel-L2 {rel_l2(outs['f32'], outs['f64']):.2e}")
    assert err64 <= TOL_MAXABS["f64"]
    assert err32 <= TOL_MAXABS["f32"]
    # gradient flow: the energy never rises (FP32: up to rounding of the sum)
    d64 = np.diff(energies["f64"])
    d32 = np.diff(energies["f32"])
    assert np.all(d64 <= 1e-12 * np.abs(energies["f64"][1:]))
    assert np.all(d32 <= 1e-6 * np.abs(energies["f32"][1:]))
    assert energies["f64"][-1] < energies["f64"][0]
    # and the GPU energy is the oracle's energy of the final field
    assert energies["f64"][-1] == pytest.approx(oracle.energy(outs["f64"], w.h, w.eps), rel=1e-12)


@pytest.mark.parametrize("dtype", ["f32", "f16s"])
def test_sphere_256_full_run(dtype):
    w = wl.SPHERE_256
    phi0 = oracle.init_sphere(w.shape, w.h, w.r0, w.eps)
    stored = phi0.astype(np.float32 if dtype == "f32" else np.float16).astype(np.float64)
    ref = oracle.step(stored, w.h, w.eps, w.dt, w.steps)
    sim = ac.Simulation(w.shape, w.h, w.eps, w.dt, dtype=dtype)
    try:
        sim.init_sphere(r0=w.r0)
        sim.step(w.steps)
        assert sim.status() == ac.AC_OK
        out = sim.to_numpy().astype(np.float64)
    finally:
        sim.close()
    print(f"\n256^3 x {w.steps} {dtype}: max-abs {np.max(np.abs(out - ref)):.2e}, "
          f"rel-L2 {rel_l2(out, ref):.2e}")
    if dtype == "f32":
        assert float(np.max(np.abs(out - ref))) <= TOL_MAXABS["f32"]
    else:
        assert rel_l2(out, ref) <= TOL_RELL2_F16S
