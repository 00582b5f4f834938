"""Grids taller than CUDA's 65535 blocks per grid dimension: 2D with
ny / 4 > 65535 block rows and 3D with nz > 65535 planes.  The cell-wise
kernels (direct stencil, initial conditions) cover y and z beyond that by
grid-stride loops; the streaming kernels index items in one dimension.
Every schedule tried must match the FP64 oracle, and the initial conditions
must match the oracle's generators, over the whole height."""
import numpy as np
import pytest

import oracle
import paper_2105_09671_gb300 as ac

from gpu_util import NP, TOL_MAXABS, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

CASES = {
    # (shape, schedules (variant, k, tile) besides the default)
    (300000, 8): [(ac.AC_VARIANT_DIRECT, 1, 0), (ac.AC_VARIANT_STREAM, 1, 0),
                  (ac.AC_VARIANT_STREAM, 4, 0)],
    (70000, 4, 8): [(ac.AC_VARIANT_DIRECT, 1, 0), (ac.AC_VARIANT_STREAM, 1, 1),
                    (ac.AC_VARIANT_STREAM, 2, 2)],
}


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape", list(CASES))
def test_tall_grid_init_and_steps(shape, dtype):
    h = 1.0 / shape[-1]
    eps, dt = 2.5 * h, 0.1 * h * h
    sim = ac.Simulation(shape, h, eps, dt, dtype=dtype)
    try:
        sim.init_random(seed=5, amplitude=0.1)
        rnd = sim.to_numpy()
        sim.init_sphere(r0=0.3, center=(0.5, 0.5, 0.5))
        sph = sim.to_numpy().astype(np.float64)
    finally:
        sim.close()
    assert np.array_equal(rnd, oracle.init_random(shape, seed=5, amplitude=0.1).astype(NP[dtype]))
    ref_sph = oracle.init_sphere(shape, h, 0.3, eps)
    if dtype == "f64":
        np.testing.assert_allclose(sph, ref_sph, rtol=0, atol=4.5e-16)
    else:
        ref = ref_sph.astype(np.float32).astype(np.float64)
        ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(sph - ref) <= ulp)

    phi0 = rnd.astype(np.float64)
    n = 5
    ref = oracle_run(phi0, h, eps, dt, n, dtype)
    for variant, k, tile in [(None, None, None)] + CASES[shape]:
        out = gpu_run(phi0, h, eps, dt, n, dtype, variant, k, tile)
        err = float(np.max(np.abs(out - ref)))
        assert err <= TOL_MAXABS[dtype], f"{shape} {dtype} v{variant} k{k} t{tile}: {err:.3e}"
