"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
the oracle on the same stored inputs."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2105_09671_gb300 as ac

NP = {"f64": np.float64, "f32": np.float32, "f16s": np.float16}
# Tolerances after the stated step counts (max-abs against the FP64 oracle on
# the same stored initial values): FP64 1e-12 and FP32 1e-5; FP16 storage is
# measured by relative L2 (1e-3).
TOL_MAXABS = {"f64": 1e-12, "f32": 1e-5}
TOL_RELL2_F16S = 1e-3


def schedules(ndim: int, dtype: str):
    """Every (variant, k, tile) the library accepts for this grid kind."""
    from paper_2105_09671_gb300 import _lib as L
    out = [(L.AC_VARIANT_DIRECT, 1, 0)]
    # deepest k per (grid kind, storage type, tile)
    kmax = {(2, "f64"): [8], (2, "f32"): [8, 6], (2, "f16s"): [6],
            (3, "f64"): [2, 2, 2], (3, "f32"): [3, 3, 3], (3, "f16s"): [3, 3, 3]}
    for tile, km in enumerate(kmax[(ndim, dtype)]):
        for k in range(1, km + 1):
            out.append((L.AC_VARIANT_STREAM, k, tile))
    return out


def stored(phi0: np.ndarray, dtype: str) -> np.ndarray:
    """The FP64 values of phi0 after rounding to the storage type."""
    return phi0.astype(NP[dtype]).astype(np.float64)


def gpu_run(phi0, h, eps, dt, n, dtype, variant=None, k=None, tile=None, pitch_x=None):
    sim = ac.Simulation(phi0.shape, h, eps, dt, dtype=dtype, pitch_x=pitch_x)
    try:
        sim.load(phi0)
        if variant is not None:
            sim.set_schedule(variant, k)
        if tile is not None:
            sim.set_tile(tile)
        sim.step(n)
        assert sim.status() == ac.AC_OK
        return sim.to_numpy().astype(np.float64)
    finally:
        sim.close()


def oracle_run(phi0, h, eps, dt, n, dtype):
    return oracle.step(stored(phi0, dtype), h, eps, dt, n)


def rel_l2(a, b) -> float:
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def assert_parity(out, ref, dtype, what=""):
    if dtype == "f16s":
        r = rel_l2(out, ref)
        assert r <= TOL_RELL2_F16S, f"{what}: rel-L2 {r:.3e}"
    else:
        err = float(np.max(np.abs(out - ref))) if out.size else 0.0
        assert err <= TOL_MAXABS[dtype], f"{what}: max-abs {err:.3e}"
