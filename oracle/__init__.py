"""FP64 CPU oracle for the explicit Allen-Cahn scheme (arXiv 2105.09671).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke``
and by the benchmark's CPU-baseline leg.  The product path never imports it.

Thin numpy/ctypes wrappers over ``ac_oracle.c``; the arithmetic lives there
(Section 2, Eq. pytorchACeq, Section 3.1).  The Err metric of Eq. (ERReq) and
the radius conversions are written here in numpy, as the paper states them.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import build as _build

_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i64, dbl, u64 = ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
        dp = ctypes.POINTER(ctypes.c_double)
        L.oracle_step2d.argtypes = [i64, i64, dbl, dbl, dbl, dp, dp, i64]
        L.oracle_step2d.restype = ctypes.c_int
        L.oracle_step3d.argtypes = [i64, i64, i64, dbl, dbl, dbl, dp, dp, i64]
        L.oracle_step3d.restype = ctypes.c_int
        L.oracle_init_sphere.argtypes = [i64, i64, i64, dbl, dbl, dbl, dbl, dbl,
                                         dbl, dbl, dbl, dbl, dp]
        L.oracle_init_sphere.restype = None
        L.oracle_splitmix64.argtypes = [u64, u64]
        L.oracle_splitmix64.restype = u64
        L.oracle_init_random.argtypes = [i64, u64, dbl, dp]
        L.oracle_init_random.restype = None
        L.oracle_energy.argtypes = [i64, i64, i64, dbl, dbl, dp]
        L.oracle_energy.restype = dbl
        L.oracle_phase_volume.argtypes = [i64, i64, i64, dbl, dp]
        L.oracle_phase_volume.restype = dbl
        L.oracle_set_num_threads.argtypes = [ctypes.c_int]
        L.oracle_set_num_threads.restype = None
        L.oracle_num_threads.argtypes = []
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def step(phi: np.ndarray, h: float, eps: float, dt: float, nsteps: int) -> np.ndarray:
    """Advance ``phi`` ([ny, nx] or [nz, ny, nx]) by ``nsteps`` Euler steps of
    Eq. (pytorchACeq) with zero-Neumann ghosts (Section 2)."""
    src = _f64c(phi)
    out = np.empty_like(src)
    if src.ndim == 2:
        ny, nx = src.shape
        rc = lib().oracle_step2d(nx, ny, h, eps, dt, _dp(src), _dp(out), int(nsteps))
    elif src.ndim == 3:
        nz, ny, nx = src.shape
        rc = lib().oracle_step3d(nx, ny, nz, h, eps, dt, _dp(src), _dp(out), int(nsteps))
    else:
        raise ValueError("phi must be 2D or 3D")
    if rc != 0:
        raise ValueError("oracle step rejected its arguments")
    return out


def init_sphere(shape, h: float, r0: float, eps: float, center=(0.5, 0.5, 0.5),
                lower=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Circle (2D) / sphere (3D) tanh profile of Section 3.1 on cell centres."""
    if len(shape) == 2:
        ny, nx = shape
        nz = 1
    else:
        nz, ny, nx = shape
    out = np.empty((nz, ny, nx), dtype=np.float64)
    lib().oracle_init_sphere(nx, ny, nz, h, lower[0], lower[1], lower[2],
                             center[0], center[1], center[2], r0, eps, _dp(out))
    return out.reshape(shape)


def splitmix64(seed: int, counter: int) -> int:
    return int(lib().oracle_splitmix64(seed, counter))


def init_random(shape, seed: int, amplitude: float = 0.1) -> np.ndarray:
    """Random initial condition 0.1*rand of Section 3.1 (counter-based SplitMix64)."""
    n = int(np.prod(shape))
    out = np.empty(n, dtype=np.float64)
    lib().oracle_init_random(n, seed, amplitude, _dp(out))
    return out.reshape(shape)


def _dims(phi: np.ndarray):
    if phi.ndim == 2:
        return phi.shape[1], phi.shape[0], 1
    return phi.shape[2], phi.shape[1], phi.shape[0]


def energy(phi: np.ndarray, h: float, eps: float) -> float:
    """Discrete Ginzburg-Landau energy (gradient-flow potential of the scheme)."""
    src = _f64c(phi)
    nx, ny, nz = _dims(src)
    return float(lib().oracle_energy(nx, ny, nz, h, eps, _dp(src)))


def phase_volume(phi: np.ndarray, h: float) -> float:
    """V = h^d * sum (1 + phi) / 2."""
    src = _f64c(phi)
    nx, ny, nz = _dims(src)
    return float(lib().oracle_phase_volume(nx, ny, nz, h, _dp(src)))


def radius_from_volume(v: float, ndim: int) -> float:
    """Equivalent circle / sphere radius of a phase volume."""
    if ndim == 2:
        return math.sqrt(v / math.pi)
    return (3.0 * v / (4.0 * math.pi)) ** (1.0 / 3.0)


def exact_radius(r0: float, t: float, ndim: int) -> float:
    """Mean-curvature shrinking law r(t) = sqrt(r0^2 + 2(1 - d) t), Eq. (exactradiusEQ)."""
    return math.sqrt(r0 * r0 + 2.0 * (1 - ndim) * t)


def err_metric(traj_a, traj_b) -> float:
    """Err of Eq. (ERReq): mean over time steps of the RMS difference."""
    terms = [math.sqrt(float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2)))
             for a, b in zip(traj_a, traj_b)]
    return sum(terms) / len(terms)


def eps_m(h: float, m: float) -> float:
    """Interface-thickness rule of Eq. (emvalue): eps_m = h m / (2 sqrt(2) atanh(0.9))."""
    return h * m / (2.0 * math.sqrt(2.0) * math.atanh(0.9))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops; n <= 0 restores all cores."""
    lib().oracle_set_num_threads(int(n))
