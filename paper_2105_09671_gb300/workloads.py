"""Seeded synthetic workloads: grid recipes and generic random fields.

This module holds parameters and seeded random arrays only -- none of the
scheme's arithmetic -- so that the CUDA path and the CPU oracle can both be
fed from it without sharing any of the method.

Recipes follow the paper's setup (Section 2 and 3): unit domain, cell size
h = 1/Nx, time step dt = 0.1 h^2, interface width eps given per workload.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    shape: tuple          # (ny, nx) or (nz, ny, nx)
    eps: float
    steps: int
    init: str             # "sphere" (circle in 2D) or "random"
    r0: float = 0.25
    seed: int = 0

    @property
    def ndim(self) -> int:
        return len(self.shape)

    @property
    def nx(self) -> int:
        return self.shape[-1]

    @property
    def h(self) -> float:
        return 1.0 / self.nx

    @property
    def dt(self) -> float:
        return 0.1 * self.h * self.h

    @property
    def cells(self) -> int:
        return int(np.prod(self.shape))


# 2D circle, 64^2, FP64 parity case; radius checked against the shrinking law.
CIRCLE_64 = Workload("circle2d_64", (64, 64), eps=0.015, steps=1000, init="sphere")
# 2D phase separation, 4096^2, random initial state in [-0.1, 0.1).
SEPARATION_4096 = Workload("separation2d_4096", (4096, 4096), eps=0.004, steps=5000,
                           init="random", seed=0)
# 3D sphere, 512^3 (the FP32 / FP16-storage throughput workload).
SPHERE_512 = Workload("sphere3d_512", (512, 512, 512), eps=0.003, steps=2000, init="sphere")
# 3D sphere at 256^3 for the FP16-storage error report against FP64.
SPHERE_256 = Workload("sphere3d_256", (256, 256, 256), eps=0.003, steps=2000, init="sphere")


def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Generic seeded FP64 field, uniform in [lo, hi) (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape)


def smooth_field(shape, seed: int, modes: int = 4, amp: float = 0.9) -> np.ndarray:
    """Seeded smooth field: a sum of a few random cosine modes on cell centres,
    scaled to max |phi| <= amp.  Used as a generic parity input with interfaces."""
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[(np.arange(n) + 0.5) / n for n in shape], indexing="ij")
    f = np.zeros(shape)
    for _ in range(modes):
        k = rng.integers(1, 6, size=len(shape))
        ph = rng.uniform(0, 2 * np.pi, size=len(shape))
        term = np.ones(shape)
        for g, kk, pp in zip(grids, k, ph):
            term = term * np.cos(np.pi * kk * g + pp)
        f += rng.uniform(-1, 1) * term
    m = np.max(np.abs(f))
    return amp * f / m if m > 0 else f


def batch_instances(count: int = 512, seed: int = 0, steps: int = 2000):
    """The batched workload: `count` independent 2D grids with sizes drawn
    uniformly from {64, 96, ..., 1024}^2, h = 1/n, dt = 0.1 h^2, eps drawn
    uniformly from [3h, 6h]; even indices hold a tanh circle of radius drawn
    from [0.1, 0.4] centred at (0.5, 0.5), odd indices a random state of
    amplitude 0.1 (SplitMix64 seed 1000 + index).  One seeded draw.
    Returns dicts with n, h, eps, dt, init, r0, seed, steps."""
    rng = np.random.default_rng(seed)
    sizes = np.arange(64, 1025, 32)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        h = 1.0 / n
        eps = float(rng.uniform(3.0, 6.0)) * h
        r0 = float(rng.uniform(0.1, 0.4))
        out.append(dict(n=n, h=h, eps=eps, dt=0.1 * h * h, init="sphere" if i % 2 == 0 else "random",
                        r0=r0, seed=1000 + i, steps=steps))
    return out


@dataclasses.dataclass(frozen=True)
class ShapeCase:
    """One of the paper's mean-curvature / separation runs (Section 3.2, 3.3,
    Tables 1-3), with the interface width eps_m given by its m (Eq. emvalue).

    Readings: h is the domain length over the cell count (on (0, 2) x (0, 1)
    the dumbbell's 400 x 200 cells have h = 1/200; on (-1, 1)^3, 200 cells
    per side give h = 0.01); the step count is the printed final time T over
    dt = 0.1 h^2 (where a table's iteration count disagrees with T, T wins)."""
    name: str
    kind: str             # "dumbbell", "star", "torus", "sphere" or "random"
    shape: tuple          # (ny, nx) or (nz, ny, nx)
    h: float
    m: float              # eps = eps_m(h, m)
    steps: int
    lower: tuple = (0.0, 0.0, 0.0)
    params: tuple = ()    # dumbbell (r0,), torus (r1, r2), sphere (r0,)
    seed: int = 0

    @property
    def ndim(self) -> int:
        return len(self.shape)

    @property
    def dt(self) -> float:
        return 0.1 * self.h * self.h

    @property
    def cells(self) -> int:
        return int(np.prod(self.shape))


# Table 3's runs: 2D with eps_10 on 200^2 (dumbbell 400 x 200 on (0,2)x(0,1));
# 3D with eps_12 on 100^3 (dumbbell 200 x 100 x 100; star and torus on
# (-1,1)^3 with 200 cells per side).
PAPER_CASES = (
    ShapeCase("circle2d", "sphere", (200, 200), 1 / 200, 10, 12000, params=(0.25,)),
    ShapeCase("dumbbell2d", "dumbbell", (200, 400), 1 / 200, 10, 3760, params=(0.2,)),
    ShapeCase("star2d", "star", (200, 200), 1 / 200, 10, 13000),
    ShapeCase("torus2d", "torus", (200, 200), 1 / 200, 10, 23000, params=(0.4, 0.3)),
    ShapeCase("separation2d", "random", (200, 200), 1 / 200, 10, 12000, seed=1),
    ShapeCase("sphere3d", "sphere", (100, 100, 100), 1 / 100, 12, 2000, params=(0.25,)),
    ShapeCase("dumbbell3d", "dumbbell", (100, 100, 200), 1 / 100, 12, 250, params=(0.25,)),
    ShapeCase("star3d", "star", (200, 200, 200), 0.01, 12, 2000, lower=(-1.0, -1.0, -1.0)),
    ShapeCase("torus3d", "torus", (200, 200, 200), 0.01, 12, 1000, lower=(-1.0, -1.0, -1.0),
              params=(0.3, 0.3)),
    ShapeCase("separation3d", "random", (100, 100, 100), 1 / 100, 12, 2000, seed=2),
)
