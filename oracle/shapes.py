"""Oracle: the initial shapes of Section 3.1 besides the circle/sphere.

Test infrastructure only (imported by tests/, the smoke check and the
benchmark's CPU baseline); the CUDA library never calls it.  Plain FP64
NumPy, evaluated at arbitrary points so that the tests can probe the
profiles anywhere; `on_grid` samples a shape at the cell centres
x_i = lower + (i + 1/2) h of Section 2.

Every profile is a tanh of a signed distance divided by sqrt(2) eps (phase
+1 inside, -1 outside).  Readings where the text is garbled are stated at
each function.
"""
from __future__ import annotations

import math

import numpy as np

SQRT2 = math.sqrt(2.0)


def _theta(u, v):
    """Polar angle of Section 3.1's star: atan(v/u) for u > 0, pi + atan(v/u)
    otherwise (the angle itself, up to a multiple of 2 pi, for u != 0)."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        base = np.arctan(v / u)
    # u == 0: the quotient is +-inf (atan -> +-pi/2) or nan at the centre
    base = np.where(u == 0.0, np.where(v > 0, math.pi / 2, np.where(v < 0, -math.pi / 2, 0.0)), base)
    return np.where(u > 0.0, base, math.pi + base)


def dumbbell(x, y, z=None, r0=0.2, eps=0.01):
    """Eqs. (2Ddumbellini) / (3Ddumbellini): phi = 1 inside the bar
    0.4 < x < 1.6, 0.4 < y (, z) < 0.6; elsewhere
    1 + tanh((r0 - |p - (0.3, 0.5[, 0.5])|) / (sqrt2 eps))
      + tanh((r0 - |p - (1.7, 0.5[, 0.5])|) / (sqrt2 eps))
    on the domain (0, 2) x (0, 1) (x (0, 1))."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    tr = (y - 0.5) ** 2
    bar = (x > 0.4) & (x < 1.6) & (y > 0.4) & (y < 0.6)
    if z is not None:
        z = np.asarray(z, dtype=np.float64)
        tr = tr + (z - 0.5) ** 2
        bar = bar & (z > 0.4) & (z < 0.6)
    w = SQRT2 * eps
    left = np.tanh((r0 - np.sqrt((x - 0.3) ** 2 + tr)) / w)
    right = np.tanh((r0 - np.sqrt((x - 1.7) ** 2 + tr)) / w)
    return np.where(bar, 1.0, 1.0 + left + right)


def star(x, y, z=None, eps=0.01):
    """Eqs. (2Dstarini) / (3Dstarini).

    2D (unit square): tanh((0.25 + 0.1 cos 6 theta - r) / (sqrt2 eps)), r and
    theta about (0.5, 0.5).

    3D (domain (-1, 1)^3): tanh((0.7 + 0.2 cos 6 theta - |p|) / (sqrt2 eps))
    with r = |p| about the origin.  Reading: the printed angle test "x > 0.5"
    belongs to the 2D form; with the centre at the origin theta is the polar
    angle of (x, z) about the origin, i.e. atan(z/x) for x > 0 and
    pi + atan(z/x) otherwise (a six-lobed body of revolution about y)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    w = SQRT2 * eps
    if z is None:
        u, v = x - 0.5, y - 0.5
        r = np.sqrt(u * u + v * v)
        return np.tanh((0.25 + 0.1 * np.cos(6.0 * _theta(u, v)) - r) / w)
    z = np.asarray(z, dtype=np.float64)
    r = np.sqrt(x * x + y * y + z * z)
    return np.tanh((0.7 + 0.2 * np.cos(6.0 * _theta(x, z)) - r) / w)


def torus(x, y, z=None, r1=0.4, r2=0.3, eps=0.01):
    """Eqs. (2Dtorusini) / (3Dtorusini).

    2D (unit square, annulus about (0.5, 0.5), radii r2 < r1):
      -1 + tanh((r1 - r) / (sqrt2 eps)) - tanh((r2 - r) / (sqrt2 eps)).

    3D (domain (-1, 1)^3, ring of major radius r1 about the z axis, tube
    radius r2).  Reading: the printed 3D expression is the signed distance
    d = sqrt(z^2 + (sqrt(x^2 + y^2) - r1)^2) - r2 to the tube (positive
    outside), not a phase field; it is used as the distance of the same tanh
    profile as every other shape, phi = tanh(-d / (sqrt2 eps)) (+1 inside the
    tube)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    w = SQRT2 * eps
    if z is None:
        r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2)
        return -1.0 + np.tanh((r1 - r) / w) - np.tanh((r2 - r) / w)
    z = np.asarray(z, dtype=np.float64)
    rho = np.sqrt(x * x + y * y)
    d = np.sqrt(z * z + (rho - r1) ** 2) - r2
    return np.tanh(-d / w)


def on_grid(fn, shape, h: float, lower=(0.0, 0.0, 0.0), **kw) -> np.ndarray:
    """Sample a shape at the cell centres lower + (i + 1/2) h of a grid of
    `shape` (ny, nx) or (nz, ny, nx)."""
    if len(shape) == 2:
        ny, nx = shape
        x = lower[0] + (np.arange(nx) + 0.5) * h
        y = lower[1] + (np.arange(ny) + 0.5) * h
        return fn(x[None, :], y[:, None], None, **kw)
    nz, ny, nx = shape
    x = lower[0] + (np.arange(nx) + 0.5) * h
    y = lower[1] + (np.arange(ny) + 0.5) * h
    z = lower[2] + (np.arange(nz) + 0.5) * h
    return fn(x[None, None, :], y[None, :, None], z[:, None, None], **kw)
