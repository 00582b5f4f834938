"""Pins of the oracle's further initial shapes (Section 3.1) against facts
the equations fix: exact values inside the dumbbell's bar, zero crossings at
the printed radii, the symmetries of each shape, and phase volumes against
closed forms (Pappus for the torus, the polar-area integral for the star,
the union of discs and bar for the dumbbell)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import shapes as S


def _volume(phi, h, ndim):
    return h ** ndim * float(np.sum((1.0 + phi) / 2.0))


# ----------------------------------------------------------------- dumbbell --

def test_dumbbell_bar_is_exactly_one_and_sharp():
    for p in [(1.0, 0.5), (0.45, 0.41), (1.59, 0.59)]:
        assert S.dumbbell(*p, r0=0.2, eps=0.01) == 1.0
        assert S.dumbbell(p[0], p[1], 0.5, r0=0.25, eps=0.01) == 1.0
    # just outside the bar between the discs: the far field -1
    assert S.dumbbell(1.0, 0.61, r0=0.2, eps=0.002) == pytest.approx(-1.0, abs=1e-12)
    assert S.dumbbell(1.0, 0.5, 0.62, r0=0.25, eps=0.002) == pytest.approx(-1.0, abs=1e-12)


def test_dumbbell_discs_cross_zero_at_r0_on_their_outer_side():
    eps = 0.002
    for r0 in (0.2, 0.25):
        assert S.dumbbell(0.3 - r0, 0.5, r0=r0, eps=eps) == pytest.approx(0.0, abs=1e-12)
        assert S.dumbbell(1.7 + r0, 0.5, r0=r0, eps=eps) == pytest.approx(0.0, abs=1e-12)
        assert S.dumbbell(0.3, 0.5 + r0, r0=r0, eps=eps) == pytest.approx(0.0, abs=1e-12)
        assert S.dumbbell(0.3, 0.5, 0.5 - r0, r0=r0, eps=eps) == pytest.approx(0.0, abs=1e-12)
        assert S.dumbbell(0.3, 0.5, r0=r0, eps=eps) == pytest.approx(1.0, abs=1e-12)


def test_dumbbell_mirror_symmetry():
    h = 1.0 / 200
    phi = S.on_grid(S.dumbbell, (200, 400), h, r0=0.2, eps=0.01)
    # coordinates of mirrored cells round differently: allow 1e-12 at the interface
    np.testing.assert_allclose(phi, phi[:, ::-1], rtol=0, atol=1e-12)
    np.testing.assert_allclose(phi, phi[::-1, :], rtol=0, atol=1e-12)


def test_dumbbell_area_is_the_union_of_discs_and_bar():
    r0, eps = 0.2, 0.0005
    # area of one disc inside the bar's strip |y - 0.5| < 0.1, x in (0.4, 0.5)
    cap, _ = integrate.quad(lambda x: 2.0 * min(0.1, math.sqrt(max(0.0, r0 * r0 - (x - 0.3) ** 2))),
                            0.4, 0.3 + r0)
    union = 2.0 * math.pi * r0 * r0 + 1.2 * 0.2 - 2.0 * cap
    h = 1.0 / 2000
    phi = S.on_grid(S.dumbbell, (2000, 4000), h, r0=r0, eps=eps)
    assert _volume(phi, h, 2) == pytest.approx(union, rel=1e-3)


# --------------------------------------------------------------------- star --

def test_star_2d_zero_set_at_the_printed_radius():
    eps = 0.002
    for th in np.linspace(0.1, 2 * math.pi - 0.1, 13):
        r = 0.25 + 0.1 * math.cos(6 * th)
        x, y = 0.5 + r * math.cos(th), 0.5 + r * math.sin(th)
        assert S.star(x, y, eps=eps) == pytest.approx(0.0, abs=1e-9)
    # tips (theta = 0) at r = 0.35, gaps (theta = pi/6) at r = 0.15
    assert S.star(0.5 + 0.34, 0.5, eps=eps) > 0.99
    assert S.star(0.5 + 0.16 * math.cos(math.pi / 6), 0.5 + 0.16 * math.sin(math.pi / 6), eps=eps) < -0.99


def test_star_2d_six_fold_and_mirror_symmetry():
    rng = np.random.default_rng(1)
    u, v = rng.uniform(-0.45, 0.45, size=(2, 500))
    a = math.pi / 3
    ur, vr = u * math.cos(a) - v * math.sin(a), u * math.sin(a) + v * math.cos(a)
    p = S.star(0.5 + u, 0.5 + v, eps=0.01)
    np.testing.assert_allclose(S.star(0.5 + ur, 0.5 + vr, eps=0.01), p, rtol=0, atol=1e-10)
    np.testing.assert_allclose(S.star(0.5 + u, 0.5 - v, eps=0.01), p, rtol=0, atol=1e-12)


def test_star_2d_area_is_the_polar_integral():
    # (1/2) int (0.25 + 0.1 cos 6t)^2 dt = pi (0.25^2 + 0.1^2 / 2)
    exact = math.pi * (0.25 ** 2 + 0.1 ** 2 / 2)
    h = 1.0 / 2000
    phi = S.on_grid(S.star, (2000, 2000), h, eps=0.0005)
    assert _volume(phi, h, 2) == pytest.approx(exact, rel=2e-3)


def test_star_3d_reading():
    eps = 0.002
    # zero set at |p| = 0.7 + 0.2 cos 6t, t the angle of (x, z): on the x axis 0.9
    assert S.star(0.9, 0.0, 0.0, eps=eps) == pytest.approx(0.0, abs=1e-12)
    assert S.star(0.0, 0.9 - 0.4, 0.0, eps=eps) > 0.99      # (x, z) = 0: t = pi, r* = 0.9
    t = math.pi / 6                                           # a gap: r* = 0.5
    assert S.star(0.5 * math.cos(t), 0.0, 0.5 * math.sin(t), eps=eps) == pytest.approx(0.0, abs=1e-9)
    rng = np.random.default_rng(2)
    x, y, z = rng.uniform(-0.95, 0.95, size=(3, 400))
    a = math.pi / 3
    xr, zr = x * math.cos(a) - z * math.sin(a), x * math.sin(a) + z * math.cos(a)
    p = S.star(x, y, z, eps=0.02)
    np.testing.assert_allclose(S.star(xr, y, zr, eps=0.02), p, rtol=0, atol=1e-10)
    np.testing.assert_allclose(S.star(x, -y, z, eps=0.02), p, rtol=0, atol=1e-12)


def test_star_3d_volume():
    # {|p| < R(t)}: (2/3) int R(t)^3 dt = (4 pi / 3) (a^3 + 1.5 a b^2), a = 0.7, b = 0.2
    a, b = 0.7, 0.2
    exact = 4 * math.pi / 3 * (a ** 3 + 1.5 * a * b * b)
    n = 240
    h = 2.0 / n
    phi = S.on_grid(S.star, (n, n, n), h, lower=(-1.0, -1.0, -1.0), eps=0.005)
    assert _volume(phi, h, 3) == pytest.approx(exact, rel=1e-2)


# -------------------------------------------------------------------- torus --

def test_torus_2d_annulus():
    eps, r1, r2 = 0.002, 0.4, 0.3
    assert S.torus(0.5 + r1, 0.5, r1=r1, r2=r2, eps=eps) == pytest.approx(0.0, abs=1e-12)
    assert S.torus(0.5, 0.5 - r2, r1=r1, r2=r2, eps=eps) == pytest.approx(0.0, abs=1e-12)
    assert S.torus(0.5 + 0.35, 0.5, r1=r1, r2=r2, eps=eps) == pytest.approx(1.0, abs=1e-12)
    assert S.torus(0.5, 0.5, r1=r1, r2=r2, eps=eps) == pytest.approx(-1.0, abs=1e-12)
    assert S.torus(0.02, 0.02, r1=r1, r2=r2, eps=eps) == pytest.approx(-1.0, abs=1e-12)
    h = 1.0 / 2000
    phi = S.on_grid(S.torus, (2000, 2000), h, r1=r1, r2=r2, eps=0.0005)
    assert _volume(phi, h, 2) == pytest.approx(math.pi * (r1 * r1 - r2 * r2), rel=1e-3)


def test_torus_3d_reading():
    eps = 0.002
    r1, r2 = 0.5, 0.2
    assert S.torus(r1 + r2, 0.0, 0.0, r1=r1, r2=r2, eps=eps) == pytest.approx(0.0, abs=1e-12)
    assert S.torus(0.0, r1 - r2, 0.0, r1=r1, r2=r2, eps=eps) == pytest.approx(0.0, abs=1e-12)
    assert S.torus(0.0, -r1, r2, r1=r1, r2=r2, eps=eps) == pytest.approx(0.0, abs=1e-12)
    assert S.torus(r1, 0.0, 0.0, r1=r1, r2=r2, eps=eps) == pytest.approx(1.0, abs=1e-12)
    assert S.torus(0.0, 0.0, 0.0, r1=r1, r2=r2, eps=eps) == pytest.approx(-1.0, abs=1e-12)
    rng = np.random.default_rng(3)
    x, y, z = rng.uniform(-0.9, 0.9, size=(3, 400))
    a = 0.7
    xr, yr = x * math.cos(a) - y * math.sin(a), x * math.sin(a) + y * math.cos(a)
    p = S.torus(x, y, z, r1=r1, r2=r2, eps=0.02)
    np.testing.assert_allclose(S.torus(xr, yr, z, r1=r1, r2=r2, eps=0.02), p, rtol=0, atol=1e-12)
    np.testing.assert_allclose(S.torus(x, y, -z, r1=r1, r2=r2, eps=0.02), p, rtol=0, atol=0)


@pytest.mark.parametrize("r1,r2", [(0.5, 0.2), (0.3, 0.3)])
def test_torus_3d_volume_is_pappus(r1, r2):
    n = 200
    h = 2.0 / n
    phi = S.on_grid(S.torus, (n, n, n), h, lower=(-1.0, -1.0, -1.0), r1=r1, r2=r2, eps=0.004)
    assert _volume(phi, h, 3) == pytest.approx(2 * math.pi ** 2 * r1 * r2 * r2, rel=1e-2)


def test_grid_sampling_uses_cell_centres():
    # on_grid evaluates at lower + (i + 1/2) h: compare with point evaluation
    h = 0.1
    phi = S.on_grid(S.torus, (3, 4, 5), h, lower=(-0.2, -0.1, 0.3), r1=0.3, r2=0.1, eps=0.05)
    assert phi.shape == (3, 4, 5)
    k, j, i = 2, 1, 3
    x, y, z = -0.2 + (i + 0.5) * h, -0.1 + (j + 0.5) * h, 0.3 + (k + 0.5) * h
    assert phi[k, j, i] == S.torus(x, y, z, r1=0.3, r2=0.1, eps=0.05)
