"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with a retyped copy of itself: hand-worked
values, closed-form eigenmodes of the Neumann Laplacian, exact fixed points,
bitwise grid symmetries, the 3D->2D and 2D->1D reductions, conservation of the Laplacian,
the energy gradient identity, the mean-curvature radius law and a published
SplitMix64 known-answer sequence.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2105_09671_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- hand work --

def test_hand_worked_small_grids():
    g = _load("hand_worked_4x4.json")
    h, eps, dt = g["h"], g["eps"], g["dt"]
    for case in g["cases"]:
        shape = tuple(case["shape"])
        phi = np.zeros(shape)
        if "impulse" in case:
            # impulse index given as (x, y[, z]); arrays are [z][y][x]
            phi[tuple(reversed(case["impulse"]))] = 1.0
        else:
            phi[...] = case["uniform"]
        out = oracle.step(phi, h, eps, dt, 1)
        expect = np.zeros(shape)
        if "expect_all" in case:
            expect[...] = case["expect_all"]
        for key, val in case.get("expect", {}).items():
            expect[tuple(reversed(json.loads(key)))] = val
        np.testing.assert_allclose(out, expect, rtol=0, atol=2e-16 * 8,
                                   err_msg=case["name"])


# ------------------------------------------------------------- fixed points --

@pytest.mark.parametrize("shape", [(9, 13), (5, 6, 7)])
@pytest.mark.parametrize("value", [1.0, -1.0, 0.0])
def test_fixed_points_bitwise(shape, value):
    phi = np.full(shape, value)
    h = 1.0 / shape[-1]
    out = oracle.step(phi, h, 0.02, 0.1 * h * h, 37)
    assert np.array_equal(out, phi)


# --------------------------------------------- closed form: Neumann eigenmodes

def _mode(shape, ks):
    """Product of cos(pi k (i + 1/2) / N) per axis -- an exact eigenvector of
    the replicate-padded second difference (the DCT-II basis)."""
    axes = [np.cos(np.pi * k * (np.arange(n) + 0.5) / n) for n, k in zip(shape, ks)]
    out = axes[0]
    for a in axes[1:]:
        out = np.multiply.outer(out, a)
    return out


@pytest.mark.parametrize("shape,ks", [
    ((7, 12), (0, 3)), ((7, 12), (2, 1)), ((16, 16), (5, 5)), ((9, 8), (8, 7)),
    ((5, 6, 7), (1, 0, 2)), ((6, 6, 6), (3, 2, 1)),
])
def test_linear_regime_matches_dct_eigenvalue(shape, ks):
    # With amplitude 1e-8 the cubic term is 1e-16 relative; the scheme is then
    # phi' = (1 + alpha) phi + (dt/h^2) D phi with D phi = lambda phi, where
    # lambda = -4 sum_axes sin^2(pi k / (2 N)).
    h, eps = 1.0 / 12, 0.07
    dt = 0.1 * h * h
    alpha, beta = dt / eps ** 2, dt / (h * h)
    delta, n = 1e-8, 40
    phi0 = delta * _mode(shape, ks)
    lam = -4.0 * sum(math.sin(math.pi * k / (2 * N)) ** 2 for N, k in zip(shape, ks))
    gain = 1.0 + alpha + beta * lam
    out = oracle.step(phi0, h, eps, dt, n)
    expect = phi0 * gain ** n
    # rounding noise is ~1e-16 of the initial amplitude; a wrong gain, sign or
    # boundary rule shows up as an O(delta * n * error) mismatch
    err = np.abs(out - expect)
    assert np.all(err <= 1e-9 * np.abs(expect) + 1e-13 * delta)


# ------------------------------------------------------------------ symmetry --

def test_mirror_and_transpose_symmetry_2d_bitwise():
    phi = wl.random_field((24, 24), seed=3, lo=-1.0, hi=1.0)
    h = 1.0 / 24
    args = (h, 0.05, 0.1 * h * h, 25)
    ref = oracle.step(phi, *args)
    assert np.array_equal(oracle.step(phi[:, ::-1].copy(), *args), ref[:, ::-1])
    assert np.array_equal(oracle.step(phi[::-1, :].copy(), *args), ref[::-1, :])
    assert np.array_equal(oracle.step(phi.T.copy(), *args), ref.T)


def test_mirror_symmetry_3d_bitwise():
    phi = wl.random_field((10, 11, 12), seed=4)
    h = 1.0 / 12
    args = (h, 0.05, 0.1 * h * h, 9)
    ref = oracle.step(phi, *args)
    for ax in range(3):
        flipped = np.flip(phi, axis=ax).copy()
        assert np.array_equal(oracle.step(flipped, *args), np.flip(ref, axis=ax))
    # exchanging x and y keeps the paired sum order, so it is bitwise too
    sq = wl.random_field((6, 10, 10), seed=5)
    r = oracle.step(sq, *args)
    assert np.array_equal(oracle.step(np.swapaxes(sq, 1, 2).copy(), *args),
                          np.swapaxes(r, 1, 2))


def test_z_invariant_3d_equals_2d():
    f2 = wl.random_field((9, 14), seed=6)
    f3 = np.repeat(f2[None], 5, axis=0)
    h = 1.0 / 14
    args = (h, 0.04, 0.1 * h * h, 30)
    o2 = oracle.step(f2, *args)
    o3 = oracle.step(f3, *args)
    for k in range(5):
        np.testing.assert_allclose(o3[k], o2, rtol=0, atol=1e-14)


def test_x_only_2d_equals_the_1d_scheme():
    # a field constant in y stays constant in y, and each row follows the 1D
    # scheme (same Euler step, second difference with replicated ends); the
    # 2D sum adds the y pair (S + N = 2 phi exactly) before subtracting 4 phi,
    # so the two agree to rounding, not bitwise
    nx, ny, n = 23, 7, 40
    h = 1.0 / nx
    eps, dt = 0.05, 0.1 * h * h
    f1 = wl.random_field((1, nx), seed=12)[0]
    got = oracle.step(np.repeat(f1[None], ny, axis=0), h, eps, dt, n)
    ref = f1.copy()
    for _ in range(n):
        w = np.concatenate(([ref[0]], ref[:-1]))
        e = np.concatenate((ref[1:], [ref[-1]]))
        ref = ref + dt * ((ref - ref ** 3) / eps ** 2 + (w - 2.0 * ref + e) / h ** 2)
    for j in range(ny):
        assert np.array_equal(got[j], got[0])
    np.testing.assert_allclose(got[0], ref, rtol=0, atol=1e-13)


# --------------------------------------------------------------- conservation

@pytest.mark.parametrize("shape", [(13, 17), (6, 7, 8)])
def test_laplacian_conserves_mass_under_neumann(shape):
    # sum(phi') - sum(phi) = alpha * sum(phi - phi^3): the Neumann Laplacian sums to 0
    phi = wl.random_field(shape, seed=7)
    h, eps = 1.0 / shape[-1], 0.3
    dt = 0.1 * h * h
    out = oracle.step(phi, h, eps, dt, 1)
    alpha = dt / eps ** 2
    lhs = out.sum() - phi.sum()
    rhs = alpha * np.sum(phi - phi ** 3)
    assert abs(lhs - rhs) <= 1e-13 * phi.size


# -------------------------------------------------------------------- energy --

@pytest.mark.parametrize("shape", [(5, 4), (3, 4, 5)])
def test_energy_gradient_is_minus_rhs(shape):
    # dE_h/dphi_c = -h^d (phi'_c - phi_c) / dt : the step is gradient descent on E_h
    phi = wl.random_field(shape, seed=8, lo=-1.2, hi=1.2)
    h, eps = 1.0 / shape[-1], 0.2
    dt = 0.1 * h * h
    d = len(shape)
    rhs = (oracle.step(phi, h, eps, dt, 1) - phi) / dt
    delta = 1e-5
    for c in range(phi.size):
        idx = np.unravel_index(c, shape)
        p, m = phi.copy(), phi.copy()
        p[idx] += delta
        m[idx] -= delta
        g = (oracle.energy(p, h, eps) - oracle.energy(m, h, eps)) / (2 * delta)
        assert g == pytest.approx(-h ** d * rhs[idx], rel=1e-6, abs=1e-10 * h ** d)


def test_energy_closed_forms():
    h, eps = 1.0 / 8, 0.1
    for c in (0.3, -0.7, 1.0):
        phi = np.full((6, 8), c)
        expect = 48 * h * h * 0.25 * (c * c - 1) ** 2 / eps ** 2
        assert oracle.energy(phi, h, eps) == pytest.approx(expect, rel=1e-14, abs=1e-300)
    # a ramp phi = a*x only has x-gradient (a) on the (nx-1)*ny interior x-faces;
    # large eps makes the bulk term negligible next to it
    a = 0.01
    x = (np.arange(8) + 0.5) * h
    phi = np.tile(a * x, (6, 1))
    bulk = h * h * np.sum(0.25 * (phi ** 2 - 1) ** 2) / 1e6 ** 2
    grad = 0.5 * a * a * 7 * 6 * h * h
    assert oracle.energy(phi, h, 1e6) == pytest.approx(bulk + grad, rel=1e-12)


def test_energy_decreases_monotonically():
    w = wl.CIRCLE_64
    phi = oracle.init_sphere(w.shape, w.h, w.r0, w.eps)
    e_prev = oracle.energy(phi, w.h, w.eps)
    for _ in range(20):
        phi = oracle.step(phi, w.h, w.eps, w.dt, 50)
        e = oracle.energy(phi, w.h, w.eps)
        assert e < e_prev
        e_prev = e
    phi = oracle.init_random((40, 40), seed=1)
    h, eps = 1 / 40, 0.03
    e_prev = oracle.energy(phi, h, eps)
    for _ in range(20):
        phi = oracle.step(phi, h, eps, 0.1 * h * h, 25)
        e = oracle.energy(phi, h, eps)
        assert e < e_prev
        e_prev = e


# ------------------------------------------------------------- radius laws --

def _r2_slope(shape, h, eps, r0, steps, samples):
    dt = 0.1 * h * h
    phi = oracle.init_sphere(shape, h, r0, eps)
    ts, r2 = [], []
    per = steps // samples
    for s in range(samples + 1):
        if s:
            phi = oracle.step(phi, h, eps, dt, per)
        v = oracle.phase_volume(phi, h)
        ts.append(s * per * dt)
        r2.append(oracle.radius_from_volume(v, len(shape)) ** 2)
    return np.polyfit(ts, r2, 1)[0]


def test_circle_radius_law_64():
    w = wl.CIRCLE_64
    slope = _r2_slope(w.shape, w.h, w.eps, w.r0, w.steps, 10)
    assert slope == pytest.approx(-2.0, rel=0.10)


@pytest.mark.slow
def test_circle_radius_law_256():
    slope = _r2_slope((256, 256), 1 / 256, 0.015, 0.25, 1000, 10)
    assert slope == pytest.approx(-2.0, rel=0.02)


@pytest.mark.slow
def test_sphere_radius_law_96():
    slope = _r2_slope((96, 96, 96), 1 / 96, 0.015, 0.25, 400, 4)
    assert slope == pytest.approx(-4.0, rel=0.05)


def test_flat_interface_nearly_stationary():
    # the tanh profile is the 1D equilibrium, so a straight interface barely moves,
    # while a circle of the same width visibly shrinks
    n, eps = 64, 0.03
    h = 1 / n
    x = (np.arange(n) + 0.5) * h
    flat = np.tile(np.tanh((x - 0.5) / (math.sqrt(2) * eps)), (n, 1))
    out = oracle.step(flat, h, eps, 0.1 * h * h, 500)
    circ = oracle.init_sphere((n, n), h, 0.25, eps)
    circ_out = oracle.step(circ, h, eps, 0.1 * h * h, 500)
    moved_flat = np.max(np.abs(out - flat))
    moved_circ = np.max(np.abs(circ_out - circ))
    assert moved_flat < 0.05 * moved_circ
    assert moved_flat < 1.5e-2  # O((h/eps)^2) discretisation drift only


# ------------------------------------------------------- initial conditions --

def test_splitmix64_known_answers():
    g = _load("splitmix64_kat.json")
    got = [oracle.splitmix64(g["seed"], i) for i in range(len(g["outputs_hex"]))]
    assert got == [int(x, 16) for x in g["outputs_hex"]]


def test_random_init_range_and_reproducible():
    a = oracle.init_random((64, 64), seed=11)
    b = oracle.init_random((64, 64), seed=11)
    c = oracle.init_random((64, 64), seed=12)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= -0.1 and a.max() < 0.1
    assert abs(a.mean()) < 0.005
    # first cell of seed 0 is the first SplitMix64 output mapped to [-0.1, 0.1)
    z = int(_load("splitmix64_kat.json")["outputs_hex"][0], 16)
    assert oracle.init_random((1,), seed=0)[0] == 0.1 * (2.0 * ((z >> 11) * 2.0 ** -53) - 1.0)


def test_circle_init_sign_and_symmetry():
    n = 64
    h, r0, eps = 1 / n, 0.25, 0.015
    phi = oracle.init_sphere((n, n), h, r0, eps)
    c = (np.arange(n) + 0.5) * h - 0.5
    r = np.sqrt(c[None, :] ** 2 + c[:, None] ** 2)
    assert np.array_equal(phi > 0, r < r0)
    assert np.array_equal(phi, phi[::-1, :]) and np.array_equal(phi, phi.T)
    # Volume of the diffuse disc/ball: the tanh step (1 + tanh((R - r)/w))/2,
    # w = sqrt(2) eps, is a Fermi function of temperature w/2, so by the
    # Sommerfeld expansion its area is pi R^2 + pi^3 w^2 / 12 and its volume
    # 4/3 pi R^3 + pi^3 R w^2 / 3 (odd moments vanish); the midpoint rule on
    # cell centres is spectrally accurate for it.
    w = math.sqrt(2) * eps
    v = oracle.phase_volume(phi, h)
    assert v == pytest.approx(math.pi * r0 ** 2 + math.pi ** 3 * w * w / 12, rel=1e-6)
    n3, r3, e3 = 64, 0.3, 0.02
    w3 = math.sqrt(2) * e3
    s = oracle.init_sphere((n3, n3, n3), 1 / n3, r3, e3)
    assert np.array_equal(s, s[::-1]) and np.array_equal(s, np.swapaxes(s, 0, 2))
    assert oracle.phase_volume(s, 1 / n3) == pytest.approx(
        4 / 3 * math.pi * r3 ** 3 + math.pi ** 3 * r3 * w3 * w3 / 3, rel=1e-6)


def test_phase_volume_extremes():
    assert oracle.phase_volume(np.ones((8, 8)), 1 / 8) == pytest.approx(1.0, rel=1e-15)
    assert oracle.phase_volume(-np.ones((4, 4, 4)), 1 / 4) == 0.0


def test_eps_m_spans_m_cells_between_pm_09():
    # Eq. (emvalue): the tanh profile goes from -0.9 to 0.9 across m cells
    for h, m in ((1 / 200, 10), (1 / 100, 12), (1 / 64, 4)):
        e = oracle.eps_m(h, m)
        assert math.tanh((m * h / 2) / (math.sqrt(2) * e)) == pytest.approx(0.9, rel=1e-14)


def test_err_metric():
    a = [np.zeros((3, 3)), np.ones((3, 3))]
    assert oracle.err_metric(a, a) == 0.0
    b = [x + 0.25 for x in a]
    assert oracle.err_metric(a, b) == pytest.approx(0.25)
