"""The heat equation phi_t = Lap phi as the eps -> infinity limit of the
scheme (no reaction term): the oracle against the exact discrete solution.

The cosine products cos(pi k (i + 1/2) / N) are exact eigenvectors of the
replicate-padded (zero-Neumann) second difference with eigenvalue
-4 sum sin^2(pi k / 2N) / h^2, so n explicit Euler steps multiply a mode by
(1 + beta lambda)^n exactly, at any amplitude (the equation is linear)."""
import math

import numpy as np
import pytest

import oracle


def _mode(shape, ks):
    axes = [np.cos(np.pi * k * (np.arange(n) + 0.5) / n) for n, k in zip(shape, ks)]
    out = axes[0]
    for a in axes[1:]:
        out = np.multiply.outer(out, a)
    return out


@pytest.mark.parametrize("shape,ks", [((12, 20), (3, 5)), ((9, 16), (8, 1)),
                                      ((6, 7, 8), (1, 2, 3)), ((5, 5, 5), (4, 0, 2))])
def test_heat_modes_decay_by_the_discrete_eigenvalue(shape, ks):
    h = 1.0 / max(shape)
    dt = 0.1 * h * h
    n = 50
    phi0 = _mode(shape, ks)
    lam = -4.0 * sum(math.sin(math.pi * k / (2 * N)) ** 2 for N, k in zip(shape, ks))
    out = oracle.step(phi0, h, math.inf, dt, n)
    expect = phi0 * (1.0 + (dt / (h * h)) * lam) ** n
    np.testing.assert_allclose(out, expect, rtol=0, atol=1e-13)


def test_heat_conserves_mass_and_sums_modes():
    rng = np.random.default_rng(4)
    shape = (10, 14)
    h = 1.0 / 14
    dt = 0.1 * h * h
    # a superposition of modes evolves mode by mode
    parts = [(c, ks) for c, ks in zip(rng.uniform(-1, 1, 4), [(0, 0), (1, 3), (4, 2), (9, 13)])]
    phi0 = sum(c * _mode(shape, ks) for c, ks in parts)
    out = oracle.step(phi0, h, math.inf, dt, 30)
    expect = sum(c * (1.0 + 0.1 * -4.0 * sum(math.sin(math.pi * k / (2 * N)) ** 2
                                             for N, k in zip(shape, ks))) ** 30 * _mode(shape, ks)
                 for c, ks in parts)
    np.testing.assert_allclose(out, expect, rtol=0, atol=1e-13)
    # the k = 0 mode (the mean) is untouched: zero-Neumann conserves mass
    assert float(np.mean(out)) == pytest.approx(float(np.mean(phi0)), abs=1e-15)


def test_heat_energy_is_the_dirichlet_energy():
    # with eps = inf the bulk term vanishes: E = h^d / 2 sum_faces (dphi / h)^2
    rng = np.random.default_rng(5)
    phi = rng.uniform(-1, 1, size=(6, 9))
    h = 0.1
    faces = np.sum(np.diff(phi, axis=0) ** 2) + np.sum(np.diff(phi, axis=1) ** 2)
    assert oracle.energy(phi, h, math.inf) == pytest.approx(0.5 * faces, rel=1e-14)
