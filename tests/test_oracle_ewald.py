"""Pins of the oracle's periodic (Ewald-summed) force."""
import math

import numpy as np
import pytest

import oracle


def bodies(N, seed, L=1.0):
    rng = np.random.default_rng(seed)
    return L * rng.random((N, 3)), rng.random(N) / N


@pytest.mark.parametrize("L", [1.0, 2.5])
def test_independent_of_the_splitting_parameter(L):
    x, m = bodies(30, 100, L)
    ref = oracle.ewald_forces(x, m, 0.01, L, G=1.3)
    for aL in (4.0, 9.0):
        got = oracle.ewald_forces(x, m, 0.01, L, G=1.3, alpha=aL / L)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_zero_on_a_perfect_lattice():
    # n = 3: no two bodies are exactly half a box apart, where the nearest
    # image (the softened one) is not unique
    n = 3
    q = (np.arange(n) + 0.5) / n
    x = np.stack(np.meshgrid(q, q, q, indexing="ij"), axis=-1).reshape(-1, 3)
    m = np.full(len(x), 1.0 / len(x))
    F = oracle.ewald_forces(x, m, 0.02, 1.0)
    scale = m[0] * n * n                       # one neighbour's pull
    assert np.abs(F).max() < 1e-12 * scale


def test_zero_between_bodies_half_a_box_apart():
    x = np.array([[0.1, 0.3, 0.7], [0.6, 0.3, 0.7]])
    F = oracle.ewald_forces(x, np.array([0.4, 0.9]), 0.0, 1.0)
    assert np.abs(F).max() < 1e-13


def test_periodic_and_translation_invariant():
    x, m = bodies(25, 101)
    ref = oracle.ewald_forces(x, m, 0.01, 1.0)
    y = x.copy()
    y[3] += np.array([1.0, -1.0, 2.0])
    y[7] -= np.array([0.0, 3.0, 0.0])
    np.testing.assert_allclose(oracle.ewald_forces(y, m, 0.01, 1.0), ref, rtol=0,
                               atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(oracle.ewald_forces(x + np.array([0.31, -0.12, 0.77]), m, 0.01, 1.0),
                               ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_newtons_third_law():
    x, m = bodies(40, 102)
    F = oracle.ewald_forces(x, m, 0.01, 1.0)
    assert np.abs((m[:, None] * F).sum(axis=0)).max() < 1e-14 * np.abs(m[:, None] * F).sum()


@pytest.mark.parametrize("L", [1.0, 3.0])
def test_close_pair_is_plummer_plus_the_background_term(L):
    # near a source the neutralised periodic field is the isolated pull minus
    # the uniform mean density's (4 pi G / 3V) m d, up to O(m |d|^3 / L^5)
    eps, G = 1e-4 * L, 0.7
    d = 0.01 * L * np.array([1.0, 2.0, 2.0]) / 3.0
    x0 = L * np.array([0.3, 0.4, 0.5])
    x = np.stack([x0, x0 + d])
    m = np.array([0.2, 0.5])
    F = oracle.ewald_forces(x, m, eps, L, G=G)
    V = L ** 3
    r2 = float(d @ d) + eps * eps
    plummer = d / r2 ** 1.5
    background = 4.0 * math.pi / (3.0 * V) * d
    np.testing.assert_allclose(F[0] - G * m[1] * plummer, -G * m[1] * background, rtol=1e-3)
    np.testing.assert_allclose(F[1] + G * m[0] * plummer, G * m[0] * background, rtol=1e-3)
