"""Pins of the oracle's pair sums (Eq. 1 and its potential) against facts
that do not come from the oracle: point-mass laws, symmetric configurations
with closed-form forces, conservation laws, finite differences of the
potential, scaling laws and a high-precision brute force on tiny inputs."""
import math

import mpmath
import numpy as np
import pytest

import oracle


def test_two_body_points_toward_partner():
    # attractive reading of Eq. 1: body 0 is pulled toward body 1
    x = np.array([[0.1, 0.2, 0.3], [0.6, -0.1, 0.4]])
    m = np.array([0.3, 0.7])
    eps, G = 0.05, 1.7
    F = oracle.forces_pairwise(x, m, eps, G)
    d = x[1] - x[0]
    r2 = d @ d
    expect0 = G * m[1] * d / (r2 + eps * eps) ** 1.5
    np.testing.assert_allclose(F[0], expect0, rtol=1e-14)
    assert F[0] @ d > 0.0 and F[1] @ d < 0.0


def test_ring_closed_form():
    # n equal masses on a circle of radius R: the net pull on each body points
    # to the centre with magnitude G m sum_k c_k sin(pi k/n)/(c_k^2+eps^2)^{3/2},
    # c_k = 2 R sin(pi k / n) the chord to the k-th neighbour.
    n, R, mass, eps = 12, 0.7, 0.05, 0.02
    th = 2.0 * np.pi * np.arange(n) / n
    x = np.stack([R * np.cos(th), R * np.sin(th), np.zeros(n)], axis=1)
    m = np.full(n, mass)
    F = oracle.forces(x, m, eps)
    ks = np.arange(1, n)
    c = 2.0 * R * np.sin(np.pi * ks / n)
    mag = mass * np.sum(c * np.sin(np.pi * ks / n) / (c * c + eps * eps) ** 1.5)
    expect = -mag * x / R
    np.testing.assert_allclose(F, expect, rtol=1e-13, atol=1e-13 * mag)


def test_tetrahedron_closed_form():
    # regular tetrahedron of side L: each vertex is pulled toward the centroid
    # with magnitude G m sqrt(6) L / (L^2 + eps^2)^{3/2}
    L, mass, eps = 0.3, 0.2, 0.01
    v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float)
    v *= L / (2.0 * math.sqrt(2.0))
    m = np.full(4, mass)
    F = oracle.forces(v, m, eps)
    mag = mass * math.sqrt(6.0) * L / (L * L + eps * eps) ** 1.5
    for k in range(4):
        np.testing.assert_allclose(F[k], -mag * v[k] / np.linalg.norm(v[k]), rtol=1e-13)


def test_pairwise_equals_rowwise():
    rng = np.random.default_rng(3)
    x, m = rng.random((200, 3)), rng.random(200)
    a = oracle.forces_pairwise(x, m, 0.01)
    b = oracle.forces(x, m, 0.01)
    scale = np.abs(b).max()
    assert np.max(np.abs(a - b)) < 1e-13 * scale


def test_momentum_and_newton3():
    rng = np.random.default_rng(4)
    x, m = rng.random((64, 3)), rng.lognormal(0.0, 0.5, 64)
    F = oracle.forces_pairwise(x, m, 0.02)
    tot = np.sum(m[:, None] * F, axis=0)
    assert np.all(np.abs(tot) < 1e-14 * np.sum(m[:, None] * np.abs(F), axis=0))
    # pair antisymmetry (Newton's third law): m_0 F_01 = -m_1 F_10
    two = oracle.forces_pairwise(x[:2], m[:2], 0.02)
    np.testing.assert_allclose(m[0] * two[0], -m[1] * two[1], rtol=1e-15, atol=0)


def test_force_is_minus_gradient_of_potential_energy():
    # m_k F_k = -dW_x/dx_k with W_x = (1/2) sum m phi; central FD
    rng = np.random.default_rng(5)
    N, eps = 20, 0.05
    x, m = rng.random((N, 3)), rng.random(N)

    def Wx(xx):
        return 0.5 * float(np.sum(m * oracle.potential(xx, m, eps)))

    F = oracle.forces(x, m, eps)
    h = 1e-6
    for k in (0, 7, 19):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, c] += h
            xm[k, c] -= h
            g = (Wx(xp) - Wx(xm)) / (2 * h)
            assert -g == pytest.approx(m[k] * F[k, c], rel=1e-7, abs=1e-9)


def test_scaling_laws_and_translation():
    rng = np.random.default_rng(6)
    x, m = rng.random((40, 3)), rng.random(40)
    eps = 0.03
    F = oracle.forces(x, m, eps)
    lam, mu = 2.5, 0.3
    sc = np.abs(F).max()
    np.testing.assert_allclose(oracle.forces(lam * x, m, lam * eps), F / lam ** 2,
                               rtol=1e-12, atol=1e-13 * sc / lam ** 2)
    np.testing.assert_allclose(oracle.forces(x, mu * m, eps), mu * F, rtol=1e-12, atol=1e-13 * sc)
    np.testing.assert_allclose(oracle.forces(x + 0.125, m, eps), F, rtol=1e-9, atol=1e-12 * sc)


def test_far_field_point_mass():
    # a compact cluster seen from distance D acts as a point mass at its centre
    rng = np.random.default_rng(7)
    cl = 0.01 * rng.standard_normal((50, 3))
    m = rng.random(50)
    D = 10.0
    x = np.vstack([cl, [[D, 0.0, 0.0]]])
    mm = np.concatenate([m, [1e-3]])
    F = oracle.forces(x, mm, 1e-4, rows=[50])[0]
    com = np.sum(m[:, None] * cl, axis=0) / m.sum()
    d = com - x[50]
    expect = m.sum() * d / np.linalg.norm(d) ** 3
    np.testing.assert_allclose(F, expect, rtol=0, atol=1e-5 * np.linalg.norm(expect))


def test_mpmath_brute_force_tiny():
    rng = np.random.default_rng(8)
    N, eps, G = 9, 0.02, 1.3
    x, m = rng.random((N, 3)), rng.lognormal(0, 0.5, N)
    F = oracle.forces(x, m, eps, G)
    mpmath.mp.dps = 40
    for k in range(N):
        acc = [mpmath.mpf(0)] * 3
        for j in range(N):
            if j == k:
                continue
            d = [mpmath.mpf(x[j, c]) - mpmath.mpf(x[k, c]) for c in range(3)]
            s2 = sum(di * di for di in d) + mpmath.mpf(eps) ** 2
            w = mpmath.mpf(m[j]) / (s2 * mpmath.sqrt(s2))
            acc = [acc[c] + w * d[c] for c in range(3)]
        ref = np.array([float(G * a) for a in acc])
        np.testing.assert_allclose(F[k], ref, rtol=1e-13, atol=1e-15 * np.abs(ref).max())


def test_potential_two_body():
    x = np.array([[0.0, 0.0, 0.0], [0.3, 0.4, 0.0]])
    m = np.array([2.0, 3.0])
    phi = oracle.potential(x, m, 0.1, 1.5)
    s = math.sqrt(0.25 + 0.01)
    np.testing.assert_allclose(phi, [-1.5 * 3.0 / s, -1.5 * 2.0 / s], rtol=1e-15)


def test_self_pair_skipped():
    # a single body feels nothing, whatever eps
    F = oracle.forces(np.array([[0.2, 0.3, 0.4]]), np.array([1.0]), 0.0)
    assert np.all(F == 0.0)
