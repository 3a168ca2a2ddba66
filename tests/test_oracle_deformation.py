"""Pins of the oracle's Eq. 6 deformation term."""
import numpy as np
import pytest

import oracle
from oracle import Cosmology

LCDM = Cosmology(0.0, 0.3, 0.0, 0.7, 1.0)


def test_equals_a_fixed_point_mass():
    # the paper: the deformation term "acts like a mass particle located in a
    # fixed position" -> with G, a body of mass C psi / G at x_psi
    rng = np.random.default_rng(60)
    N, eps, G = 40, 0.03, 1.7
    x, m = rng.random((N, 3)), rng.random(N) / N
    Cpsi, xpsi = 0.35, np.array([0.4, 0.6, 0.5])
    F = oracle.total_force(x, m, eps, G, (Cpsi, xpsi))
    xa = np.vstack([x, xpsi])
    ma = np.concatenate([m, [Cpsi / G]])
    ref = oracle.forces(xa, ma, eps, G, rows=np.arange(N))
    np.testing.assert_allclose(F, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def test_single_body_closed_form():
    x = np.array([[0.3, 0.0, 0.0]])
    F = oracle.deformation_force(x, 2.0, np.zeros(3), 0.1)
    np.testing.assert_allclose(F[0], [-2.0 * 0.3 / (0.09 + 0.01) ** 1.5, 0.0, 0.0], rtol=1e-15)


def test_deformation_derivatives_match_finite_differences():
    rng = np.random.default_rng(61)
    x = rng.random((7, 3))
    Cpsi, xpsi, eps = 0.8, np.array([0.5, 0.5, 0.5]), 0.05
    u, lam = rng.standard_normal((7, 3)), rng.standard_normal((7, 3))
    h = 1e-6
    fd = (oracle.deformation_force(x + h * u, Cpsi, xpsi, eps)
          - oracle.deformation_force(x - h * u, Cpsi, xpsi, eps)) / (2 * h)
    np.testing.assert_allclose(oracle.deformation_jvp(x, Cpsi, xpsi, eps, u), fd, rtol=1e-7, atol=1e-8)
    g = oracle.deformation_vjp(x, Cpsi, xpsi, eps, lam)
    assert float(np.sum(g * u)) == pytest.approx(float(np.sum(lam * fd)), rel=1e-7)


def test_trajectory_adjoint_with_deformation_matches_finite_differences():
    rng = np.random.default_rng(62)
    N = 8
    x, v, m = rng.random((N, 3)), 0.05 * rng.standard_normal((N, 3)), rng.random(N) / N
    defo = (0.3, np.array([0.5, 0.4, 0.6]))
    a0, tau, n = 0.3, 0.004, 6
    gvT = rng.standard_normal((N, 3))

    def loss(xx):
        r = oracle.run(xx, v, m, 0.05, 1.0, LCDM, a0, tau, n, "kdk", defo=defo)
        return float(np.sum(gvT * r["v"]))

    gx, gv, gm = oracle.adjoint_run(x, v, m, 0.05, 1.0, LCDM, a0, tau, n, np.zeros((N, 3)), gvT,
                                    scheme="kdk", defo=defo)
    d = rng.standard_normal((N, 3))
    h = 1e-6
    fd = (loss(x + h * d) - loss(x - h * d)) / (2 * h)
    assert float(np.sum(gx * d)) == pytest.approx(fd, rel=1e-6)
