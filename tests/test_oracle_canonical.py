"""Pins of the oracle's canonical (symplectic) kick-drift-kick: the
reformulation of Sec. II with p = a^2 v (per unit mass), drift
x += p int dt/a^2 and kick p += G F int dt/a."""
import math

import numpy as np
import pytest

import oracle
from oracle import Cosmology

EDS = Cosmology(0.0, 1.0, 0.0, 0.0, 1.3)
DESITTER = Cosmology(0.0, 0.0, 0.0, 1.0, 0.7)
STATIC = Cosmology(0.0, 0.3, 0.0, 0.7, 0.0)
LCDM = Cosmology(0.0, 0.3, 0.0, 0.7, 1.0)


def eds_a(a0, t, H0):
    return (a0 ** 1.5 + 1.5 * H0 * t) ** (2.0 / 3.0)


@pytest.mark.parametrize("a0,dt", [(0.02, 1e-4), (0.3, 5e-3), (1.0, 0.05)])  # H dt <= 0.07
def test_integrals_eds_closed_form(a0, dt):
    a1, K, D = oracle.friedmann_integrals(a0, dt, EDS, 8)
    H0 = EDS.H0
    assert a1 == pytest.approx(eds_a(a0, dt, H0), rel=1e-10)
    assert K == pytest.approx(2.0 / H0 * (math.sqrt(a1) - math.sqrt(a0)), rel=1e-9)
    assert D == pytest.approx(2.0 / H0 * (1.0 / math.sqrt(a0) - 1.0 / math.sqrt(a1)), rel=1e-9)


def test_integrals_de_sitter_and_static_closed_forms():
    a0, dt, H0 = 0.2, 0.1, DESITTER.H0
    a1, K, D = oracle.friedmann_integrals(a0, dt, DESITTER, 8)
    assert a1 == pytest.approx(a0 * math.exp(H0 * dt), rel=1e-10)
    # RK4 truncation with H dt / 8 ~ 0.009 per sub-step: ~3e-10
    assert K == pytest.approx((1.0 / a0 - 1.0 / a1) / H0, rel=1e-9)
    assert D == pytest.approx((1.0 / a0 ** 2 - 1.0 / a1 ** 2) / (2.0 * H0), rel=1e-9)
    a1, K, D = oracle.friedmann_integrals(0.5, 0.3, STATIC, 8)
    assert (a1, K, D) == (0.5, pytest.approx(0.3 / 0.5, rel=1e-15), pytest.approx(0.3 / 0.25, rel=1e-15))


def test_integrals_converge_at_fourth_order_and_keep_a_bitwise():
    a0, dt = 0.02, 4e-4
    exact_K = 2.0 / EDS.H0 * (math.sqrt(eds_a(a0, dt, EDS.H0)) - math.sqrt(a0))
    err = [abs(oracle.friedmann_integrals(a0, dt, EDS, n)[1] - exact_K) for n in (1, 2, 4)]
    assert 12.0 < err[0] / err[1] < 20.0 and 12.0 < err[1] / err[2] < 20.0
    for a in (0.02, 0.3):
        assert oracle.friedmann_integrals(a, 0.01, LCDM, 8)[0] == oracle.friedmann_advance(a, 0.01, LCDM, 8)


def system(N=5, seed=90):
    # light bodies: the steps below resolve their orbits at these a and tau
    rng = np.random.default_rng(seed)
    return rng.random((N, 3)), 0.3 * rng.standard_normal((N, 3)), 1e-3 * rng.random(N) / N


def test_static_universe_reduces_to_the_drag_kdk():
    x, v, m = system()
    r_c = oracle.run(x, v, m, 0.05, 1.0, STATIC, 0.7, 0.01, 20, "canonical")
    r_k = oracle.run(x, v, m, 0.05, 1.0, STATIC, 0.7, 0.01, 20, "kdk")
    np.testing.assert_allclose(r_c["x"], r_k["x"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(r_c["v"], r_k["v"], rtol=1e-12, atol=1e-13)


def test_drag_only_canonical_momentum_is_exact():
    # G = 0: p = a^2 v is constant and x = x0 + p int dt/a^2, exactly (EdS closed form)
    x, v, m = system()
    a0, tau, n = 0.02, 2e-3, 50
    rc = oracle.run(x, v, m, 0.05, 0.0, EDS, a0, tau, n, "canonical")
    aT = rc["schedule"]["a"][-1]
    np.testing.assert_allclose(aT ** 2 * rc["v"], a0 ** 2 * v, rtol=1e-12)
    D_exact = 2.0 / EDS.H0 * (1.0 / math.sqrt(a0) - 1.0 / math.sqrt(eds_a(a0, n * tau, EDS.H0)))
    np.testing.assert_allclose(rc["x"], x + a0 ** 2 * v * D_exact, rtol=0, atol=1e-9)
    # the trapezoidal drag of the plain KDK is only second order here
    rk = oracle.run(x, v, m, 0.05, 0.0, EDS, a0, tau, n, "kdk")
    assert np.abs(aT ** 2 * rk["v"] - a0 ** 2 * v).max() > 1e-4 * np.abs(a0 ** 2 * v).max()


def one_step_map(scheme, h, a0=0.05, tau=0.01):
    """Central-difference Jacobian of one step as a map of (x, P), P = m a^2 v:
    returns (max abs(M^T J M - J), det M)."""
    x0, v0, m = system(3, 91)
    m = 300.0 * m
    sch = oracle.schedule(LCDM, a0, tau, 1, scheme)
    a1 = sch["a"][-1]

    def phi(z):
        x = z[:9].reshape(3, 3)
        v = z[9:].reshape(3, 3) / (m[:, None] * a0 ** 2)
        r = oracle.run(x, v, m, 0.1, 1.0, LCDM, a0, tau, 1, scheme)
        return np.concatenate([r["x"].ravel(), (m[:, None] * a1 ** 2 * r["v"]).ravel()])

    z0 = np.concatenate([x0.ravel(), (m[:, None] * a0 ** 2 * v0).ravel()])
    M = np.empty((18, 18))
    for k in range(18):
        e = np.zeros(18)
        e[k] = h
        M[:, k] = (phi(z0 + e) - phi(z0 - e)) / (2 * h)
    J = np.block([[np.zeros((9, 9)), np.eye(9)], [-np.eye(9), np.zeros((9, 9))]])
    return np.abs(M.T @ J @ M - J).max(), np.linalg.det(M)


def test_canonical_step_is_symplectic_and_the_drag_kdk_is_not():
    # the canonical defect is the difference quotient's own h^2 error
    d5, det5 = one_step_map("canonical", 1e-5)
    d6, det6 = one_step_map("canonical", 1e-6)
    assert d6 < 1e-5 and 50.0 < d5 / d6 < 150.0 and abs(det6 - 1.0) < 1e-8
    k5, kdet5 = one_step_map("kdk", 1e-5)
    k6, _ = one_step_map("kdk", 1e-6)
    assert k6 > 1e-2 and abs(k5 / k6 - 1.0) < 1e-3 and abs(kdet5 - 1.0) > 0.1


def test_second_order_convergence_to_the_drag_kdk_limit():
    x, v, m = system(4, 92)
    a0, T = 0.1, 0.08

    def xT(scheme, n):
        return oracle.run(x, v, m, 0.1, 1.0, LCDM, a0, T / n, n, scheme)["x"]

    xs = [xT("canonical", n) for n in (16, 32, 64, 128)]
    d = [np.abs(xs[k] - xs[k + 1]).max() for k in range(3)]
    assert 3.5 < d[0] / d[1] < 4.5 and 3.5 < d[1] / d[2] < 4.5
    # both schemes discretise the same equations: their gap shrinks as tau^2
    g16 = np.abs(xT("canonical", 16) - xT("kdk", 16)).max()
    g128 = np.abs(xs[3] - xT("kdk", 128)).max()
    assert 40.0 < g16 / g128 < 90.0
