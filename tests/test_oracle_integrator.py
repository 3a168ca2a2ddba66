"""Pins of the oracle's leapfrog (Eqs. 3-5 and the KDK variant) against
textbook dynamics and exact discrete invariants."""
import math

import numpy as np
import pytest

import oracle
from oracle import Cosmology

STATIC = Cosmology(0.0, 1.0, 0.0, 0.0, 0.0)   # H0 = 0: a stays at a_start
EDS = Cosmology(0.0, 1.0, 0.0, 0.0, 1.0)
LCDM = Cosmology(0.0, 0.3, 0.0, 0.7, 1.0)


def _kepler(scheme, nsteps, G=1.0, sign=1.0):
    """Equal-mass circular binary: omega^2 = G (m1+m2) / (d^2+eps^2)^{3/2}."""
    d, eps, mtot = 1.0, 0.1, 1.0
    w = math.sqrt(G * mtot / (d * d + eps * eps) ** 1.5)
    x = np.array([[-0.5 * d, 0, 0], [0.5 * d, 0, 0]], float)
    v = np.array([[0, -0.5 * w * d, 0], [0, 0.5 * w * d, 0]], float)
    m = np.array([0.5, 0.5])
    T = 2.0 * math.pi / w
    r = oracle.run(x, v, m, eps, sign * G, STATIC, 1.0, T / nsteps, nsteps, scheme)
    return x, r


@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
def test_kepler_circular_orbit_closes(scheme):
    x0, r1 = _kepler(scheme, 1000)
    _, r2 = _kepler(scheme, 2000)
    e1 = np.abs(r1["x"] - x0).max()
    e2 = np.abs(r2["x"] - x0).max()
    assert e1 < 1e-4
    assert 3.6 < e1 / e2 < 4.4          # second order in tau
    sep = np.linalg.norm(r2["x"][1] - r2["x"][0])
    assert abs(sep - 1.0) < 1e-5


def test_printed_sign_of_eq1_is_repulsive():
    # Plant the printed Eq. 1 orientation (x_k - x_j) in the oracle by
    # flipping G: a pair released from rest must approach under gravity; with
    # the printed sign it separates, so the attractive reading is the one kept.
    x = np.array([[0.0, 0, 0], [1.0, 0, 0]])
    v = np.zeros((2, 3))
    m = np.array([0.5, 0.5])
    good = oracle.run(x, v, m, 0.01, 1.0, STATIC, 1.0, 0.01, 50)
    printed = oracle.run(x, v, m, 0.01, -1.0, STATIC, 1.0, 0.01, 50)
    assert np.linalg.norm(good["x"][1] - good["x"][0]) < 1.0
    assert np.linalg.norm(printed["x"][1] - printed["x"][0]) > 1.0


@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
def test_drag_only_velocity_decays_as_a_minus2(scheme):
    # G = 0: dv/dt = -2 H v gives v = v0 (a0/a)^2; EdS closed-form a(t)
    a0, T = 0.1, 0.2
    x = np.zeros((1, 3))
    v0 = np.array([[1.0, -2.0, 0.5]])

    def err(n):
        r = oracle.run(x, v0, np.ones(1), 0.1, 0.0, EDS, a0, T / n, n, scheme)
        aT = (a0 ** 1.5 + 1.5 * T) ** (2.0 / 3.0)
        return np.abs(r["v"] - v0 * (a0 / aT) ** 2).max()

    e1, e2 = err(100), err(200)
    assert e1 < 1e-3
    assert 3.6 < e1 / e2 < 4.4


@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
def test_discrete_momentum_and_angular_momentum_scale_by_c(scheme):
    # sum m F = 0 and sum m x cross F = 0, so every kick multiplies sum m v
    # and sum m x cross v by its drag factor c, and drifts leave them alone.
    rng = np.random.default_rng(11)
    N = 32
    x, v, m = rng.random((N, 3)), 0.1 * rng.standard_normal((N, 3)), rng.random(N)
    n = 12
    r = oracle.run(x, v, m, 0.05, 1.0, LCDM, 0.3, 0.002, n, scheme)
    sch = r["schedule"]
    fac = np.prod(sch["c"]) if scheme == "dkd" else np.prod(sch["c1"] * sch["c2"])
    P0 = np.sum(m[:, None] * v, axis=0)
    P1 = np.sum(m[:, None] * r["v"], axis=0)
    np.testing.assert_allclose(P1, fac * P0, rtol=1e-12, atol=1e-13)
    L0 = np.sum(m[:, None] * np.cross(x, v), axis=0)
    L1 = np.sum(m[:, None] * np.cross(r["x"], r["v"]), axis=0)
    np.testing.assert_allclose(L1, fac * L0, rtol=1e-11, atol=1e-13)


def test_dkd_time_reversible():
    rng = np.random.default_rng(12)
    N = 16
    x, v, m = rng.random((N, 3)), 0.2 * rng.standard_normal((N, 3)), rng.random(N) / N
    f = oracle.run(x, v, m, 0.05, 1.0, STATIC, 1.0, 0.01, 40, "dkd")
    b = oracle.run(f["x"], f["v"], m, 0.05, 1.0, STATIC, 1.0, -0.01, 40, "dkd")
    np.testing.assert_allclose(b["x"], x, atol=1e-12)
    np.testing.assert_allclose(b["v"], v, atol=1e-12)


def test_layzer_irvine_converges_second_order():
    rng = np.random.default_rng(13)
    N = 27
    x = rng.random((N, 3))
    v = 0.05 * rng.standard_normal((N, 3))
    m = np.full(N, 0.2 / N)
    eps, a0, T = 0.1, 0.5, 0.3

    def resid(n):
        r = oracle.run(x, v, m, eps, 1.0, LCDM, a0, T / n, n, "kdk", diag_every=1)
        t = [k * T / n for k, _ in r["diagnostics"]]
        return np.abs(oracle.layzer_irvine([d for _, d in r["diagnostics"]], t)).max()

    r1, r2 = resid(60), resid(120)
    assert r1 < 1e-3
    assert 3.0 < r1 / r2 < 5.0


def test_schedule_matches_eds_closed_form_and_kick_limits():
    sch = oracle.schedule(EDS, 0.02, 1e-4, 50, "kdk", 8)
    exact = (0.02 ** 1.5 + 1.5 * sch["t"]) ** (2.0 / 3.0)
    np.testing.assert_allclose(sch["a"], exact, rtol=1e-12)
    # H -> 0 limit of the kick: c -> 1, d -> h / a^3
    c, d = oracle.kick_coefficients(2.0, 0.0, 0.1)
    assert c == 1.0 and d == pytest.approx(0.1 / 8.0, rel=1e-15)
