"""Pins of the oracle's derivative models: the force VJP/JVP against central
finite differences of the force, the discrete adjoint and tangent of a whole
trajectory against finite differences of that trajectory, and the
adjoint-tangent duality."""
import numpy as np
import pytest

import oracle
from oracle import Cosmology

LCDM = Cosmology(0.0, 0.3, 0.0, 0.7, 1.0)


def _system(N, seed):
    rng = np.random.default_rng(seed)
    x = rng.random((N, 3))
    v = 0.1 * rng.standard_normal((N, 3))
    m = rng.lognormal(0, 0.5, N) / N
    return x, v, m


def test_vjp_matches_finite_differences():
    N, eps, G = 12, 0.05, 1.3
    x, _, m = _system(N, 21)
    lam = np.random.default_rng(22).standard_normal((N, 3))
    gx, gm = oracle.vjp(x, m, lam, eps, G)

    def L(xx, mm):
        return float(np.sum(lam * oracle.forces(xx, mm, eps, G)))

    h = 1e-6
    for q in range(N):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[q, c] += h
            xm[q, c] -= h
            fd = (L(xp, m) - L(xm, m)) / (2 * h)
            assert gx[q, c] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(gx).max())
        mp, mmn = m.copy(), m.copy()
        mp[q] += h * m[q]
        mmn[q] -= h * m[q]
        fd = (L(x, mp) - L(x, mmn)) / (2 * h * m[q])
        assert gm[q] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(gm).max())


def test_jvp_matches_finite_differences_and_duality():
    N, eps, G = 15, 0.04, 0.9
    x, _, m = _system(N, 23)
    rng = np.random.default_rng(24)
    u, dm = rng.standard_normal((N, 3)), rng.standard_normal(N) * m
    J = oracle.jvp(x, m, u, eps, G, dm=dm)
    h = 1e-6
    fd = (oracle.forces(x + h * u, m + h * dm, eps, G)
          - oracle.forces(x - h * u, m - h * dm, eps, G)) / (2 * h)
    np.testing.assert_allclose(J, fd, rtol=1e-6, atol=1e-7 * np.abs(J).max())
    lam = rng.standard_normal((N, 3))
    gx, gm = oracle.vjp(x, m, lam, eps, G)
    lhs = float(np.sum(lam * J))
    rhs = float(np.sum(gx * u) + np.sum(gm * dm))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def _loss_and_grads(scheme):
    N, eps, G, a0, tau, n = 10, 0.08, 1.0, 0.2, 0.003, 8
    x, v, m = _system(N, 31)
    tr = np.array([1, 4, 7])

    def loss(xx, vv, mm):
        r = oracle.run(xx, vv, mm, eps, G, LCDM, a0, tau, n, scheme)
        aT = r["schedule"]["a"][-1]
        return 0.5 * aT * aT * float(np.sum(mm[tr] * np.sum(r["v"][tr] ** 2, axis=1))), r

    L0, r = loss(x, v, m)
    aT = r["schedule"]["a"][-1]
    gvT = np.zeros((N, 3))
    gvT[tr] = aT * aT * m[tr, None] * r["v"][tr]
    gmT = np.zeros(N)
    gmT[tr] = 0.5 * aT * aT * np.sum(r["v"][tr] ** 2, axis=1)
    g = oracle.adjoint_run(x, v, m, eps, G, LCDM, a0, tau, n, np.zeros((N, 3)), gvT, gmT,
                           scheme=scheme)
    return (x, v, m), loss, g


@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
def test_trajectory_adjoint_matches_finite_differences(scheme):
    (x, v, m), loss, (gx, gv, gm) = _loss_and_grads(scheme)
    h = 1e-6
    for (arr, grad, name) in ((x, gx, "x"), (v, gv, "v")):
        for idx in [(0, 0), (3, 1), (7, 2), (9, 0)]:
            p, q = arr.copy(), arr.copy()
            p[idx] += h
            q[idx] -= h
            args_p = dict(x=x, v=v, m=m)
            args_q = dict(x=x, v=v, m=m)
            args_p[name], args_q[name] = p, q
            fd = (loss(args_p["x"], args_p["v"], args_p["m"])[0]
                  - loss(args_q["x"], args_q["v"], args_q["m"])[0]) / (2 * h)
            assert grad[idx] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(grad).max())
    for k in (1, 5):
        p, q = m.copy(), m.copy()
        hh = h * m[k]
        p[k] += hh
        q[k] -= hh
        fd = (loss(x, v, p)[0] - loss(x, v, q)[0]) / (2 * hh)
        assert gm[k] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(gm).max())


@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
def test_tangent_matches_finite_differences_and_adjoint_duality(scheme):
    N, eps, G, a0, tau, n = 10, 0.08, 1.0, 0.2, 0.003, 8
    x, v, m = _system(N, 41)
    rng = np.random.default_rng(42)
    dx0, dv0 = rng.standard_normal((N, 3)), rng.standard_normal((N, 3))
    dxT, dvT, _ = oracle.tangent_run(x, v, m, eps, G, LCDM, a0, tau, n, dx0, dv0, scheme)
    h = 1e-6
    rp = oracle.run(x + h * dx0, v + h * dv0, m, eps, G, LCDM, a0, tau, n, scheme)
    rm = oracle.run(x - h * dx0, v - h * dv0, m, eps, G, LCDM, a0, tau, n, scheme)
    np.testing.assert_allclose(dxT, (rp["x"] - rm["x"]) / (2 * h), rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(dvT, (rp["v"] - rm["v"]) / (2 * h), rtol=1e-6, atol=1e-8)
    lx, lv = rng.standard_normal((N, 3)), rng.standard_normal((N, 3))
    gx, gv, _ = oracle.adjoint_run(x, v, m, eps, G, LCDM, a0, tau, n, lx, lv, scheme=scheme)
    lhs = float(np.sum(gx * dx0) + np.sum(gv * dv0))
    rhs = float(np.sum(lx * dxT) + np.sum(lv * dvT))
    assert lhs == pytest.approx(rhs, rel=1e-11)


def test_ftle_of_free_particle_is_zero_growth_in_velocity_free_static_case():
    # With G = 0 and H0 = 0 a position perturbation neither grows nor decays.
    static = Cosmology(0.0, 1.0, 0.0, 0.0, 0.0)
    x, v, m = _system(6, 51)
    f = oracle.ftle(x, v, m, 0.05, 0.0, static, 1.0, 0.01, 5, tracer=2)
    np.testing.assert_allclose(f, 0.0, atol=1e-12)
