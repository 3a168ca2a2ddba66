"""Pins of the oracle's derivatives of the periodic (Ewald-summed) force:
ewald_jvp against central differences of ewald_forces, ewald_vjp against
ewald_jvp by duality and against differences of lam . F, both independent of
the splitting parameter, translation invariance, the close-pair limit, and
the periodic trajectory adjoint and tangent against finite differences."""
import math

import numpy as np
import pytest

import oracle
from oracle import Cosmology

LCDM = Cosmology(0.0, 0.3, 0.0, 0.7, 1.0)


def bodies(N, seed, L=1.0):
    rng = np.random.default_rng(seed)
    return L * rng.random((N, 3)), 0.3 + rng.random(N)


@pytest.mark.parametrize("L", [1.0, 2.0])
def test_jvp_matches_central_differences_in_x_and_m(L):
    x, m = bodies(14, 200, L)
    rng = np.random.default_rng(201)
    dx, dm = rng.standard_normal(x.shape), rng.standard_normal(len(m))
    eps, G, h = 0.03 * L, 1.2, 1e-6 * L
    got = oracle.ewald_jvp(x, m, dx, eps, L, G)
    fd = (oracle.ewald_forces(x + h * dx, m, eps, L, G) -
          oracle.ewald_forces(x - h * dx, m, eps, L, G)) / (2 * h)
    np.testing.assert_allclose(got, fd, rtol=0, atol=1e-7 * np.abs(fd).max())
    gotm = oracle.ewald_jvp(x, m, np.zeros_like(x), eps, L, G, dm=dm)
    fdm = (oracle.ewald_forces(x, m + 1e-6 * dm, eps, L, G) -
           oracle.ewald_forces(x, m - 1e-6 * dm, eps, L, G)) / 2e-6
    np.testing.assert_allclose(gotm, fdm, rtol=0, atol=1e-8 * np.abs(fdm).max())


def test_vjp_is_the_transpose_of_the_jvp_and_matches_differences_in_m():
    x, m = bodies(17, 202)
    rng = np.random.default_rng(203)
    lam, dx, dm = rng.standard_normal(x.shape), rng.standard_normal(x.shape), rng.standard_normal(17)
    eps, G = 0.02, 0.9
    gx, gm = oracle.ewald_vjp(x, m, lam, eps, 1.0, G)
    jx = oracle.ewald_jvp(x, m, dx, eps, 1.0, G)
    jm = oracle.ewald_jvp(x, m, np.zeros_like(x), eps, 1.0, G, dm=dm)
    assert float(np.sum(gx * dx)) == pytest.approx(float(np.sum(lam * jx)), rel=1e-11)
    assert float(np.sum(gm * dm)) == pytest.approx(float(np.sum(lam * jm)), rel=1e-11)
    # dL/dm_k directly by central differences of lam . F
    for k in (0, 5, 16):
        p, q = m.copy(), m.copy()
        p[k] += 1e-6
        q[k] -= 1e-6
        fd = (np.sum(lam * oracle.ewald_forces(x, p, eps, 1.0, G)) -
              np.sum(lam * oracle.ewald_forces(x, q, eps, 1.0, G))) / 2e-6
        assert gm[k] == pytest.approx(fd, rel=1e-7, abs=1e-9 * np.abs(gm).max())


@pytest.mark.parametrize("aL", [4.0, 9.0])
def test_derivatives_do_not_depend_on_the_splitting_parameter(aL):
    x, m = bodies(20, 204)
    rng = np.random.default_rng(205)
    lam, dx = rng.standard_normal(x.shape), rng.standard_normal(x.shape)
    ref_j = oracle.ewald_jvp(x, m, dx, 0.02, 1.0)
    ref_x, ref_m = oracle.ewald_vjp(x, m, lam, 0.02, 1.0)
    np.testing.assert_allclose(oracle.ewald_jvp(x, m, dx, 0.02, 1.0, alpha=aL), ref_j, rtol=0,
                               atol=1e-11 * np.abs(ref_j).max())
    gx, gm = oracle.ewald_vjp(x, m, lam, 0.02, 1.0, alpha=aL)
    np.testing.assert_allclose(gx, ref_x, rtol=0, atol=1e-11 * np.abs(ref_x).max())
    np.testing.assert_allclose(gm, ref_m, rtol=0, atol=1e-11 * np.abs(ref_m).max())


def test_translation_invariance():
    x, m = bodies(16, 206)
    rng = np.random.default_rng(207)
    lam = rng.standard_normal(x.shape)
    gx, _ = oracle.ewald_vjp(x, m, lam, 0.02, 1.0)
    assert np.abs(gx.sum(axis=0)).max() < 1e-12 * np.abs(gx).sum()
    # moving every body by the same vector changes no force
    shift = np.tile(np.array([0.3, -1.1, 0.6]), (16, 1))
    dF = oracle.ewald_jvp(x, m, shift, 0.02, 1.0)
    ref = oracle.ewald_jvp(x, m, rng.standard_normal(x.shape), 0.02, 1.0)
    assert np.abs(dF).max() < 1e-12 * np.abs(ref).max()


def test_close_pair_jacobian_is_plummer_minus_the_background_term():
    # separations << L: Phi(d) = P(d) - (4 pi/3V) d + O(|d|^3/L^5), so the
    # Jacobian is the isolated one minus (4 pi/3V) m I
    L, eps, G = 1.0, 1e-4, 0.8
    d = 0.01 * np.array([1.0, 2.0, 2.0]) / 3.0
    x0 = np.array([0.3, 0.4, 0.5])
    x = np.stack([x0, x0 + d])
    m = np.array([0.2, 0.5])
    rng = np.random.default_rng(208)
    dx = rng.standard_normal((2, 3))
    got = oracle.ewald_jvp(x, m, dx, eps, L, G)
    iso = oracle.jvp(x, m, dx, eps, G)
    bg = -G * 4.0 * math.pi / 3.0 * np.stack([m[1] * (dx[1] - dx[0]), m[0] * (dx[0] - dx[1])])
    np.testing.assert_allclose(got, iso + bg, rtol=0, atol=1e-3 * np.abs(bg).max())
    assert np.abs(got - iso).max() > 0.5 * np.abs(bg).max()


def _traj_system(seed):
    rng = np.random.default_rng(seed)
    N = 10
    x = rng.random((N, 3))
    v = 0.2 * rng.standard_normal((N, 3))
    m = (0.5 + rng.random(N)) * 0.02 / N
    return x, v, m


def test_periodic_trajectory_adjoint_matches_finite_differences():
    x, v, m = _traj_system(210)
    eps, G, a0, tau, n = 0.05, 1.0, 0.4, 0.01, 6
    rng = np.random.default_rng(211)
    cx, cv = rng.standard_normal(x.shape), rng.standard_normal(x.shape)

    def loss(xx, vv, mm):
        r = oracle.run(xx, vv, mm, eps, G, LCDM, a0, tau, n, "kdk", box=1.0)
        return float(np.sum(cx * r["x"]) + np.sum(cv * r["v"]))

    gx, gv, gm = oracle.adjoint_run(x, v, m, eps, G, LCDM, a0, tau, n, cx, cv, box=1.0)
    h = 1e-6
    for k, c in ((0, 0), (4, 1), (9, 2)):
        p, q = x.copy(), x.copy()
        p[k, c] += h
        q[k, c] -= h
        assert gx[k, c] == pytest.approx((loss(p, v, m) - loss(q, v, m)) / (2 * h), rel=1e-6,
                                         abs=1e-8 * np.abs(gx).max())
        p, q = v.copy(), v.copy()
        p[k, c] += h
        q[k, c] -= h
        assert gv[k, c] == pytest.approx((loss(x, p, m) - loss(x, q, m)) / (2 * h), rel=1e-6,
                                         abs=1e-8 * np.abs(gv).max())
    for k in (2, 7):
        p, q = m.copy(), m.copy()
        hh = 1e-6 * m[k]
        p[k] += hh
        q[k] -= hh
        assert gm[k] == pytest.approx((loss(x, v, p) - loss(x, v, q)) / (2 * hh), rel=1e-6,
                                      abs=1e-8 * np.abs(gm).max())


def test_periodic_tangent_matches_finite_differences_and_the_adjoint():
    x, v, m = _traj_system(212)
    eps, G, a0, tau, n = 0.05, 1.0, 0.4, 0.01, 6
    rng = np.random.default_rng(213)
    dx0, dv0 = rng.standard_normal(x.shape), rng.standard_normal(x.shape)
    dxT, dvT, _ = oracle.tangent_run(x, v, m, eps, G, LCDM, a0, tau, n, dx0, dv0, box=1.0)
    h = 1e-6
    rp = oracle.run(x + h * dx0, v + h * dv0, m, eps, G, LCDM, a0, tau, n, "kdk", box=1.0)
    rm = oracle.run(x - h * dx0, v - h * dv0, m, eps, G, LCDM, a0, tau, n, "kdk", box=1.0)
    np.testing.assert_allclose(dxT, (rp["x"] - rm["x"]) / (2 * h), rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(dvT, (rp["v"] - rm["v"]) / (2 * h), rtol=1e-6, atol=1e-8)
    lx, lv = rng.standard_normal(x.shape), rng.standard_normal(x.shape)
    gx, gv, _ = oracle.adjoint_run(x, v, m, eps, G, LCDM, a0, tau, n, lx, lv, box=1.0)
    assert float(np.sum(gx * dx0) + np.sum(gv * dv0)) == pytest.approx(
        float(np.sum(lx * dxT) + np.sum(lv * dvT)), rel=1e-11)
