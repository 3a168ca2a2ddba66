"""Pins of the oracle's diagnostics (momentum, angular momentum, centre of
mass, kinetic and potential energy) and of its finite-time Lyapunov growth.

The diagnostics follow the Hamiltonian section (Sec. II): the canonical
momentum is p = m a^2 v, so P = sum p and L = sum x cross p, and the
potential energy of the literal Eq. 1 dynamics is W_x / a.  Each test below
compares with a closed form of mechanics that the oracle's formulas do not
restate: the inertia tensor of a rigid rotation (L = a^2 I omega,
K = omega . L / 2), Galilean boosts and translations, mirror symmetry, the
two-body Plummer energy and the scale-factor powers.  A dropped a^2, a
swapped cross product, a missing 1/sum(m) or a wrong power of a fails one.

The FTLE is pinned by central differences of two oracle trajectories, and by
the exact discrete solution of a harmonic case: two bodies at the same point
interact through the linear force G m (x_j - x_k) / eps^3, so their relative
coordinate under the KDK leapfrog obeys x_{n+1} + x_{n-1} = 2 cos(theta) x_n
with cos(theta) = 1 - (omega tau)^2 / 2, omega^2 = G M / eps^3.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import Cosmology

STATIC = Cosmology(0.0, 1.0, 0.0, 0.0, 0.0)
LCDM = Cosmology(0.0, 0.3, 0.0, 0.7, 1.0)


def _cloud(N, seed):
    rng = np.random.default_rng(seed)
    x = rng.random((N, 3))
    v = 0.3 * rng.standard_normal((N, 3))
    m = 0.5 + rng.random(N)          # sum m != 1, so a missing 1/sum(m) shows
    return x, v, m


def _inertia_by_hand(r, m):
    """I_ab = sum_k m_k (|r_k|^2 delta_ab - r_ka r_kb), entry by entry."""
    I = np.zeros((3, 3))
    for k in range(len(m)):
        rr = r[k, 0] ** 2 + r[k, 1] ** 2 + r[k, 2] ** 2
        for p in range(3):
            for q in range(3):
                I[p, q] += m[k] * ((rr if p == q else 0.0) - r[k, p] * r[k, q])
    return I


@pytest.mark.parametrize("a", [1.0, 0.37, 2.5])
def test_rigid_rotation_angular_momentum_is_inertia_times_omega(a):
    x, _, m = _cloud(23, 1)
    c = (m[:, None] * x).sum(0) / m.sum()
    r = x - c                               # centre of mass at the origin
    w = np.array([0.3, -1.1, 0.7])
    # v = omega cross r, written out component by component
    v = np.stack([w[1] * r[:, 2] - w[2] * r[:, 1],
                  w[2] * r[:, 0] - w[0] * r[:, 2],
                  w[0] * r[:, 1] - w[1] * r[:, 0]], axis=1)
    d = oracle.diagnostics(r, v, m, a, 0.05, 1.0)
    L_exact = a * a * _inertia_by_hand(r, m) @ w
    np.testing.assert_allclose(d["L"], L_exact, rtol=1e-13, atol=1e-14 * np.abs(L_exact).max())
    # rotation about the centre of mass carries no momentum
    assert np.abs(d["P"]).max() < 1e-13 * a * a * np.abs(v).max() * m.sum()
    np.testing.assert_allclose(d["COM"], 0.0, atol=1e-15)
    # rotational kinetic energy K = (1/2) omega . L
    assert d["K"] == pytest.approx(0.5 * float(w @ d["L"]), rel=1e-13)


def test_boost_adds_total_mass_times_velocity_and_keeps_angular_momentum_about_com():
    x, v, m = _cloud(31, 2)
    a = 0.6
    u = np.array([0.25, -0.4, 1.3])
    d0 = oracle.diagnostics(x, v, m, a, 0.05, 1.0)
    d1 = oracle.diagnostics(x, v + u, m, a, 0.05, 1.0)
    np.testing.assert_allclose(d1["P"] - d0["P"], a * a * m.sum() * u, rtol=1e-13)
    # angular momentum about the centre of mass: L - COM x P
    c = d0["COM"]
    L0c = d0["L"] - np.cross(c, d0["P"])
    L1c = d1["L"] - np.cross(c, d1["P"])
    np.testing.assert_allclose(L1c, L0c, atol=1e-13 * np.abs(d0["L"]).max())
    # the potential energy depends on positions only
    assert d1["W"] == d0["W"]
    # K' = K + u . P + (1/2) a^2 M |u|^2
    dk = float(u @ d0["P"]) + 0.5 * a * a * m.sum() * float(u @ u)
    assert d1["K"] == pytest.approx(d0["K"] + dk, rel=1e-13)


def test_translation_moves_com_and_shifts_angular_momentum():
    x, v, m = _cloud(19, 3)
    a = 1.7
    s = np.array([3.0, -0.25, 0.5])
    d0 = oracle.diagnostics(x, v, m, a, 0.05, 1.0)
    d1 = oracle.diagnostics(x + s, v, m, a, 0.05, 1.0)
    np.testing.assert_allclose(d1["COM"], d0["COM"] + s, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(d1["P"], d0["P"], rtol=1e-14)
    np.testing.assert_allclose(d1["L"], d0["L"] + np.cross(s, d0["P"]),
                               atol=1e-13 * np.abs(d1["L"]).max())
    assert d1["W"] == pytest.approx(d0["W"], rel=1e-13)


def test_mirror_symmetric_configuration():
    # bodies in mirror pairs about the plane z = z0 with mirrored velocities
    rng = np.random.default_rng(4)
    half = rng.random((12, 3))
    z0 = 0.3
    mir = half.copy()
    mir[:, 2] = 2 * z0 - half[:, 2]
    x = np.vstack([half, mir])
    vh = rng.standard_normal((12, 3))
    vm = vh.copy()
    vm[:, 2] = -vh[:, 2]
    v = np.vstack([vh, vm])
    mh = 0.2 + rng.random(12)
    m = np.concatenate([mh, mh])
    d = oracle.diagnostics(x, v, m, 0.8, 0.05, 1.0)
    assert d["COM"][2] == pytest.approx(z0, rel=1e-14)
    assert abs(d["P"][2]) < 1e-14 * np.abs(d["P"]).max()
    # under the mirror L_x and L_y change sign pairwise relative to the plane:
    # about the point (0, 0, z0) they cancel, L_z doubles the half's
    ref = np.array([0.0, 0.0, z0])
    Lp = d["L"] - np.cross(ref, d["P"])
    assert abs(Lp[0]) < 1e-13 * np.abs(Lp).max()
    assert abs(Lp[1]) < 1e-13 * np.abs(Lp).max()


def test_two_body_energies_and_scale_factor_powers():
    # two bodies at rest in their centre-of-mass frame, separation d
    m1, m2, d, eps, G = 0.7, 1.9, 0.8, 0.1, 1.3
    x = np.array([[0.0, 0.0, 0.0], [d, 0.0, 0.0]])
    v = np.array([[0.0, 0.5, 0.0], [0.0, -0.5 * m1 / m2, 0.0]])
    for a in (1.0, 0.25, 3.0):
        dd = oracle.diagnostics(x, v, np.array([m1, m2]), a, eps, G)
        # Plummer pair energy -G m1 m2 / sqrt(d^2 + eps^2), divided by a
        assert dd["W"] == pytest.approx(-G * m1 * m2 / math.hypot(d, eps) / a, rel=1e-14)
        assert dd["Wx"] == pytest.approx(-G * m1 * m2 / math.hypot(d, eps), rel=1e-14)
        # K = (1/2) a^2 (m1 |v1|^2 + m2 |v2|^2)
        k = 0.5 * a * a * (m1 * 0.25 + m2 * (0.5 * m1 / m2) ** 2)
        assert dd["K"] == pytest.approx(k, rel=1e-14)
        # the orbit's angular momentum about body 1: body 2 at (d,0,0) moving in -y
        assert dd["L"][2] == pytest.approx(-a * a * m2 * d * 0.5 * m1 / m2, rel=1e-14)
    d1 = oracle.diagnostics(x, v, np.array([m1, m2]), 1.0, eps, G)
    d2 = oracle.diagnostics(x, v, np.array([m1, m2]), 2.0, eps, G)
    for key in ("K",):
        assert d2[key] == pytest.approx(4.0 * d1[key], rel=1e-14)
    np.testing.assert_allclose(d2["L"], 4.0 * d1["L"], rtol=1e-14)
    assert d2["W"] == pytest.approx(0.5 * d1["W"], rel=1e-14)


def test_diagnostics_hubble_matches_cosmology():
    x, v, m = _cloud(5, 6)
    d = oracle.diagnostics(x, v, m, 0.5, 0.05, 1.0, LCDM)
    # flat LCDM: H = H0 sqrt(0.3 a^-3 + 0.7)
    assert d["H"] == pytest.approx(math.sqrt(0.3 / 0.125 + 0.7), rel=1e-15)


# ------------------------------------------------------------------ FTLE
def test_ftle_matches_central_differences_of_two_trajectories():
    rng = np.random.default_rng(7)
    N = 14
    x = rng.random((N, 3))
    v = 0.1 * rng.standard_normal((N, 3))
    m = np.full(N, 0.05 / N) * (0.5 + rng.random(N))
    eps, a0, tau, n, tr = 0.08, 0.3, 0.004, 12, 5
    direction = np.array([0.2, -0.7, 0.4])
    f = oracle.ftle(x, v, m, eps, 1.0, LCDM, a0, tau, n, tracer=tr, direction=direction)
    e = direction / np.linalg.norm(direction)
    h = 1e-7
    xp, xm = x.copy(), x.copy()
    xp[tr] += h * e
    xm[tr] -= h * e
    fd = np.empty(n)
    for k in range(1, n + 1):
        rp = oracle.run(xp, v, m, eps, 1.0, LCDM, a0, tau, k, "kdk")
        rm = oracle.run(xm, v, m, eps, 1.0, LCDM, a0, tau, k, "kdk")
        ddx = (rp["x"][tr] - rm["x"][tr]) / (2 * h)
        ddv = (rp["v"][tr] - rm["v"][tr]) / (2 * h)
        fd[k - 1] = math.log(math.sqrt(float(ddx @ ddx + ddv @ ddv))) / (k * tau)
    # FD truncation O(h^2) and rounding 1e-16/h on ln(g) ~ 1e-9, over t >= tau
    np.testing.assert_allclose(f, fd, atol=1e-9 / tau)
    assert np.abs(f).max() > 1e-2          # the growth is not trivially zero


@pytest.mark.parametrize("m1,m2", [(0.5, 0.5), (0.2, 1.4)])
def test_ftle_of_coincident_pair_is_the_discrete_harmonic_closed_form(m1, m2):
    eps, G, tau, n = 0.1, 1.0, 0.002, 300
    M = m1 + m2
    w2 = G * M / eps ** 3                   # omega^2 of the relative coordinate
    theta = math.acos(1.0 - 0.5 * w2 * tau * tau)
    x = np.array([[0.4, 0.5, 0.6], [0.4, 0.5, 0.6]])
    v = np.zeros((2, 3))
    f = oracle.ftle(x, v, np.array([m1, m2]), eps, G, STATIC, 1.0, tau, n, tracer=0,
                    direction=(0.0, 1.0, 0.0))
    k = np.arange(1, n + 1)
    # tracer 0 = centre of mass (unmoved, m1/M) minus (m2/M) x relative coordinate
    dx = m1 / M + (m2 / M) * np.cos(k * theta)
    dv = -(m2 / M) * (math.sin(theta) / tau) * np.sin(k * theta)
    exact = np.log(np.sqrt(dx * dx + dv * dv)) / (k * tau)
    np.testing.assert_allclose(f, exact, rtol=1e-9, atol=1e-9)
    # velocity part of the norm matters (a position-only norm differs)
    pos_only = np.log(np.abs(dx)) / (k * tau)
    assert np.abs(f - pos_only).max() > 1.0
