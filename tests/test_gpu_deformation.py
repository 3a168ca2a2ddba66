"""GPU parity of the Eq. 6 deformation term against the FP64 oracle: in the
force, through the KDK and DKD steps, in the force VJP and the trajectory
adjoint, and in the tangent-linear model.

The term is the pull of a fixed point "mass" C psi / G at x_psi, so besides the
oracle comparisons the force must equal the GPU's own all-pairs force with that
extra body appended.

The trajectory cases start at a = 0.5.  Eq. 6 softens the term with the
bodies' own eps, so at a = 1/51 (a^-3 ~ 1.3e5) a point mass of a few percent of
the box's mass throws its neighbours across the box within a step, and the
FP64 oracle itself then amplifies a 6e-8 change of the initial positions to
O(0.1).  At a = 0.5 the same perturbation stays below 3e-7 over 10-20 steps
while the term still changes the velocities by O(1).
"""
import numpy as np
import pytest

import oracle
from paper_1208_3444_b300 import binding as B
from paper_1208_3444_b300 import inputs

pytestmark = pytest.mark.gpu

LCDM_D = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
LCDM = oracle.Cosmology(0.0, 0.3, 0.0, 0.7, 1.0)
TAU = inputs.lcdm_tau(2000)
A_LATE = 0.5
XPSI = np.array([0.5, 0.5, 0.5])      # trajectories: between grid nodes (nearest body >= 0.05 away)
XPSI_F = np.array([0.51, 0.47, 0.53])  # single evaluations: not float-representable
FORCE_TOL = {B.FP32: 1e-5, B.FP32_COMP: 1e-6, B.FP64: 1e-11}
PRECS = [B.FP32, B.FP32_COMP, B.FP64]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_rms(a, b):
    return float(np.sqrt(np.mean(np.sum((a - b) ** 2, axis=1))) /
                 np.mean(np.linalg.norm(b, axis=1)))


def random_system(N, seed):
    rng = np.random.default_rng(seed)
    x = inputs.f32(rng.random((N, 3)))
    m = inputs.f32(rng.lognormal(0.0, 0.5, N) / N)
    return x, m


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [1, 257, 3000])
def test_force_with_deformation_matches_oracle(N, prec):
    x, m = random_system(N, 700 + N)
    a, G, eps, Cpsi = 0.5, 1.3, 0.01, 0.4
    sim = B.Simulation(m, eps, LCDM_D, a, prec=prec, G=G)
    try:
        sim.set_state(x)
        sim.set_deformation(Cpsi, XPSI_F)
        got = sim.forces()
    finally:
        sim.close()
    ref = oracle.total_force(x, m, eps, G, (Cpsi, XPSI_F)) / a ** 3
    assert rel_rms(got, ref) < FORCE_TOL[prec]


@pytest.mark.parametrize("prec", [B.FP32_COMP, B.FP64])
def test_deformation_equals_an_appended_fixed_body(prec):
    x, m = random_system(2000, 710)
    G, eps, Cpsi = 0.8, 0.02, 0.25
    sim = B.Simulation(m, eps, LCDM_D, 1.0, prec=prec, G=G)
    try:
        sim.set_state(x)
        sim.set_deformation(Cpsi, inputs.f32(XPSI_F))
        got = sim.forces()
    finally:
        sim.close()
    xa = np.vstack([x, inputs.f32(XPSI_F)[None, :]])
    ma = np.concatenate([m, [Cpsi / G]])
    sim = B.Simulation(ma, eps, LCDM_D, 1.0, prec=prec, G=G)
    try:
        sim.set_state(xa)
        ref = sim.forces()[:-1]
    finally:
        sim.close()
    assert rel_rms(got, ref) < (1e-6 if prec == B.FP32_COMP else 1e-12)


def test_zero_strength_is_off_and_zero_G_is_rejected():
    x, m = random_system(600, 720)
    sim = B.Simulation(m, 0.01, LCDM_D, 1.0, prec=B.FP32)
    try:
        sim.set_state(x)
        base = sim.forces()
        sim.set_deformation(0.3, XPSI)
        on = sim.forces()
        sim.set_deformation(0.0)
        off = sim.forces()
    finally:
        sim.close()
    assert np.array_equal(base, off) and not np.array_equal(base, on)
    sim = B.Simulation(m, 0.01, LCDM_D, 1.0, prec=B.FP32, G=0.0)
    try:
        with pytest.raises(B.ColatusError):
            sim.set_deformation(0.3, XPSI)
        with pytest.raises(B.ColatusError):
            sim.set_deformation(float("nan"), XPSI)
    finally:
        sim.close()


@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
@pytest.mark.parametrize("prec", PRECS)
def test_ten_steps_with_deformation(prec, scheme):
    # 16^3 at the background density, a point mass of 30% of the box's mass
    ic = inputs.grid16(critical=True)
    Cpsi = 0.3 * float(np.sum(ic.m))
    n = 10
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, A_LATE, prec=prec,
                       scheme={"kdk": B.KDK, "dkd": B.DKD}[scheme])
    try:
        sim.set_state(ic.x, ic.v)
        sim.set_deformation(Cpsi, XPSI)
        sim.step(TAU, 4)
        sim.step(TAU, n - 4)
        x, v, t, a = sim.state()
    finally:
        sim.close()
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, A_LATE, TAU, n, scheme, defo=(Cpsi, XPSI))
    r0 = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, A_LATE, TAU, n, scheme)
    # the term moves the bodies by much more than the tolerance
    assert np.abs(r["v"] - r0["v"]).max() > 100 * (1e-5 if prec != B.FP64 else 1e-11) * np.abs(r["v"]).max()
    assert np.abs(x - r["x"]).max() < (1e-5 if prec != B.FP64 else 1e-9)
    dv = np.linalg.norm(v - r["v"], axis=1)
    vn = np.linalg.norm(r["v"], axis=1)
    tol = 1e-11 if prec == B.FP64 else 1e-5
    assert np.sqrt(np.mean(dv ** 2)) < tol * np.sqrt(np.mean(vn ** 2))


@pytest.mark.parametrize("prec,tol", [(B.FP32, 1e-5), (B.FP64, 1e-10)])
def test_force_vjp_with_deformation(prec, tol):
    rng = np.random.default_rng(730)
    x, m = random_system(1500, 731)
    w = inputs.f32(rng.standard_normal((1500, 3)))
    a, G, eps, Cpsi = 0.5, 1.3, 0.01, 0.4
    sim = B.Simulation(m, eps, LCDM_D, a, prec=prec, G=G)
    try:
        sim.set_state(x)
        sim.set_deformation(Cpsi, XPSI_F)
        gx, gm = sim.force_vjp(w)
    finally:
        sim.close()
    rx, rm = oracle.vjp(x, m, w, eps, G)
    rx = rx + oracle.deformation_vjp(x, Cpsi, XPSI_F, eps, w)
    assert rel(gx, rx / a ** 3) < tol
    assert rel(gm, rm / a ** 3) < tol


@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
@pytest.mark.parametrize("prec,tol", [(B.FP64, 1e-9), (B.FP32_COMP, 1e-4)])
def test_trajectory_adjoint_with_deformation(prec, tol, scheme):
    # DKD: the term's Jacobian at the half-drift positions
    ic = inputs.perturbed_grid(8, 0.1, 0.02, 4, zeldovich=True, total_mass=inputs.CRITICAL_MATTER_DENSITY)
    defo = (0.3 * inputs.CRITICAL_MATTER_DENSITY, XPSI)
    n = 20
    rng = np.random.default_rng(740)
    gxT = rng.standard_normal(ic.x.shape)
    gvT = rng.standard_normal(ic.v.shape)
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, A_LATE, prec=prec,
                       scheme=B.KDK if scheme == "kdk" else B.DKD)
    try:
        sim.set_state(ic.x, ic.v)
        sim.set_deformation(*defo)
        sim.adjoint_forward(TAU, n, 6)
        gx, gv, gm = sim.adjoint_backward(gxT, gvT)
    finally:
        sim.close()
    rx, rv, rm = oracle.adjoint_run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, A_LATE, TAU, n,
                                    gxT, gvT, scheme=scheme, defo=defo)
    for got, ref, k in ((gx, rx, "gx"), (gv, rv, "gv"), (gm, rm, "gm")):
        assert rel(got, ref) < tol, k


@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
def test_tangent_growth_with_deformation(scheme):
    ic = inputs.grid16(critical=True)
    defo = (0.3 * float(np.sum(ic.m)), XPSI)
    seeds = [7, 2049, 4000]
    n = 8
    d = np.array([0.5, -1.0, 2.0])
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, A_LATE, prec=B.FP32,
                       scheme=B.KDK if scheme == "kdk" else B.DKD)
    try:
        sim.set_state(ic.x, ic.v)
        sim.set_deformation(*defo)
        sim.tangent_init(seeds, n, d)
        sim.tangent_step(TAU, n)
        growth = sim.tangent_growth()
    finally:
        sim.close()
    for b, s in enumerate(seeds):
        dx0 = np.zeros_like(ic.x)
        dx0[s] = d / np.linalg.norm(d)
        _, _, hist = oracle.tangent_run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, A_LATE, TAU, n,
                                        dx0, np.zeros_like(ic.v), scheme, defo=defo)
        ref = np.array([np.sqrt(np.sum(h[0][s] ** 2) + np.sum(h[1][s] ** 2)) for h in hist[1:]])
        np.testing.assert_allclose(growth[:, b], ref, rtol=1e-4)
