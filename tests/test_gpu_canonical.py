"""GPU parity of the canonical (symplectic) kick-drift-kick of Sec. II
(p = a^2 v; kick p += G F int dt/a, drift x += p int dt/a^2) against the
oracle: trajectories, the exact drag-only solution, the adjoint and the
tangent model, and a switch of scheme in the middle of a run."""
import math

import numpy as np
import pytest

import oracle
from paper_1208_3444_b300 import binding as B
from paper_1208_3444_b300 import inputs

pytestmark = pytest.mark.gpu

LCDM_D = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
LCDM = oracle.Cosmology(0.0, 0.3, 0.0, 0.7, 1.0)
TAU = inputs.lcdm_tau(2000)
POS_TOL = {B.FP32: 1e-5, B.FP32_COMP: 1e-5, B.FP64: 1e-9}
VEL_RMS_TOL = {B.FP32: 1e-5, B.FP32_COMP: 1e-5, B.FP64: 1e-11}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_gpu(ic, prec, scheme, chunks, a_start=inputs.A_START, G=1.0, cosmo=LCDM_D):
    sim = B.Simulation(ic.m, ic.eps, cosmo, a_start, prec=prec, scheme=scheme, G=G)
    try:
        sim.set_state(ic.x, ic.v)
        for n in chunks:
            sim.step(TAU, n)
        return sim.state()
    finally:
        sim.close()


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP, B.FP64])
def test_ten_canonical_steps_critical_density(prec):
    ic = inputs.grid16(critical=True)
    x, v, t, a = run_gpu(ic, prec, B.KDK_CANONICAL, [3, 7])
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, 10, "canonical")
    rk = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, 10, "kdk")
    # the two schemes differ by far more than the tolerance here
    assert np.abs(r["v"] - rk["v"]).max() > 100 * VEL_RMS_TOL[prec] * np.abs(r["v"]).max()
    assert np.abs(x - r["x"]).max() < POS_TOL[prec]
    dv = np.linalg.norm(v - r["v"], axis=1)
    assert np.sqrt(np.mean(dv ** 2)) < VEL_RMS_TOL[prec] * np.sqrt(np.mean(np.sum(r["v"] ** 2, axis=1)))
    assert a == pytest.approx(r["schedule"]["a"][-1], rel=1e-13)


def test_drag_only_momentum_is_exact_on_the_gpu():
    # G = 0 in an Einstein-de Sitter universe: a^2 v is conserved and the drift
    # is p int dt/a^2 with the closed-form integral
    ic = inputs.grid8()
    eds = dict(Omega_R=0.0, Omega_M=1.0, Omega_K=0.0, Omega_L=0.0, H0=1.0)
    a0, n = 0.05, 40
    sim = B.Simulation(ic.m, ic.eps, eds, a0, prec=B.FP64, scheme=B.KDK_CANONICAL, G=0.0)
    try:
        sim.set_state(ic.x, ic.v + 0.1)
        sim.step(TAU, n)
        x, v, t, a = sim.state()
    finally:
        sim.close()
    v0 = ic.v + 0.1
    np.testing.assert_allclose(a * a * v, a0 * a0 * v0, rtol=1e-12, atol=1e-15)
    aT = (a0 ** 1.5 + 1.5 * n * TAU) ** (2.0 / 3.0)
    assert a == pytest.approx(aT, rel=1e-12)
    D = 2.0 * (1.0 / math.sqrt(a0) - 1.0 / math.sqrt(aT))
    np.testing.assert_allclose(x, ic.x + a0 * a0 * v0 * D, rtol=0, atol=1e-10)


def test_switching_scheme_mid_run():
    ic = inputs.grid16(critical=True)
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP64, scheme=B.KDK)
    try:
        sim.set_state(ic.x, ic.v)
        sim.step(TAU, 4)
        sim.configure(scheme=B.KDK_CANONICAL)
        sim.step(TAU, 5)
        x, v, t, a = sim.state()
    finally:
        sim.close()
    r1 = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, 4, "kdk")
    a4 = r1["schedule"]["a"][-1]
    r2 = oracle.run(r1["x"], r1["v"], ic.m, ic.eps, 1.0, LCDM, a4, TAU, 5, "canonical")
    assert np.abs(x - r2["x"]).max() < 1e-9
    assert rel(v, r2["v"]) < 1e-10


def adjoint_case(prec, loss):
    """Gradients of a final-state loss after 20 canonical steps (checkpoints
    every 7), from the GPU and from the oracle's exact transpose."""
    ic = inputs.perturbed_grid(8, 0.1, 0.02, 4, zeldovich=True, total_mass=inputs.CRITICAL_MATTER_DENSITY)
    n = 20
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=prec, scheme=B.KDK_CANONICAL)
    try:
        sim.set_state(ic.x, ic.v)
        sim.adjoint_forward(TAU, n, 7)
        xT, vT, _, aT = sim.state()
        gxT, gvT, gmT = loss(xT, vT, ic.m, aT)
        g = sim.adjoint_backward(gxT, gvT, gmT)
    finally:
        sim.close()
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "canonical")
    gxT, gvT, gmT = loss(r["x"], r["v"], ic.m, r["schedule"]["a"][-1])
    ref = oracle.adjoint_run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n,
                             np.zeros_like(ic.x) if gxT is None else gxT, gvT, gmT,
                             scheme="canonical")
    return g, ref


def test_canonical_adjoint_fp64_random_covectors():
    rng = np.random.default_rng(750)
    cx, cv = rng.standard_normal((512, 3)), rng.standard_normal((512, 3))
    g, ref = adjoint_case(B.FP64, lambda xT, vT, m, aT: (cx, cv, None))
    for got, r, k in zip(g, ref, ("gx", "gv", "gm")):
        assert rel(got, r) < 1e-9, k


def test_canonical_adjoint_fp32_tracer_energy():
    # the tracer kinetic-energy loss: a 6e-8 change of the initial positions
    # moves its gradient by ~1e-5 in the oracle (random co-vectors on every
    # body: ~3e-4, beyond what any FP32 trajectory can match)
    tr = inputs.tracers(512, 64, 7)

    def loss(xT, vT, m, aT):
        gv = np.zeros_like(vT)
        gv[tr] = aT * aT * m[tr, None] * vT[tr]
        gm = np.zeros_like(m)
        gm[tr] = 0.5 * aT * aT * np.sum(vT[tr] ** 2, axis=1)
        return None, gv, gm

    g, ref = adjoint_case(B.FP32_COMP, loss)
    for got, r, k in zip(g, ref, ("gx", "gv", "gm")):
        assert rel(got, r) < 1e-4, k


def test_canonical_tangent_growth():
    ic = inputs.grid16(critical=True)
    seeds = [11, 3000]
    n = 10
    d = np.array([1.0, -1.0, 0.5])
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32, scheme=B.KDK_CANONICAL)
    try:
        sim.set_state(ic.x, ic.v)
        sim.tangent_init(seeds, n, d)
        sim.tangent_step(TAU, 6)
        sim.tangent_step(TAU, n - 6)
        growth = sim.tangent_growth()
    finally:
        sim.close()
    for b, s in enumerate(seeds):
        dx0 = np.zeros_like(ic.x)
        dx0[s] = d / np.linalg.norm(d)
        _, _, hist = oracle.tangent_run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n,
                                        dx0, np.zeros_like(ic.v), "canonical")
        ref = np.array([np.sqrt(np.sum(h[0][s] ** 2) + np.sum(h[1][s] ** 2)) for h in hist[1:]])
        np.testing.assert_allclose(growth[:, b], ref, rtol=1e-4)
