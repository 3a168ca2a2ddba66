"""GPU parity of feature combinations against the FP64 oracle: the canonical
(symplectic) KDK with the Eq. 6 deformation term and with periodic
boundaries, and precision switches while periodic boundaries are on.

Trajectory tolerances as in the single-feature tests: positions 1e-5 (FP32
modes) and 1e-9 (FP64) in max abs; velocities RMS-relative 1e-5 and 1e-11.
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
PRECS = [B.FP32, B.FP32_COMP, B.FP64]


def rms(d):
    return float(np.sqrt(np.mean(np.sum(d ** 2, axis=1))))


def check(x, v, r, prec):
    assert np.abs(x - r["x"]).max() < (1e-9 if prec == B.FP64 else 1e-5)
    assert rms(v - r["v"]) < (1e-11 if prec == B.FP64 else 1e-5) * rms(r["v"])


@pytest.mark.parametrize("prec", PRECS)
def test_canonical_steps_with_deformation(prec):
    # the deformation cases' setting: 16^3 at the background density from
    # a = 0.5, a point mass of 30 % of the box's mass between grid nodes
    ic = inputs.grid16(critical=True)
    a0, xpsi = 0.5, np.array([0.5, 0.5, 0.5])
    cpsi = 0.3 * float(np.sum(ic.m))
    n = 10
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, a0, prec=prec, scheme=B.KDK_CANONICAL)
    try:
        sim.set_state(ic.x, ic.v)
        sim.set_deformation(cpsi, xpsi)
        sim.step(TAU, 3)
        sim.step(TAU, n - 3)
        x, v, t, a = sim.state()
    finally:
        sim.close()
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, a0, TAU, n, "canonical", defo=(cpsi, xpsi))
    r0 = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, a0, TAU, n, "canonical")
    assert rms(r["v"] - r0["v"]) > 1e3 * (1e-11 if prec == B.FP64 else 1e-5) * rms(r["v"])
    check(x, v, r, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_canonical_steps_with_periodic_boundaries(prec):
    ic = inputs.perturbed_grid(8, 0.1, 0.02, 4, zeldovich=True, total_mass=inputs.CRITICAL_MATTER_DENSITY)
    n = 10
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=prec, scheme=B.KDK_CANONICAL)
    try:
        sim.set_state(ic.x, ic.v)
        sim.set_periodic(1.0)
        sim.step(TAU, 4)
        sim.step(TAU, n - 4)
        x, v, t, a = sim.state()
    finally:
        sim.close()
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "canonical", box=1.0)
    check(x, v, r, prec)


def test_precision_switches_with_periodic_boundaries():
    # the Ewald parameters follow the precision (FP32 modes share them; FP64
    # takes a larger alpha and nk), and the forces follow the switch
    rng = np.random.default_rng(960)
    x, m = inputs.f32(rng.random((2000, 3))), inputs.f32(rng.random(2000) / 2000)
    ref = oracle.ewald_forces(x, m, 0.01, 1.0)
    sim = B.Simulation(m, 0.01, LCDM_D, 1.0, prec=B.FP32)
    try:
        sim.set_state(x)
        sim.set_periodic(1.0)
        p32 = sim.periodic_params()
        errs = {}
        for prec in (B.FP64, B.FP32_COMP, B.FP32, B.FP64):
            sim.configure(prec=prec)
            f = sim.forces()
            errs.setdefault(prec, []).append(rms(f - ref) / np.mean(np.linalg.norm(ref, axis=1)))
            p = sim.periodic_params()
            assert (p["nk"] > p32["nk"]) == (prec == B.FP64)
    finally:
        sim.close()
    assert max(errs[B.FP64]) < 1e-11
    assert max(errs[B.FP32_COMP]) < 1e-6 and max(errs[B.FP32]) < 1e-5
