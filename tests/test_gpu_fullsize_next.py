"""The 'next' rows at the paper-scale size, in the configuration the
benchmark times (N = 32^3, FP32 compensated): sampled rows or whole-run
statistics against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1208_3444_b300 import binding as B
from paper_1208_3444_b300 import inputs

pytestmark = pytest.mark.gpu

LCDM_D = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
LCDM = oracle.Cosmology(0.0, 0.3, 0.0, 0.7, 1.0)
TAU = inputs.lcdm_tau(2000)


def rel_rms(a, b):
    return float(np.sqrt(np.mean(np.sum((a - b) ** 2, axis=1))) /
                 np.mean(np.linalg.norm(b, axis=1)))


def rows32(n, seed):
    return np.sort(np.random.default_rng(seed).choice(32768, n, replace=False))


def test_periodic_forces_grid32_sampled_rows():
    ic = inputs.grid32()
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, 1.0, prec=B.FP32_COMP)
    try:
        sim.set_state(ic.x)
        sim.set_periodic(1.0)
        got = sim.forces()
    finally:
        sim.close()
    rows = rows32(192, 900)
    # alpha L = 4 keeps the oracle's reciprocal sum small (|n| <= 9); the
    # result does not depend on alpha (pinned in test_oracle_ewald.py)
    ref = oracle.ewald_forces(ic.x, ic.m, ic.eps, 1.0, alpha=4.0, rows=rows)
    # On this near-uniform box the neutralised periodic force is ~30x smaller
    # than the pair terms it sums (their scale is the isolated pull), and the
    # FP32 arithmetic and the 1.5e-7 erfc bound act on the terms: the
    # compensated bound holds against the terms' scale, and 1e-5 against the
    # small total.
    iso = oracle.forces(ic.x, ic.m, ic.eps, rows=rows)
    err = np.sqrt(np.mean(np.sum((got[rows] - ref) ** 2, axis=1)))
    assert err < 1e-6 * np.mean(np.linalg.norm(iso, axis=1))
    assert rel_rms(got[rows], ref) < 1e-5


def test_deformation_forces_grid32_sampled_rows():
    ic = inputs.grid32()
    defo = (0.3, np.array([0.51, 0.47, 0.53]))
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, 1.0, prec=B.FP32_COMP)
    try:
        sim.set_state(ic.x)
        sim.set_deformation(*defo)
        got = sim.forces()
    finally:
        sim.close()
    rows = rows32(384, 901)
    ref = oracle.forces(ic.x, ic.m, ic.eps, rows=rows) + \
        oracle.deformation_force(ic.x[rows], defo[0], defo[1], ic.eps)
    assert rel_rms(got[rows], ref) < 1e-6


def test_canonical_steps_grid32_before_collapse():
    ic = inputs.grid32()
    n = 2
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32_COMP,
                       scheme=B.KDK_CANONICAL)
    try:
        sim.set_state(ic.x, ic.v)
        sim.step(TAU, n)
        x, v, t, a = sim.state()
    finally:
        sim.close()
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "canonical")
    assert np.abs(x - r["x"]).max() < 1e-5
    dv = np.linalg.norm(v - r["v"], axis=1)
    assert np.sqrt(np.mean(dv ** 2)) < 1e-5 * np.sqrt(np.mean(np.sum(r["v"] ** 2, axis=1)))


def test_tracer_spectrum_of_the_paper_scale_run():
    # the 32^3 run of 2000 steps from a = 1/51 with its 64 tracers recorded
    # every step; the spectrum of the recorded velocities against the oracle's
    ic = inputs.grid32()
    tr = inputs.tracers(ic.N, 64, 7)
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32_COMP)
    try:
        sim.set_state(ic.x, ic.v)
        sim.record_tracers(tr, 2000)
        sim.step(TAU, 2000)
        rec = sim.read_tracers()
        E = sim.tracer_spectrum(TAU, "hann")
        _, _, t, a = sim.state()
    finally:
        sim.close()
    assert rec.shape == (2000, 64, 6) and np.all(np.isfinite(rec))
    assert a == pytest.approx(1.0, abs=2e-3)          # tau was chosen to reach a = 1 in 2000 steps
    ref = oracle.velocity_spectrum(rec[:, :, 3:].astype(np.float64), TAU, "hann")
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(E - ref) <= 1e-9 * np.abs(ref) + 1e-10 * scale)


def test_periodic_force_vjp_grid32_sampled_rows():
    # the periodic force VJP the benchmark times (32^3, FP32 compensated
    # context, unit box), on 192 sampled rows against the oracle's FP64
    # ewald_vjp (alpha L = 4 for a small oracle k-sum; alpha does not matter,
    # pinned in test_oracle_ewald_derivatives.py)
    ic = inputs.grid32()
    w = inputs.f32(np.random.default_rng(901).standard_normal(ic.x.shape))
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, 1.0, prec=B.FP32_COMP)
    try:
        sim.set_state(ic.x)
        sim.set_periodic(1.0)
        gx, gm = sim.force_vjp(w)
    finally:
        sim.close()
    rows = rows32(192, 902)
    rx, rm = oracle.ewald_vjp(ic.x, ic.m, w, ic.eps, 1.0, alpha=4.0, rows=rows)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert rel(gx[rows], rx) < 1e-5
    assert rel(gm[rows], rm) < 1e-5
