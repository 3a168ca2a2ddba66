"""Failure detection through a step: the device's non-finite flag.

Every step epilogue checks the positions and velocities it writes and raises
a device flag when one is not finite; the host reports COLATUS_E_NONFINITE at
the next synchronising call and clears the flag.  These tests feed finite
inputs whose force overflows in the first step, so the flag is raised by the
device arithmetic, not by host-side validation: two bodies at +-3e38 (FP32)
or +-1e308 (FP64) have a coordinate difference that overflows to infinity,
so 1/s is 0 and the pair term inf * 0 is NaN (IEEE arithmetic, no fault).  A
second case scales G so that the FP64 kick coefficient no longer fits in a
float.  Afterwards the same context takes a fresh state and steps on, matching
the oracle.
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
HUGE = {B.FP32: 3e38, B.FP32_COMP: 3e38, B.FP64: 1e308}


def _far_pair(x, prec):
    bad = np.asarray(x, dtype=np.float64).copy()
    bad[5] = (HUGE[prec], 0.25, 0.5)
    bad[9] = (-HUGE[prec], 0.25, 0.5)
    return bad


def _continue_from_oracle(ic, a_from, n):
    # the schedule depends on a only, so the oracle restarted at a_from
    # reproduces the context's continued clock
    return oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, a_from, TAU, n, "kdk")


@pytest.mark.parametrize("scheme", [B.KDK, B.DKD])
@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP, B.FP64])
def test_overflowing_pair_raises_nonfinite_then_context_recovers(prec, scheme):
    ic = inputs.grid16(critical=True)
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=prec, scheme=scheme)
    try:
        sim.set_state(_far_pair(ic.x, prec), ic.v)       # finite: host validation passes
        with pytest.raises(B.ColatusError) as e:
            sim.step(TAU, 2)
            sim.synchronize()
        assert e.value.status == B.E_NONFINITE
        sim.synchronize()                                 # the flag was cleared
        # a fresh state on the same context steps on and matches the oracle
        sim.set_state(ic.x, ic.v)
        sim.step(TAU, 2)
        x, v, t, a = sim.state()
    finally:
        sim.close()
    a2 = oracle.schedule(LCDM, inputs.A_START, TAU, 2, "kdk")["a"][-1]
    sch = "kdk" if scheme == B.KDK else "dkd"
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, a2, TAU, 2, sch)
    tol = 1e-9 if prec == B.FP64 else 1e-5
    assert np.abs(x - r["x"]).max() < tol
    assert a == pytest.approx(r["schedule"]["a"][-1], rel=1e-13)
    assert t == pytest.approx(4 * TAU, rel=1e-13)


def test_overflowing_kick_coefficient_raises_nonfinite():
    # G = 1e300: the FP64 kick coefficient G d rounds to +inf in float
    ic = inputs.grid16(critical=True)
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32_COMP, G=1e300)
    try:
        sim.set_state(ic.x, ic.v)
        with pytest.raises(B.ColatusError) as e:
            sim.step(TAU, 1)
            sim.synchronize()
        assert e.value.status == B.E_NONFINITE
        sim.configure(G=1.0)
        sim.set_state(ic.x, ic.v)
        sim.step(TAU, 1)
        x = sim.state()[0]
    finally:
        sim.close()
    a1 = oracle.schedule(LCDM, inputs.A_START, TAU, 1, "kdk")["a"][-1]
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, a1, TAU, 1, "kdk")
    assert np.abs(x - r["x"]).max() < 1e-5


def _ensemble(counts, seed=9):
    ics = []
    for r, N in enumerate(counts):
        n = int(np.ceil(N ** (1.0 / 3.0) - 1e-9))
        ics.append(inputs.perturbed_grid(n, 0.1, 0.02, seed * 100 + r, zeldovich=True, count=N,
                                         total_mass=inputs.CRITICAL_MATTER_DENSITY))
    x = np.concatenate([ic.x for ic in ics])
    v = np.concatenate([ic.v for ic in ics])
    m = np.concatenate([ic.m for ic in ics])
    return ics, x, v, m, np.array([ic.eps for ic in ics]), np.array([ic.N for ic in ics])


@pytest.mark.parametrize("nsteps", [1, 16])   # a direct step, and one captured-graph replay
def test_ensemble_overflowing_pair_raises_nonfinite_then_recovers(nsteps):
    ics, x, v, m, eps, Ns = _ensemble([300, 700, 1000])
    bad = np.asarray(x, dtype=np.float64).copy()
    off = np.concatenate([[0], np.cumsum(Ns)])
    bad[off[1] + 3] = (3e38, 0.5, 0.5)       # one pair inside the second realisation
    bad[off[1] + 8] = (-3e38, 0.5, 0.5)
    ens = B.Ensemble(Ns, m, eps, LCDM_D, inputs.A_START)
    try:
        ens.set_state(bad, np.asarray(v, dtype=np.float64))
        with pytest.raises(B.ColatusError) as e:
            ens.step(TAU, nsteps)
            ens.synchronize()
        assert e.value.status == B.E_NONFINITE
        ens.synchronize()
        ens.set_state(x, v)
        ens.step(TAU, 2)
        gx, gv, t, a = ens.state()
    finally:
        ens.close()
    a0 = oracle.schedule(LCDM, inputs.A_START, TAU, nsteps, "kdk")["a"][-1]
    for r, ic in enumerate(ics):
        ref = _continue_from_oracle(ic, a0, 2)
        assert np.abs(gx[off[r]:off[r + 1]] - ref["x"]).max() < 1e-5, r
        assert a == pytest.approx(ref["schedule"]["a"][-1], rel=1e-13)
