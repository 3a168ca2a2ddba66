"""GPU parity of the tangent-linear model under periodic boundaries (Sec. II;
Ewald summation) against the oracle's FP64 tangent_run with box = L, for
single-tracer seeds, through KDK and DKD steps: the real-space periodic JVP
kernel and the per-tangent reciprocal-space JVP."""
import functools

import numpy as np
import pytest

import oracle
from paper_1208_3444_b300 import binding as B
from paper_1208_3444_b300 import inputs

pytestmark = pytest.mark.gpu

LCDM_D = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
LCDM = oracle.Cosmology(0.0, 0.3, 0.0, 0.7, 1.0)
TAU = inputs.lcdm_tau(2000)
D = np.array([1.0, 2.0, -0.5])
NSTEPS = 8


def case():
    # 6^3 bodies at the background density in the unit periodic box
    return inputs.perturbed_grid(6, 0.1, 0.02, 4, zeldovich=True,
                                 total_mass=inputs.CRITICAL_MATTER_DENSITY)


@functools.lru_cache(maxsize=None)
def oracle_growth(seed, scheme="kdk"):
    ic = case()
    dx0 = np.zeros_like(ic.x)
    dx0[seed] = D / np.linalg.norm(D)
    _, _, hist = oracle.tangent_run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, NSTEPS,
                                    dx0, np.zeros_like(ic.v), scheme, box=1.0)
    return np.array([np.sqrt(np.sum(h[0][seed] ** 2) + np.sum(h[1][seed] ** 2)) for h in hist[1:]])


@pytest.mark.parametrize("seeds,check,scheme", [([5, 100, 215], [0, 1, 2], "kdk"),
                                                ([0, 3, 7, 50, 99, 120, 150, 180, 201], [0, 8], "kdk"),
                                                ([5, 100, 215], [0, 2], "dkd")])
def test_periodic_tracer_growth_matches_oracle_tangent(seeds, check, scheme):
    # the second case has 9 tangents: a full chunk of 8 and a partial one;
    # the third takes the paper's DKD steps (JVP at the half-drift positions)
    ic = case()
    sch = B.KDK if scheme == "kdk" else B.DKD
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32, scheme=sch)
    try:
        sim.set_state(ic.x, ic.v)
        sim.set_periodic(1.0)
        sim.tangent_init(seeds, NSTEPS, D)
        sim.tangent_step(TAU, 3)
        sim.tangent_step(TAU, NSTEPS - 3)
        growth = sim.tangent_growth()
        xs, vs, _, _ = sim.state()
    finally:
        sim.close()
    assert growth.shape == (NSTEPS, len(seeds))
    for b in check:
        np.testing.assert_allclose(growth[:, b], oracle_growth(seeds[b], scheme), rtol=1e-4)
    # the state advanced exactly as colatus_step advances it
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32, scheme=sch)
    try:
        sim.set_state(ic.x, ic.v)
        sim.set_periodic(1.0)
        sim.step(TAU, NSTEPS)
        xp, vp, _, _ = sim.state()
    finally:
        sim.close()
    assert np.array_equal(xs, xp) and np.array_equal(vs, vp)
