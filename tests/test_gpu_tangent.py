"""GPU parity of the tangent-linear model (JVP of Eq. 1 through the KDK and
DKD steps) against the oracle's FP64 tangent, for single-tracer seeds; a
change of step size or scheme between calls against the oracle's tangent
run in two legs."""
import numpy as np
import pytest

import oracle
from paper_1208_3444_b300 import binding as B
from paper_1208_3444_b300 import inputs

pytestmark = pytest.mark.gpu

LCDM_D = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
LCDM = oracle.Cosmology(0.0, 0.3, 0.0, 0.7, 1.0)
TAU = inputs.lcdm_tau(2000)


@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
@pytest.mark.parametrize("seeds", [[5, 1000, 4000], [0, 17, 333, 2222, 4095]])
def test_tracer_growth_matches_oracle_tangent(seeds, scheme):
    ic = inputs.grid16(critical=True)
    n = 10
    d = np.array([1.0, 2.0, -0.5])
    sch = B.KDK if scheme == "kdk" else B.DKD
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32, scheme=sch)
    try:
        sim.set_state(ic.x, ic.v)
        sim.tangent_init(seeds, n, d)
        sim.tangent_step(TAU, 4)
        sim.tangent_step(TAU, n - 4)
        growth = sim.tangent_growth()
        xs, vs, t, a = sim.state()
    finally:
        sim.close()
    assert growth.shape == (n, len(seeds))
    for b, s in enumerate(seeds):
        dx0 = np.zeros_like(ic.x)
        dx0[s] = d / np.linalg.norm(d)
        _, _, hist = oracle.tangent_run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n,
                                        dx0, np.zeros_like(ic.v), scheme)
        ref = np.array([np.sqrt(np.sum(h[0][s] ** 2) + np.sum(h[1][s] ** 2)) for h in hist[1:]])
        np.testing.assert_allclose(growth[:, b], ref, rtol=1e-4)
    # the state advanced exactly as colatus_step advances it
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32, scheme=sch)
    try:
        sim.set_state(ic.x, ic.v)
        sim.step(TAU, n)
        xp, vp, _, _ = sim.state()
    finally:
        sim.close()
    assert np.array_equal(xs, xp) and np.array_equal(vs, vp)


def test_tangent_state_checks():
    ic = inputs.grid16(critical=True)
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32)
    try:
        sim.set_state(ic.x, ic.v)
        sim.tangent_init([3], 5)
        sim.step(TAU, 1)
        with pytest.raises(B.ColatusError) as e:
            sim.tangent_step(TAU, 1)
        assert e.value.status == B.E_STATE
    finally:
        sim.close()


@pytest.mark.parametrize("second", ["smaller_step", "dkd", "canonical"])
def test_step_size_or_scheme_change_between_calls(second):
    # 4 KDK steps, then 6 more with a smaller step or another scheme: the
    # tangent re-opens from (dx, dv) at the state's step, as the state does
    ic = inputs.grid16(critical=True)
    seeds, d = [5, 1000, 4000], np.array([1.0, 2.0, -0.5])
    tau2 = TAU if second != "smaller_step" else 0.7 * TAU
    sch2 = {"smaller_step": B.KDK, "dkd": B.DKD, "canonical": B.KDK_CANONICAL}[second]
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32)
    try:
        sim.set_state(ic.x, ic.v)
        sim.tangent_init(seeds, 10, d)
        sim.tangent_step(TAU, 4)
        a4 = sim.state()[3]
        sim.configure(scheme=sch2)
        sim.tangent_step(tau2, 6)
        growth = sim.tangent_growth()
    finally:
        sim.close()
    for b, s in enumerate(seeds):
        dx0 = np.zeros_like(ic.x)
        dx0[s] = d / np.linalg.norm(d)
        dx4, dv4, h1 = oracle.tangent_run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, 4,
                                          dx0, np.zeros_like(ic.v), "kdk")
        r4 = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, 4, "kdk")
        assert r4["schedule"]["a"][-1] == pytest.approx(a4, rel=1e-12)
        _, _, h2 = oracle.tangent_run(r4["x"], r4["v"], ic.m, ic.eps, 1.0, LCDM, a4, tau2, 6, dx4, dv4,
                                      {"smaller_step": "kdk", "dkd": "dkd", "canonical": "canonical"}[second])
        hist = h1[1:] + h2[1:]
        ref = np.array([np.sqrt(np.sum(h[0][s] ** 2) + np.sum(h[1][s] ** 2)) for h in hist])
        np.testing.assert_allclose(growth[:, b], ref, rtol=1e-4)
