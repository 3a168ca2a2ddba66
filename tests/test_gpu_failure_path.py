"""The device-side failure path, exercised without a fault: a bounded wait on
a barrier that nothing completes gives up, raises the timeout flag, the host
reports COLATUS_E_TIMEOUT, and the context keeps working."""
import time

import numpy as np
import pytest

import oracle
from paper_1208_3444_b300 import binding as B
from paper_1208_3444_b300 import inputs

pytestmark = pytest.mark.gpu

LCDM_D = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)


def test_bounded_wait_times_out_and_the_context_stays_usable():
    ic = inputs.grid8()
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, 1.0, prec=B.FP32)
    try:
        sim.set_state(ic.x)
        t0 = time.perf_counter()
        with pytest.raises(B.ColatusError) as e:
            B.colatus_selftest_wait(sim.h, 2_000_000)        # about 1 ms of SM cycles
        assert e.value.status == B.E_TIMEOUT
        assert "gave up" in str(e.value)
        assert time.perf_counter() - t0 < 5.0
        got = sim.forces()                                   # flag cleared, context usable
        sim.synchronize()
        with pytest.raises(B.ColatusError) as e:
            B.colatus_selftest_wait(sim.h, 0)
        assert e.value.status == B.E_ARG
    finally:
        sim.close()
    ref = oracle.forces(ic.x, ic.m, ic.eps)
    assert np.sqrt(np.mean(np.sum((got - ref) ** 2, 1))) < 1e-5 * np.mean(np.linalg.norm(ref, axis=1))
