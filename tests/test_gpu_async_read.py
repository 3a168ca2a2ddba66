"""Asynchronous state read-back (colatus_get_state_async) returns exactly what
the synchronous colatus_get_state returns at the same point of the run."""
import numpy as np
import pytest

from paper_1208_3444_b300 import binding as B
from paper_1208_3444_b300 import inputs

pytestmark = pytest.mark.gpu

LCDM_D = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
TAU = inputs.lcdm_tau(2000)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_async_reads_match_synchronous_reads(dtype):
    import torch
    ic = inputs.grid16(critical=True)
    n = 10
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32_COMP)
    try:
        sim.set_state(ic.x, ic.v)
        tdt = torch.float32 if dtype == np.float32 else torch.float64
        bufs = [(torch.empty((ic.N, 3), dtype=tdt).pin_memory(),
                 torch.empty((ic.N, 3), dtype=tdt).pin_memory()) for _ in range(n)]
        for k in range(n):            # more read-backs in flight than slots
            sim.step(TAU, 1)
            B.colatus_get_state_async(sim.h, *bufs[k])
        B.colatus_wait_state(sim.h)
        got = [(a.numpy().copy(), b.numpy().copy()) for a, b in bufs]
    finally:
        sim.close()
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32_COMP)
    try:
        sim.set_state(ic.x, ic.v)
        for k in range(n):
            sim.step(TAU, 1)
            x, v, _, _ = sim.state(dtype=dtype)
            assert np.array_equal(got[k][0], x) and np.array_equal(got[k][1], v), k
    finally:
        sim.close()


def test_async_read_argument_checks():
    ic = inputs.grid8()
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START)
    try:
        x = np.empty((ic.N, 3))
        with pytest.raises(B.ColatusError):
            B.colatus_get_state_async(sim.h, x, None)            # no state yet
        sim.set_state(ic.x, ic.v)
        with pytest.raises(ValueError):
            B.colatus_get_state_async(sim.h, np.empty((ic.N, 3), dtype=np.int32), None)
        with pytest.raises(ValueError):
            B.colatus_get_state_async(sim.h, np.empty((3, ic.N)).T, None)   # not C-contiguous
        B.colatus_get_state_async(sim.h, x, None)
        B.colatus_wait_state(sim.h)
        xs, _, _, _ = sim.state()
        np.testing.assert_array_equal(x, xs)
    finally:
        sim.close()
