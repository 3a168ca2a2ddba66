"""The chaos horizon of the workloads, measured with the oracle alone.

The m = 1/N boxes hold 28x the background matter density, so they collapse
within ~5 steps of the 2000-step schedule; after that, a rounding-sized
(6e-8 relative) change of the initial positions grows past 1e-4 in the FP64
oracle itself.  Element-wise position parity of any float32 path is therefore
only meaningful before the collapse, or for boxes at the background density,
where the same perturbation stays below 1e-6 for 10 steps.  In FP64 the
collapse multiplies a 1e-15 change by ~1e6 over 20 steps (to 2.4e-9)."""
import numpy as np

import oracle
from paper_1208_3444_b300 import inputs

LCDM = oracle.Cosmology(0.0, 0.3, 0.0, 0.7, 1.0)
TAU = inputs.lcdm_tau(2000)


def _growth(ic, n):
    rng = np.random.default_rng(0)
    xp = ic.x * (1.0 + 6e-8 * rng.standard_normal(ic.x.shape))
    a = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "kdk",
                   keep_states=True)
    b = oracle.run(xp, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "kdk",
                   keep_states=True)
    return [np.abs(sa[0] - sb[0]).max() for sa, sb in zip(a["states"], b["states"])]


def test_overdense_box_collapses_and_amplifies_rounding():
    d = _growth(inputs.grid16(), 8)   # d[n]: difference after n steps
    assert max(d[:4]) < 1e-6          # before collapse: rounding stays rounding
    assert min(d[5:]) > 1e-4          # after collapse: amplified by >1e3


def test_overdense_32cubed_box_collapses_after_two_steps():
    d = _growth(inputs.grid32(), 3)
    assert max(d[:3]) < 1e-6 and d[3] > 1e-4


def test_critical_density_box_stays_regular_for_ten_steps():
    d = _growth(inputs.grid16(critical=True), 10)
    assert max(d) < 1e-6
