"""GPU parity of the derivative kernels at the full 32^3 size, in the launch
configurations the benchmark times, against the FP64 oracle:

* the force VJP (the adjoint's kernel; every 32^3 i-tile takes the scaled
  form) on 512 seeded rows, normwise 1e-5 as for the small systems;
* the tangent model with the benchmark's 64 single-tracer tangents over two
  KDK steps, checked for 3 of the tracers against the oracle's tangent run
  (which evaluates every force and JVP row), 1e-4 relative as for the small
  systems.
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


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def test_vjp_grid32_sampled_rows():
    ic = inputs.grid32()
    w = inputs.f32(np.random.default_rng(950).standard_normal((ic.N, 3)))
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32_COMP)
    try:
        sim.set_state(ic.x, ic.v)
        gx, gm = sim.force_vjp(w)
    finally:
        sim.close()
    rows = np.sort(np.random.default_rng(951).choice(ic.N, 512, replace=False))
    rx, rm = oracle.vjp(ic.x, ic.m, w, ic.eps, rows=rows)
    s = 1.0 / inputs.A_START ** 3
    assert rel(gx[rows], s * rx) < 1e-5
    assert rel(gm[rows], s * rm) < 1e-5


def test_tangent_grid32_benchmark_tracers():
    ic = inputs.grid32()
    seeds = inputs.tracers(ic.N, 64, 7)
    n = 2
    d = np.array([1.0, 0.0, 0.0])
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32)
    try:
        sim.set_state(ic.x, ic.v)
        sim.tangent_init(seeds, n, d)
        sim.tangent_step(TAU, n)
        growth = sim.tangent_growth()
    finally:
        sim.close()
    assert growth.shape == (n, 64) and np.all(np.isfinite(growth))
    for b in (0, 31, 63):
        s = seeds[b]
        dx0 = np.zeros_like(ic.x)
        dx0[s] = d
        _, _, hist = oracle.tangent_run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n,
                                        dx0, np.zeros_like(ic.v), "kdk")
        ref = np.array([np.sqrt(np.sum(h[0][s] ** 2) + np.sum(h[1][s] ** 2)) for h in hist[1:]])
        np.testing.assert_allclose(growth[:, b], ref, rtol=1e-4)
