"""GPU parity at sizes on and around the launch plans' tile boundaries.

The FP32 force takes 2048-body i-tiles and 512-body j-tiles, the VJP 1024 and
256, the FP64 kernels their own; every size below is a tile multiple, one
off it, or a prime, so full tiles, ragged tails and single-body tails all
occur.  Equal masses select the kernels' equal-mass form (one lane-op fewer
per pair), lognormal masses the general one.  Above 20000 bodies the oracle
evaluates 512 seeded rows against every source.

Tolerances as in test_gpu_forces.py and test_gpu_adjoint.py: force RMS over
bodies relative to the mean abs(F), 1e-5 FP32, 1e-6 FP32 compensated, 1e-11
FP64; VJP normwise 1e-5 (FP32) and 1e-10 (FP64); tangent growth 1e-4; the
potential energy W of the diagnostics 1e-6 (FP32 modes) and 1e-11 (FP64).
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
TOL = {B.FP32: 1e-5, B.FP32_COMP: 1e-6, B.FP64: 1e-11}
SIZES = [511, 512, 513, 1024, 1025, 2047, 2048, 2049, 4097, 10007, 32769, 65537]
SAMPLE_ABOVE = 20000
VJP_SIZES = [n for n in SIZES if n <= 32769]   # the FP32 VJP's bound holds to the 32^3 scale


def rel_rms(a, b):
    return float(np.sqrt(np.mean(np.sum((a - b) ** 2, axis=1))) /
                 np.mean(np.linalg.norm(b, axis=1)))


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def system(N, equal, seed):
    rng = np.random.default_rng(seed)
    x = inputs.f32(rng.random((N, 3)))
    m = np.full(N, 1.0 / N) if equal else rng.lognormal(0.0, 0.5, N) / N
    w = inputs.f32(rng.standard_normal((N, 3)))
    return x, inputs.f32(m), w


def rows_for(N, seed):
    if N <= SAMPLE_ABOVE:
        return None
    return np.sort(np.random.default_rng(seed).choice(N, 512, replace=False))


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP, B.FP64])
@pytest.mark.parametrize("equal", [True, False])
@pytest.mark.parametrize("N", SIZES)
def test_forces_at_tile_boundaries(N, equal, prec):
    x, m, _ = system(N, equal, 7000 + N)
    eps = 0.003
    sim = B.Simulation(m, eps, LCDM_D, 1.0, prec=prec)
    try:
        sim.set_state(x)
        f = sim.forces()
    finally:
        sim.close()
    rows = rows_for(N, 7100 + N)
    ref = oracle.forces(x, m, eps, rows=rows)
    got = f if rows is None else f[rows]
    assert rel_rms(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec,tol", [(B.FP32, 1e-5), (B.FP64, 1e-10)])
@pytest.mark.parametrize("equal", [True, False])
@pytest.mark.parametrize("N", VJP_SIZES)
def test_vjp_at_tile_boundaries(N, equal, prec, tol):
    x, m, w = system(N, equal, 7200 + N)
    eps = 0.003
    sim = B.Simulation(m, eps, LCDM_D, 1.0, prec=prec)
    try:
        sim.set_state(x)
        gx, gm = sim.force_vjp(w)
    finally:
        sim.close()
    rows = rows_for(N, 7300 + N)
    rx, rm = oracle.vjp(x, m, w, eps, rows=rows)
    if rows is not None:
        gx, gm = gx[rows], gm[rows]
    assert rel(gx, rx) < tol
    assert rel(gm, rm) < tol


@pytest.mark.parametrize("B_", [1, 7, 8, 9, 17])
def test_tangent_chunks_and_ragged_size(B_):
    # 8 tangents share one pass: 7, 8, 9 and 17 give a partial, a full, a
    # full plus one, and two full chunks plus one; 4001 bodies are not a
    # multiple of any tile
    ic = inputs.grid16(critical=True)
    N = 4001
    x, v, m = ic.x[:N], ic.v[:N], ic.m[:N]
    seeds = np.sort(np.random.default_rng(7400 + B_).choice(N, B_, replace=False))
    n = 3
    d = np.array([0.3, -1.0, 0.6])
    sim = B.Simulation(m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32)
    try:
        sim.set_state(x, v)
        sim.tangent_init(seeds, n, d)
        sim.tangent_step(TAU, n)
        growth = sim.tangent_growth()
    finally:
        sim.close()
    assert growth.shape == (n, B_)
    for b, s in enumerate(seeds):
        dx0 = np.zeros_like(x)
        dx0[s] = d / np.linalg.norm(d)
        _, _, hist = oracle.tangent_run(x, v, m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n,
                                        dx0, np.zeros_like(v), "kdk")
        ref = np.array([np.sqrt(np.sum(h[0][s] ** 2) + np.sum(h[1][s] ** 2)) for h in hist[1:]])
        np.testing.assert_allclose(growth[:, b], ref, rtol=1e-4)


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP, B.FP64])
@pytest.mark.parametrize("N", [1, 2, 255, 1023, 1025, 4097, 10007])
def test_potential_energy_at_tile_boundaries(N, prec):
    # W of the diagnostics: the tiled pair sums with the self pair masked in
    # the tiles that hold it, against the oracle's potential
    x, m, _ = system(N, False, 7500 + N)
    eps = 0.003
    sim = B.Simulation(m, eps, LCDM_D, 1.0, prec=prec)
    try:
        sim.set_state(x)
        W = sim.diagnostics()["W"]
    finally:
        sim.close()
    ref = oracle.diagnostics(x, np.zeros_like(x), m, 1.0, eps, 1.0)["W"]
    if N == 1:
        assert W == 0.0 and ref == 0.0
        return
    assert W == pytest.approx(ref, rel=1e-11 if prec == B.FP64 else 1e-6)
