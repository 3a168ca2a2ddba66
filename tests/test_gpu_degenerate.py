"""GPU parity on the degenerate inputs of Eq. 1 against the FP64 oracle.

* coincident bodies (d = 0 between distinct bodies: each such pair adds
  nothing to the force, and J(0) = I / eps^3 to the VJP);
* every body at one point (all forces exactly zero);
* massless bodies (they feel the field but pull nothing);
* a far outlier (its pull on the cluster and the cluster's on it span many
  orders of magnitude);
* equal masses with a ragged size, where the padding must contribute nothing.

Tolerances as in test_gpu_forces.py: RMS over bodies of the force error
relative to the mean abs(F): 1e-5 FP32, 1e-6 FP32 compensated, 1e-11 FP64;
VJPs normwise 1e-5 (FP32) and 1e-10 (FP64).
"""
import numpy as np
import pytest

import oracle
from paper_1208_3444_b300 import binding as B
from paper_1208_3444_b300 import inputs

pytestmark = pytest.mark.gpu

LCDM = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
TOL = {B.FP32: 1e-5, B.FP32_COMP: 1e-6, B.FP64: 1e-11}
VJP_TOL = {B.FP32: 1e-5, B.FP64: 1e-10}
PRECS = [B.FP32, B.FP32_COMP, B.FP64]


def rel_rms(a, b):
    return float(np.sqrt(np.mean(np.sum((a - b) ** 2, axis=1))) /
                 np.mean(np.linalg.norm(b, axis=1)))


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def run(x, m, eps, prec, w=None):
    sim = B.Simulation(m, eps, LCDM, 1.0, prec=prec)
    try:
        sim.set_state(x)
        f = sim.forces()
        g = sim.force_vjp(w) if w is not None else None
    finally:
        sim.close()
    return f, g


def coincident_system(N, seed):
    rng = np.random.default_rng(seed)
    x = rng.random((N, 3))
    x[: N // 3] = x[0]                      # a third of the bodies at one point
    x[N // 3: N // 2] = x[N // 3]           # another group at a second point
    m = rng.lognormal(0.0, 0.5, N) / N
    m[::7] = 0.0                            # massless bodies among them
    return inputs.f32(x), inputs.f32(m), inputs.f32(rng.standard_normal((N, 3)))


@pytest.mark.parametrize("prec", PRECS)
def test_coincident_and_massless_bodies(prec):
    x, m, w = coincident_system(1500, 900)
    eps = 0.01
    f, g = run(x, m, eps, prec, w if prec != B.FP32_COMP else None)
    assert rel_rms(f, oracle.forces(x, m, eps)) < TOL[prec]
    # a body with no pull of its own still feels the others
    assert np.all(np.linalg.norm(f[::7], axis=1) > 0)
    if g is not None:
        rx, rm = oracle.vjp(x, m, w, eps)
        assert rel(g[0], rx) < VJP_TOL[prec]
        assert rel(g[1], rm) < VJP_TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_every_body_at_one_point(prec):
    N = 777
    x = np.tile(np.array([[0.25, 0.5, 0.75]]), (N, 1))
    m = np.full(N, 1.0 / N)
    f, _ = run(x, m, 0.01, prec)
    assert np.all(f == 0.0)


@pytest.mark.parametrize("prec", PRECS)
def test_far_outlier(prec):
    rng = np.random.default_rng(901)
    N = 1000
    x = rng.random((N, 3))
    x[-1] = (1e4, -2e4, 3e4)
    m = inputs.f32(rng.lognormal(0.0, 0.5, N) / N)
    x = inputs.f32(x)
    eps = 0.01
    f, _ = run(x, m, eps, prec)
    ref = oracle.forces(x, m, eps)
    assert rel_rms(f[:-1], ref[:-1]) < TOL[prec]
    # the outlier feels the cluster as one point mass: relative error per component
    assert np.max(np.abs(f[-1] - ref[-1]) / np.abs(ref[-1])) < (1e-5 if prec != B.FP64 else 1e-11)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [2049, 5000])
def test_equal_masses_ragged_size(N, prec):
    rng = np.random.default_rng(902 + N)
    x = inputs.f32(rng.random((N, 3)))
    m = inputs.f32(np.full(N, 1.0 / N))
    eps = 0.005
    f, _ = run(x, m, eps, prec)
    assert rel_rms(f, oracle.forces(x, m, eps)) < TOL[prec]
