"""GPU parity of the derivatives under periodic boundaries (Sec. II; Ewald
summation): the force VJP against the oracle's converged FP64 ewald_vjp, and
the checkpointed discrete adjoint of the KDK and DKD leapfrogs against the
oracle's exact transpose (adjoint_run with box = L).

Tolerances as for isolated boundaries: normwise relative error of the
gradient vector, FP32 VJP 1e-5, FP64 1e-10; FP32 trajectory adjoint 1e-4,
FP64 1e-9."""
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
VJP_TOL = {B.FP32: 1e-5, B.FP32_COMP: 1e-5, B.FP64: 1e-10}


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def periodic_vjp(x, m, w, eps, L, prec, a, G):
    sim = B.Simulation(m, eps, LCDM_D, a, prec=prec, G=G)
    try:
        sim.set_state(x)
        sim.set_periodic(L)
        return sim.force_vjp(w)
    finally:
        sim.close()


def vjp_case(N):
    rng = np.random.default_rng(900 + N)
    L = 2.5
    x = inputs.f32(L * rng.random((N, 3)))
    m = inputs.f32(rng.lognormal(0.0, 0.5, N) / N)
    w = inputs.f32(rng.standard_normal((N, 3)))
    return x, m, w, L


@functools.lru_cache(maxsize=None)
def vjp_reference(N, eps, G):
    x, m, w, L = vjp_case(N)
    return oracle.ewald_vjp(x, m, w, eps, L, G)


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP, B.FP64])
@pytest.mark.parametrize("N", [2, 37, 257, 3000])
def test_periodic_force_vjp_matches_oracle(N, prec):
    x, m, w, L = vjp_case(N)
    eps, a, G = 0.01, 0.5, 1.3
    gx, gm = periodic_vjp(x, m, w, eps, L, prec, a, G)
    rx, rm = vjp_reference(N, eps, G)
    s = 1.0 / a ** 3
    assert rel(gx, s * rx) < VJP_TOL[prec]
    assert rel(gm, s * rm) < VJP_TOL[prec]


def clustered_case():
    # clustered bodies (close pairs inside the real-space series region), some
    # moved by whole boxes (the minimum image is taken per pair)
    ic = inputs.plummer_clusters(2000, 19)
    x = ic.x.copy()
    x[::7] += np.array([1.0, -2.0, 0.0])
    rng = np.random.default_rng(930)
    return inputs.f32(x), ic.m, inputs.f32(rng.standard_normal(x.shape))


@functools.lru_cache(maxsize=None)
def clustered_reference():
    x, m, w = clustered_case()
    return oracle.ewald_vjp(x, m, w, 0.005, 1.0)


@pytest.mark.parametrize("prec", [B.FP32, B.FP64])
def test_periodic_force_vjp_clustered_and_unwrapped(prec):
    x, m, w = clustered_case()
    gx, gm = periodic_vjp(x, m, w, 0.005, 1.0, prec, 1.0, 1.0)
    rx, rm = clustered_reference()
    # FP32 positions a few boxes apart round at ~ulp(3)
    tol = 3e-5 if prec == B.FP32 else 1e-9
    assert rel(gx, rx) < tol
    assert rel(gm, rm) < tol


def tracer_loss_grads(xT, vT, m, aT, tr):
    gv = np.zeros_like(vT)
    gv[tr] = aT * aT * m[tr, None] * vT[tr]
    gm = np.zeros_like(m)
    gm[tr] = 0.5 * aT * aT * np.sum(vT[tr] ** 2, axis=1)
    return gv, gm


def adjoint_case():
    # 6^3 bodies at the background density in the unit periodic box
    ic = inputs.perturbed_grid(6, 0.1, 0.02, 4, zeldovich=True,
                               total_mass=inputs.CRITICAL_MATTER_DENSITY)
    return ic, inputs.tracers(ic.N, 64, 7)


@functools.lru_cache(maxsize=None)
def adjoint_reference(n, scheme="kdk"):
    ic, tr = adjoint_case()
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, scheme, box=1.0)
    rgvT, rgmT = tracer_loss_grads(r["x"], r["v"], ic.m, r["schedule"]["a"][-1], tr)
    return oracle.adjoint_run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n,
                              np.zeros_like(ic.x), rgvT, rgmT, scheme=scheme, box=1.0)


@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
@pytest.mark.parametrize("prec,tol", [(B.FP64, 1e-9), (B.FP32, 1e-4), (B.FP32_COMP, 1e-4)])
def test_periodic_adjoint_matches_oracle_transpose(prec, tol, scheme):
    # 12 steps with checkpoints every 5 (uneven segments 5 + 5 + 2)
    ic, tr = adjoint_case()
    n = 12
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=prec,
                       scheme=B.KDK if scheme == "kdk" else B.DKD)
    try:
        sim.set_state(ic.x, ic.v)
        sim.set_periodic(1.0)
        sim.adjoint_forward(TAU, n, 5)
        xT, vT, t, aT = sim.state()
        gvT, gmT = tracer_loss_grads(xT, vT, ic.m, aT, tr)
        gx, gv, gm = sim.adjoint_backward(None, gvT, gmT)
    finally:
        sim.close()
    rx, rv, rm = adjoint_reference(n, scheme)
    assert rel(gx, rx) < tol
    assert rel(gv, rv) < tol
    assert rel(gm, rm) < tol
    # translation invariance holds in a periodic box too
    assert np.all(np.abs(gx.sum(axis=0)) < 10 * tol * np.abs(gx).sum(axis=0))


@pytest.mark.parametrize("prec", [B.FP32, B.FP64])
def test_periodic_force_vjp_degenerate_cases(prec):
    # one body: every pair is the self pair (masked in real space, exactly
    # cancelling in the reciprocal sum); two distinct bodies at one point take
    # the finite d -> 0 limit of the pair Jacobian; a third body elsewhere
    rng = np.random.default_rng(940)
    one_x = inputs.f32(rng.random((1, 3)))
    gx, gm = periodic_vjp(one_x, np.array([0.7]), inputs.f32(rng.standard_normal((1, 3))), 0.02, 1.0,
                          prec, 1.0, 1.0)
    # the reciprocal terms are O(100) each here; they cancel to FP32 / FP64 rounding
    small = 1e-3 if prec == B.FP32 else 1e-9
    assert np.abs(gx).max() < small and np.abs(gm).max() < small
    x = inputs.f32(np.array([[0.3, 0.4, 0.5], [0.3, 0.4, 0.5], [0.8, 0.1, 0.6]]))
    m = inputs.f32(np.array([0.5, 0.25, 1.0]))
    w = inputs.f32(rng.standard_normal((3, 3)))
    gx, gm = periodic_vjp(x, m, w, 0.02, 1.0, prec, 1.0, 1.0)
    rx, rm = oracle.ewald_vjp(x, m, w, 0.02, 1.0)
    tol = 1e-5 if prec == B.FP32 else 1e-10
    assert rel(gx, rx) < tol
    assert rel(gm, rm) < tol
