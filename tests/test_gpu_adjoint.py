"""GPU parity of the hand-written derivative kernels.

* the force VJP (gradient of sum w . acc with respect to positions and
  masses) against the oracle's FP64 VJP;
* the checkpointed discrete adjoint of the KDK and DKD leapfrogs against the oracle's
  exact FP64 transpose and against central finite differences;
* the torch.autograd wrappers.

Tolerances: normwise relative error of the gradient vector; FP32 VJP 1e-5,
FP64 1e-10; FP32 trajectory adjoint 1e-4 (the stated target for gradients),
FP64 1e-9.

Conditioning: the tracer kinetic-energy gradient of the 8^3 workload is
well conditioned for ~20 steps (a 6e-8 change of the initial positions moves
it by 1e-6), but chaotic by 100-200 steps (the same change moves it by O(1) at
100 steps; a 1e-15 change moves it by 5e-3 at 200 steps).  Element-wise
gradient parity is therefore checked over 20 steps; the 200-step pass is
checked through exact symmetries of the discrete map that chaos does not
amplify: translation invariance (sum_i dL/dx0_i = 0 for a loss of the final
velocities) and the Galilean boost (sum_i dL/dv0_i = prod(c1 c2) sum_i dL/dvT_i).
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


def random_system(N, seed):
    rng = np.random.default_rng(seed)
    x = inputs.f32(rng.random((N, 3)))
    m = inputs.f32(rng.lognormal(0.0, 0.5, N) / N)
    w = inputs.f32(rng.standard_normal((N, 3)))
    return x, m, w


@pytest.mark.parametrize("prec,tol", [(B.FP32, 1e-5), (B.FP64, 1e-10)])
@pytest.mark.parametrize("N", [1, 5, 257, 3000])
def test_force_vjp_matches_oracle(N, prec, tol):
    x, m, w = random_system(N, 300 + N)
    a, G, eps = 0.5, 1.3, 0.01
    sim = B.Simulation(m, eps, LCDM_D, a, prec=prec, G=G)
    try:
        sim.set_state(x)
        gx, gm = sim.force_vjp(w)
    finally:
        sim.close()
    rx, rm = oracle.vjp(x, m, w, eps, G)
    scale = 1.0 / a ** 3
    if N == 1:
        assert np.all(gx == 0) and np.all(gm == 0)
        return
    assert rel(gx, scale * rx) < tol
    assert rel(gm, scale * rm) < tol


@pytest.mark.parametrize("case", ["massless", "tiny", "huge", "zero_covector"])
def test_force_vjp_mass_edge_cases(case):
    # The FP32 VJP takes a shorter form (co-vector divided by the mass) in
    # blocks of bodies whose masses and scaled co-vectors are of moderate
    # size, and the general form elsewhere.  These inputs mix both within one
    # call: a massless body with a co-vector, masses of 1e-25 or 1e25, and
    # bodies whose co-vector is zero.
    N = 3000
    x, m, w = random_system(N, 320)
    m = m.astype(np.float64)
    G = 1.3
    if case == "massless":
        m[[1500, 2500, 2999]] = 0.0
    elif case == "tiny":
        m[[1200, 2600]] = 1e-25
    elif case == "huge":            # ~3e11: the short form; ~3e21: the general one
        m *= 1e15
        m[2048:] *= 1e10
        G = 1.3e-20
    else:
        w[1000:2100] = 0.0
        m[2000:2050] = 0.0
    m = inputs.f32(m)
    a, eps = 0.5, 0.01
    sim = B.Simulation(m, eps, LCDM_D, a, prec=B.FP32, G=G)
    try:
        sim.set_state(x)
        gx, gm = sim.force_vjp(w)
    finally:
        sim.close()
    rx, rm = oracle.vjp(x, m, w, eps, G)
    assert rel(gx, rx / a ** 3) < 1e-5
    assert rel(gm, rm / a ** 3) < 1e-5


def tracer_loss_grads(xT, vT, m, aT, tr):
    """L = 1/2 sum_tracers m a^2 |v|^2 and its gradients at the final state."""
    gv = np.zeros_like(vT)
    gv[tr] = aT * aT * m[tr, None] * vT[tr]
    gm = np.zeros_like(m)
    gm[tr] = 0.5 * aT * aT * np.sum(vT[tr] ** 2, axis=1)
    L = 0.5 * aT * aT * float(np.sum(m[tr] * np.sum(vT[tr] ** 2, axis=1)))
    return L, gv, gm


def gpu_adjoint(ic, prec, nsteps, k, tr):
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=prec)
    try:
        sim.set_state(ic.x, ic.v)
        sim.adjoint_forward(TAU, nsteps, k)
        xT, vT, t, aT = sim.state()
        L, gvT, gmT = tracer_loss_grads(xT, vT, ic.m, aT, tr)
        gx, gv, gm = sim.adjoint_backward(None, gvT, gmT)
        return dict(L=L, gx=gx, gv=gv, gm=gm, xT=xT, vT=vT, aT=aT)
    finally:
        sim.close()


def oracle_adjoint(ic, nsteps, tr):
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, nsteps, "kdk")
    aT = r["schedule"]["a"][-1]
    L, gvT, gmT = tracer_loss_grads(r["x"], r["v"], ic.m, aT, tr)
    gx, gv, gm = oracle.adjoint_run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, nsteps,
                                    np.zeros_like(ic.x), gvT, gmT, scheme="kdk")
    return dict(L=L, gx=gx, gv=gv, gm=gm)


def test_fp64_adjoint_matches_oracle_transpose():
    ic = inputs.perturbed_grid(8, 0.1, 0.02, 4, zeldovich=True, total_mass=inputs.CRITICAL_MATTER_DENSITY)
    tr = inputs.tracers(ic.N, 64, 7)
    g = gpu_adjoint(ic, B.FP64, 20, 7, tr)     # uneven segments: 7 + 7 + 6
    r = oracle_adjoint(ic, 20, tr)
    for k in ("gx", "gv", "gm"):
        assert rel(g[k], r[k]) < 1e-9, k


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP])
def test_fp32_adjoint_matches_oracle_over_the_conditioned_horizon(prec):
    # 8^3 bodies at the background density, 20 KDK steps, checkpoints every 5
    ic = inputs.perturbed_grid(8, 0.1, 0.02, 4, zeldovich=True, total_mass=inputs.CRITICAL_MATTER_DENSITY)
    tr = inputs.tracers(ic.N, 64, 7)
    g = gpu_adjoint(ic, prec, 20, 5, tr)
    r = oracle_adjoint(ic, 20, tr)
    for k in ("gx", "gv", "gm"):
        assert rel(g[k], r[k]) < 1e-4, k


@pytest.mark.parametrize("prec", [B.FP32, B.FP64])
def test_200_step_adjoint_satisfies_translation_and_boost_identities(prec):
    # the adjoint-sensitivity workload: 8^3 bodies (the 32^3 recipe), 200 KDK
    # steps, checkpoints every 20, loss = tracer kinetic energy
    ic = inputs.grid8()
    tr = inputs.tracers(ic.N, 64, 7)
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=prec)
    try:
        sim.set_state(ic.x, ic.v)
        sim.adjoint_forward(TAU, 200, 20)
        xT, vT, t, aT = sim.state()
        L, gvT, gmT = tracer_loss_grads(xT, vT, ic.m, aT, tr)
        gx, gv, gm = sim.adjoint_backward(None, gvT, gmT)
    finally:
        sim.close()
    assert np.all(np.isfinite(gx)) and np.all(np.isfinite(gv)) and np.all(np.isfinite(gm))
    tol = 1e-4 if prec == B.FP32 else 1e-10
    # translation: a uniform shift of the initial positions leaves v_T unchanged
    assert np.all(np.abs(gx.sum(axis=0)) < tol * np.abs(gx).sum(axis=0))
    # boost: a uniform initial velocity u becomes prod(c1 c2) u at the end
    sch = oracle.schedule(LCDM, inputs.A_START, TAU, 200, "kdk")
    P = float(np.prod(sch["c1"] * sch["c2"]))
    np.testing.assert_allclose(gv.sum(axis=0), P * gvT.sum(axis=0), rtol=tol,
                               atol=tol * np.abs(gv).sum(axis=0).max())


def test_fp64_adjoint_directional_derivative_matches_finite_differences():
    ic = inputs.perturbed_grid(8, 0.1, 0.02, 4, zeldovich=True, total_mass=inputs.CRITICAL_MATTER_DENSITY)
    tr = inputs.tracers(ic.N, 64, 7)
    n = 30
    g = gpu_adjoint(ic, B.FP64, n, 8, tr)
    rng = np.random.default_rng(9)
    dx, dv = rng.standard_normal(ic.x.shape), rng.standard_normal(ic.v.shape)
    # the loss is strongly nonlinear: the central difference converges as h^2
    # (3e-5 at h = 1e-6, 7e-9 at h = 1e-8 in the oracle), so h = 1e-8
    h = 1e-8

    def loss(x, v):
        sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP64)
        try:
            sim.set_state(x, v)
            sim.step(TAU, n)
            xT, vT, t, aT = sim.state()
        finally:
            sim.close()
        return tracer_loss_grads(xT, vT, ic.m, aT, tr)[0]

    fd = (loss(ic.x + h * dx, ic.v + h * dv) - loss(ic.x - h * dx, ic.v - h * dv)) / (2 * h)
    ad = float(np.sum(g["gx"] * dx) + np.sum(g["gv"] * dv))
    assert ad == pytest.approx(fd, rel=1e-6)


def test_adjoint_state_checks():
    ic = inputs.grid8()
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32)
    try:
        sim.set_state(ic.x, ic.v)
        with pytest.raises(B.ColatusError) as e:
            sim.adjoint_backward(None, np.ones_like(ic.v))
        assert e.value.status == B.E_STATE
        sim.adjoint_forward(TAU, 4, 2)
        sim.step(TAU, 1)
        with pytest.raises(B.ColatusError) as e:
            sim.adjoint_backward(None, np.ones_like(ic.v))
        assert e.value.status == B.E_STATE
        # the recorded pass is replayed with its own scheme and G: a change of
        # either is refused
        sim.adjoint_forward(TAU, 4, 2)
        sim.configure(scheme=B.DKD)
        with pytest.raises(B.ColatusError) as e:
            sim.adjoint_backward(None, np.ones_like(ic.v))
        assert e.value.status == B.E_STATE
        sim.configure(scheme=B.KDK, G=2.0)
        with pytest.raises(B.ColatusError) as e:
            sim.adjoint_backward(None, np.ones_like(ic.v))
        assert e.value.status == B.E_STATE
        sim.configure(G=1.0)
        gx, gv, gm = sim.adjoint_backward(None, np.ones_like(ic.v))
        assert np.all(np.isfinite(gx)) and np.all(np.isfinite(gv))
    finally:
        sim.close()


def test_autograd_force_and_trajectory():
    import torch
    from paper_1208_3444_b300.autograd import AllPairsForce, Trajectory
    x, m, w = random_system(700, 5)
    sim = B.Simulation(m, 0.02, LCDM_D, 0.7, prec=B.FP64)
    try:
        xt = torch.tensor(x, device="cuda", requires_grad=True)
        mt = torch.tensor(m, device="cuda", requires_grad=True)
        acc = AllPairsForce.apply(xt, mt, sim)
        (acc * torch.tensor(w, device="cuda")).sum().backward()
        rx, rm = oracle.vjp(x, m, w, 0.02, 1.0)
        assert rel(xt.grad.cpu().numpy(), rx / 0.7 ** 3) < 1e-10
        assert rel(mt.grad.cpu().numpy(), rm / 0.7 ** 3) < 1e-10
    finally:
        sim.close()
    ic = inputs.perturbed_grid(8, 0.1, 0.02, 4, zeldovich=True, total_mass=inputs.CRITICAL_MATTER_DENSITY)
    tr = inputs.tracers(ic.N, 64, 7)
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP64)
    try:
        x0 = torch.tensor(ic.x, device="cuda", requires_grad=True)
        v0 = torch.tensor(ic.v, device="cuda", requires_grad=True)
        mt = torch.tensor(ic.m, device="cuda", requires_grad=True)
        xT, vT = Trajectory.apply(x0, v0, mt, sim, TAU, 12, 5)
        aT = sim.state()[3]
        idx = torch.tensor(tr, device="cuda")
        L = 0.5 * aT * aT * (mt[idx] * (vT[idx] ** 2).sum(1)).sum()
        L.backward()
    finally:
        sim.close()
    r = oracle_adjoint(ic, 12, tr)
    assert rel(x0.grad.cpu().numpy(), r["gx"]) < 1e-9
    assert rel(v0.grad.cpu().numpy(), r["gv"]) < 1e-9
    assert rel(mt.grad.cpu().numpy(), r["gm"]) < 1e-9


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP])
@pytest.mark.parametrize("k", [5, 1])
def test_equal_mass_adjoint_matches_oracle_transpose(prec, k):
    # 16^3 equal masses at the background density: no padding enters the
    # VJP's 1024-body tiles, so the backward pass takes the equal-mass VJP,
    # whose mass gradient uses the forces the recompute keeps per position.
    # 12 steps; checkpoints every 5 (segments 5 + 5 + 2) or every step.
    ic = inputs.grid16(critical=True)
    tr = inputs.tracers(ic.N, 64, 7)
    n = 12
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=prec)
    try:
        sim.set_state(ic.x, ic.v)
        sim.adjoint_forward(TAU, n, k)
        xT, vT, t, aT = sim.state()
        L, gvT, gmT = tracer_loss_grads(xT, vT, ic.m, aT, tr)
        gx, gv, gm = sim.adjoint_backward(None, gvT, gmT)
    finally:
        sim.close()
    r = oracle_adjoint(ic, n, tr)
    for key, g in (("gx", gx), ("gv", gv), ("gm", gm)):
        assert rel(g, r[key]) < 1e-4, key


def _dkd_case():
    ic = inputs.perturbed_grid(8, 0.1, 0.02, 4, zeldovich=True, total_mass=inputs.CRITICAL_MATTER_DENSITY)
    return ic, inputs.tracers(ic.N, 64, 7)


@pytest.mark.parametrize("prec,tol", [(B.FP64, 1e-9), (B.FP32, 1e-4), (B.FP32_COMP, 1e-4)])
@pytest.mark.parametrize("k,n", [(5, 12), (1, 6)])
def test_dkd_adjoint_matches_oracle_transpose(prec, tol, k, n):
    # the paper's own drift-kick-drift leapfrog (Eqs. 3-5): one VJP per step
    # at the half-drift position; checkpoints every 5 (5 + 5 + 2) or every step
    ic, tr = _dkd_case()
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=prec, scheme=B.DKD)
    try:
        sim.set_state(ic.x, ic.v)
        sim.adjoint_forward(TAU, n, k)
        xT, vT, t, aT = sim.state()
        L, gvT, gmT = tracer_loss_grads(xT, vT, ic.m, aT, tr)
        gx, gv, gm = sim.adjoint_backward(None, gvT, gmT)
    finally:
        sim.close()
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "dkd")
    _, rgvT, rgmT = tracer_loss_grads(r["x"], r["v"], ic.m, r["schedule"]["a"][-1], tr)
    rx, rv, rm = oracle.adjoint_run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n,
                                    np.zeros_like(ic.x), rgvT, rgmT, scheme="dkd")
    assert rel(gx, rx) < tol
    assert rel(gv, rv) < tol
    assert rel(gm, rm) < tol


def test_dkd_adjoint_directional_derivative_matches_finite_differences():
    # FP64, 8 DKD steps: <dL/dx0, dx> + <dL/dv0, dv> against central
    # differences of the GPU's own forward runs
    ic, tr = _dkd_case()
    n = 8
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP64, scheme=B.DKD)
    try:
        sim.set_state(ic.x, ic.v)
        sim.adjoint_forward(TAU, n, 3)
        xT, vT, t, aT = sim.state()
        L, gvT, gmT = tracer_loss_grads(xT, vT, ic.m, aT, tr)
        gx, gv, gm = sim.adjoint_backward(None, gvT, gmT)
    finally:
        sim.close()
    rng = np.random.default_rng(19)
    dx, dv = rng.standard_normal(ic.x.shape), rng.standard_normal(ic.v.shape)
    h = 1e-7

    def loss(x, v):
        s = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP64, scheme=B.DKD)
        try:
            s.set_state(x, v)
            s.step(TAU, n)
            x1, v1, _, a1 = s.state()
        finally:
            s.close()
        return tracer_loss_grads(x1, v1, ic.m, a1, tr)[0]

    fd = (loss(ic.x + h * dx, ic.v + h * dv) - loss(ic.x - h * dx, ic.v - h * dv)) / (2 * h)
    ad = float(np.sum(gx * dx) + np.sum(gv * dv))
    assert ad == pytest.approx(fd, rel=1e-6)
