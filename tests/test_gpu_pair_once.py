"""GPU parity of the pair-once force shape (tile shape 3: every pair evaluated
once and applied to both bodies) against the FP64 oracle.

Shape 3 cuts the bodies into 2048-body tiles and visits the tile pairs
it <= jt; sizes below are on, one off and between tile multiples, so the
diagonal, symmetric and ragged (zero-mass padding) units all occur, with
equal masses (the equal-mass form) and lognormal ones.  Tolerances as in
test_gpu_forces.py: RMS over bodies relative to the mean abs(F), 1e-5 FP32,
1e-6 FP32 compensated.  Above 20000 bodies the oracle evaluates 512 seeded
rows against every source.
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
TOL = {B.FP32: 1e-5, B.FP32_COMP: 1e-6}
SAMPLE_ABOVE = 20000
SHAPE = 3


def rel_rms(a, b):
    return float(np.sqrt(np.mean(np.sum((a - b) ** 2, axis=1))) /
                 np.mean(np.linalg.norm(b, axis=1)))


def system(N, equal, seed):
    rng = np.random.default_rng(seed)
    x = inputs.f32(rng.random((N, 3)))
    m = np.full(N, 1.0 / N) if equal else rng.lognormal(0.0, 0.5, N) / N
    return x, inputs.f32(m)


def forces(x, m, eps, prec, shape=SHAPE, a=1.0, G=1.0):
    sim = B.Simulation(m, eps, LCDM_D, a, prec=prec, G=G)
    try:
        sim.set_state(x)
        sim.set_tuning(shape)
        return sim.forces(), sim.force_plan()
    finally:
        sim.close()


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP])
@pytest.mark.parametrize("equal", [True, False])
@pytest.mark.parametrize("N", [2049, 4096, 6143, 10007, 16384, 24577])
def test_forces_match_oracle(N, equal, prec):
    x, m = system(N, equal, 900 + N)
    eps = 0.002
    got, plan = forces(x, m, eps, prec, a=0.5, G=1.3)
    n = -(-N // 2048)
    assert plan["kind"] == "force_sym_f32" and plan["units"] == n * (n + 1) // 2
    assert plan["eqm"] == (equal and N % 2048 == 0)
    if N > SAMPLE_ABOVE:
        rows = np.sort(np.random.default_rng(N).choice(N, 512, replace=False))
        ref = oracle.forces(x, m, eps, 1.3, rows=rows) / 0.5 ** 3
        got = got[rows]
    else:
        ref = oracle.forces(x, m, eps, 1.3) / 0.5 ** 3
    assert rel_rms(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP])
def test_clustered_bodies(prec):
    ic = inputs.plummer_clusters(30000, 9)
    got, _ = forces(ic.x, ic.m, ic.eps, prec)
    rows = np.sort(np.random.default_rng(3).choice(ic.N, 512, replace=False))
    assert rel_rms(got[rows], oracle.forces(ic.x, ic.m, ic.eps, rows=rows)) < TOL[prec]


def test_antisymmetric_pair_sum_and_momentum():
    # each pair is evaluated once and applied with both signs: sum_k m_k F_k
    # vanishes up to the FP32 rounding of the per-body sums
    x, m = system(8192, False, 5)
    got, _ = forces(x, m, 0.002, B.FP32_COMP)
    p = (m[:, None].astype(np.float64) * got).sum(0)
    scale = (m[:, None].astype(np.float64) * np.abs(got)).sum(0)
    assert np.all(np.abs(p) < 1e-6 * scale)


def test_deterministic_and_close_to_shape_0():
    x, m = system(20000, False, 7)
    a, _ = forces(x, m, 0.002, B.FP32_COMP)
    b, _ = forces(x, m, 0.002, B.FP32_COMP)
    assert np.array_equal(a, b)
    c, p0 = forces(x, m, 0.002, B.FP32_COMP, shape=0)
    assert p0["kind"] == "force_f32"
    assert rel_rms(a, c) < 2e-6


def run_steps(ic, scheme, shape, n):
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32_COMP,
                       scheme=B.KDK if scheme == "kdk" else B.DKD)
    try:
        sim.set_state(ic.x, ic.v)
        sim.set_tuning(shape)
        kind = sim.force_plan()["kind"]
        sim.step(TAU, n)
        xg, vg, t, a = sim.state()
    finally:
        sim.close()
    return kind, xg, vg


@pytest.mark.parametrize("N", [6144, 6143])
@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
def test_steps_match_oracle(scheme, N):
    # a perturbed-grid box at the background matter density with growing-mode
    # velocities, 10 steps (before the dynamics amplify rounding), 3 tiles:
    # equal masses take the equal-mass form at 6144 bodies, the general one
    # (with padding) at 6143.  Positions within 1e-5 of the oracle.  The FP32
    # state's rounding alone (the FP64 context matches the oracle to 1e-14)
    # leaves the DKD velocities about 3e-5 (RMS, relative) from the oracle
    # with either force shape, hence 5e-5 there; the two shapes, which differ
    # only in the order of the pair sums, agree far closer.
    ic = inputs.perturbed_grid(19, 0.1, 0.02, 31, zeldovich=True, count=N,
                               total_mass=inputs.CRITICAL_MATTER_DENSITY)
    n = 10
    kind, xg, vg = run_steps(ic, scheme, SHAPE, n)
    kind0, x0, v0 = run_steps(ic, scheme, 0, n)
    assert kind == "force_sym_f32" and kind0 == "force_f32"
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, scheme)
    assert np.abs(xg - r["x"]).max() < 1e-5
    vn = np.sqrt(np.mean(np.sum(r["v"] ** 2, axis=1)))
    assert np.sqrt(np.mean(np.sum((vg - r["v"]) ** 2, axis=1))) < 5e-5 * vn
    assert np.abs(xg - x0).max() < 1e-6
    assert np.sqrt(np.mean(np.sum((vg - v0) ** 2, axis=1))) < 5e-6 * vn


def test_does_not_fit_one_tile():
    x, m = system(2048, True, 1)
    sim = B.Simulation(m, 0.01, LCDM_D, 1.0, prec=B.FP32)
    try:
        sim.set_state(x)
        with pytest.raises(B.ColatusError):
            sim.set_tuning(SHAPE)
        shape, ms = sim.autotune(1)
        assert shape != SHAPE and ms[SHAPE] == 0.0
    finally:
        sim.close()


def test_default_choice_from_eight_tiles():
    for N, kind in ((14336, "force_f32"), (14337, "force_sym_f32"), (32768, "force_sym_f32")):
        x, m = system(N, True, 2)
        sim = B.Simulation(m, 0.01, LCDM_D, 1.0, prec=B.FP32_COMP)
        try:
            sim.set_state(x)
            assert sim.force_plan()["kind"] == kind, N
        finally:
            sim.close()


# ---- the pair-once equal-mass VJP (the KDK adjoint's kernel from 8 tiles of
# 1024 bodies): gradients against the oracle's exact transpose of the steps

def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def tracer_loss_grads(xT, vT, m, aT, tr):
    """L = 1/2 sum_tracers m a^2 |v|^2 and its gradients at the final state."""
    gv = np.zeros_like(vT)
    gv[tr] = aT * aT * m[tr, None] * vT[tr]
    gm = np.zeros_like(m)
    gm[tr] = 0.5 * aT * aT * np.sum(vT[tr] ** 2, axis=1)
    return gv, gm


def adjoint_pair(ic, prec, n, k, tr):
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=prec)
    try:
        sim.set_state(ic.x, ic.v)
        plan = sim.vjp_plan()
        sim.adjoint_forward(TAU, n, k)
        xT, vT, t, aT = sim.state()
        gvT, gmT = tracer_loss_grads(xT, vT, ic.m, aT, tr)
        g = sim.adjoint_backward(None, gvT, gmT)
    finally:
        sim.close()
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "kdk")
    gvO, gmO = tracer_loss_grads(r["x"], r["v"], ic.m, r["schedule"]["a"][-1], tr)
    gx, gv, gm = oracle.adjoint_run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n,
                                    np.zeros_like(ic.x), gvO, gmO, scheme="kdk")
    return plan, g, dict(gx=gx, gv=gv, gm=gm)


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP])
@pytest.mark.parametrize("k", [3, 1])
def test_equal_mass_adjoint_pair_once_vjp(prec, k):
    # 8192 equal-mass bodies at the background density (8 tiles of 1024), 8
    # KDK steps; checkpoints every 3 (segments 3 + 3 + 2) or every step
    ic = inputs.perturbed_grid(21, 0.1, 0.02, 41, zeldovich=True, count=8192,
                               total_mass=inputs.CRITICAL_MATTER_DENSITY)
    tr = inputs.tracers(ic.N, 64, 7)
    plan, g, ref = adjoint_pair(ic, prec, 8, k, tr)
    assert plan["kind"] == "vjp_sym_eqm_f32" and plan["units"] == 8 * 9 // 2
    for key, got in zip(("gx", "gv", "gm"), g):
        assert rel(got, ref[key]) < 1e-4, key


def test_grid32_adjoint_pair_once_vjp():
    # the adjoint configuration's workload (32^3, the benchmark's kernel and
    # launch plan) over two steps, checkpoints every step
    ic = inputs.grid32()
    tr = inputs.tracers(ic.N, 64, 7)
    plan, g, ref = adjoint_pair(ic, B.FP32_COMP, 2, 1, tr)
    assert plan["kind"] == "vjp_sym_eqm_f32" and plan["units"] == 32 * 33 // 2
    for key, got in zip(("gx", "gv", "gm"), g):
        assert rel(got, ref[key]) < 1e-4, key


def test_vjp_plan_kinds():
    # from 8 tiles of 1024 bodies: the equal-mass pair-once VJP for the KDK
    # adjoint with equal masses, the pair-once VJP for any masses otherwise
    # (DKD, unequal masses); below 8 tiles the per-ordered-pair kernels;
    # FP64 its own kernel
    x, m = system(8192, True, 3)
    cases = [(dict(), "vjp_sym_eqm_f32"), (dict(scheme=B.DKD), "vjp_sym_f32"),
             (dict(prec=B.FP64), "vjp_f64")]
    for kw, kind in cases:
        sim = B.Simulation(m, 0.01, LCDM_D, 1.0, **{"prec": B.FP32, **kw})
        try:
            sim.set_state(x)
            assert sim.vjp_plan()["kind"] == kind, kw
        finally:
            sim.close()
    for N, mm, kind in ((7168, np.full(7168, 1 / 7168), "vjp_eqm_f32"),
                        (7168, system(7168, False, 4)[1], "vjp_f32"),
                        (8192, system(8192, False, 4)[1], "vjp_sym_f32"),
                        (8193, system(8193, False, 4)[1], "vjp_sym_f32")):
        sim = B.Simulation(inputs.f32(mm), 0.01, LCDM_D, 1.0, prec=B.FP32)
        try:
            sim.set_state(system(N, True, 5)[0])
            assert sim.vjp_plan()["kind"] == kind, N
        finally:
            sim.close()


# ---- the pair-once real-space kernel under periodic boundaries (Ewald
# summation; 1024-body tiles, the built-in choice from 8 tiles on)

def periodic_forces(x, m, eps, L, prec, shape=-1, a=1.0, G=1.0):
    sim = B.Simulation(m, eps, LCDM_D, a, prec=prec, G=G)
    try:
        sim.set_state(x)
        sim.set_tuning(shape)
        sim.set_periodic(L)
        return sim.forces(), sim.force_plan()
    finally:
        sim.close()


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP])
@pytest.mark.parametrize("N,equal", [(8192, True), (8192, False), (9001, False)])
def test_periodic_pair_once_forces_match_oracle(N, equal, prec):
    rng = np.random.default_rng(950 + N)
    L = 2.5
    x = inputs.f32(L * rng.random((N, 3)))
    m = inputs.f32(np.full(N, 1.0 / N) if equal else rng.lognormal(0.0, 0.5, N) / N)
    eps, a, G = 0.01, 0.5, 1.3
    got, plan = periodic_forces(x, m, eps, L, prec, a=a, G=G)
    n = -(-N // 1024)
    assert plan["kind"] == "ewald_sym_f32" and plan["units"] == n * (n + 1) // 2
    assert plan["eqm"] == (equal and N % 1024 == 0)
    rows = np.sort(np.random.default_rng(N).choice(N, 512, replace=False))
    ref = oracle.ewald_forces(x, m, eps, L, G, rows=rows) / a ** 3
    # the FP32 real-space term carries the error of its erfc (Abramowitz &
    # Stegun 7.1.26, 1.5e-7 absolute), which compensated sums do not remove:
    # at 9001 lognormal bodies both real-space forms measure 2.6e-6 against
    # the converged FP64 sum (FP64 1e-14), so the oracle bound is 5e-6 in
    # both FP32 modes here; the two forms must agree far closer
    assert rel_rms(got[rows], ref) < 5e-6
    got0, plan0 = periodic_forces(x, m, eps, L, prec, shape=2, a=a, G=G)   # any shape but 3
    assert plan0["kind"] == "ewald_f32"
    assert rel_rms(got, got0) < (2e-6 if prec == B.FP32 else 5e-7)


@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
def test_periodic_pair_once_steps_match_per_pair_kernel(scheme):
    # 8192 bodies of the 32^3 recipe in a periodic unit box, 6 steps with
    # either real-space form: the two differ only in the order of the pair sums
    ic = inputs.perturbed_grid(21, 0.1, 0.02, 43, zeldovich=True, count=8192,
                               total_mass=inputs.CRITICAL_MATTER_DENSITY)
    out = []
    for shape in (3, 2):   # any shape but 3 takes the per-ordered-pair kernel
        sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32_COMP,
                           scheme=B.KDK if scheme == "kdk" else B.DKD)
        try:
            sim.set_state(ic.x, ic.v)
            sim.set_tuning(shape)
            sim.set_periodic(1.0)
            kind = sim.force_plan()["kind"]
            sim.step(TAU, 6)
            out.append((kind,) + tuple(sim.state()[:2]))
        finally:
            sim.close()
    (k3, x3, v3), (k0, x0, v0) = out
    assert k3 == "ewald_sym_f32" and k0 == "ewald_f32"
    assert np.abs(x3 - x0).max() < 1e-6
    vn = np.sqrt(np.mean(np.sum(v0 ** 2, axis=1)))
    assert np.sqrt(np.mean(np.sum((v3 - v0) ** 2, axis=1))) < 5e-6 * vn


# ---- the pair-once VJP for any masses (colatus_force_vjp and the DKD adjoint
# from 8 tiles of 1024 bodies)

def vjp_system(N, seed, equal=False):
    rng = np.random.default_rng(seed)
    x = inputs.f32(rng.random((N, 3)))
    m = np.full(N, 1.0 / N) if equal else rng.lognormal(0.0, 0.5, N) / N
    w = inputs.f32(rng.standard_normal((N, 3)))
    return x, inputs.f32(m), w


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP])
@pytest.mark.parametrize("N,equal", [(8192, False), (8192, True), (9001, False), (20481, False)])
def test_force_vjp_pair_once_matches_oracle(N, equal, prec):
    x, m, w = vjp_system(N, 340 + N, equal)
    a, G, eps = 0.5, 1.3, 0.002
    sim = B.Simulation(m, eps, LCDM_D, a, prec=prec, G=G)
    try:
        sim.set_state(x)
        assert sim.vjp_plan()["kind"] == ("vjp_sym_eqm_f32" if equal and N % 1024 == 0 else "vjp_sym_f32")
        gx, gm = sim.force_vjp(w)
    finally:
        sim.close()
    rows = None if N <= SAMPLE_ABOVE else np.sort(np.random.default_rng(N).choice(N, 512, replace=False))
    rx, rm = oracle.vjp(x, m, w, eps, G, rows=rows)
    sel = slice(None) if rows is None else rows
    assert rel(gx[sel], rx / a ** 3) < 1e-5
    assert rel(gm[sel], rm / a ** 3) < 1e-5


@pytest.mark.parametrize("N", [8192, 9001])
def test_force_vjp_pair_once_uniform_covector_position_term_is_exactly_zero(N):
    # equal masses and one co-vector for every body: u' = m_i w_j - m_j w_i = 0
    # for every pair, so dL/dx is 0 in exact arithmetic.  The pair-once form
    # computes u' from the co-vector difference, so it returns exactly 0: at
    # 8192 in the equal-mass form, at 9001 in the form for any masses, where
    # the 215 padding bodies (zero mass and co-vector) must add exactly 0 too.
    # dL/dm = -sum_j inv^3 (w . d) does not vanish and is checked as usual.
    x, m, _ = vjp_system(N, 370 + N, equal=True)
    w = np.tile(inputs.f32(np.array([[0.3, -1.2, 0.7]])), (N, 1))
    a, G, eps = 0.5, 1.3, 0.002
    sim = B.Simulation(m, eps, LCDM_D, a, prec=B.FP32, G=G)
    try:
        sim.set_state(x)
        gx, gm = sim.force_vjp(w)
    finally:
        sim.close()
    assert np.count_nonzero(gx) == 0
    _, rm = oracle.vjp(x, m, w, eps, G)
    assert rel(gm, rm / a ** 3) < 1e-5


@pytest.mark.parametrize("case", ["massless", "tiny", "huge", "zero_covector", "coincident"])
def test_force_vjp_pair_once_mass_edge_cases(case):
    # massless bodies with co-vectors, masses of 1e-25 and of 3e11 / 3e21,
    # zero co-vectors, and distinct bodies at one point (inv = 1/eps there)
    N = 9000
    x, m, w = vjp_system(N, 360)
    m = m.astype(np.float64)
    G = 1.3
    if case == "massless":
        m[[1500, 2500, 8999]] = 0.0
    elif case == "tiny":
        m[[1200, 4600]] = 1e-25
    elif case == "huge":
        m *= 1e15
        m[4096:] *= 1e10
        G = 1.3e-20
    elif case == "zero_covector":
        w[1000:5100] = 0.0
        m[2000:2050] = 0.0
    else:
        x[[10, 3000, 8000]] = x[5]
    m = inputs.f32(m)
    a, eps = 0.5, 0.01
    sim = B.Simulation(m, eps, LCDM_D, a, prec=B.FP32, G=G)
    try:
        sim.set_state(x)
        assert sim.vjp_plan()["kind"] == "vjp_sym_f32"
        gx, gm = sim.force_vjp(w)
    finally:
        sim.close()
    rx, rm = oracle.vjp(x, m, w, eps, G)
    assert rel(gx, rx / a ** 3) < 1e-5
    assert rel(gm, rm / a ** 3) < 1e-5


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP])
@pytest.mark.parametrize("k", [3, 1])
def test_dkd_adjoint_pair_once_vjp(prec, k):
    # the paper's DKD scheme takes the VJP for any masses: 8192 bodies at the
    # background density, 8 steps, against the oracle's DKD transpose
    ic = inputs.perturbed_grid(21, 0.1, 0.02, 47, zeldovich=True, count=8192,
                               total_mass=inputs.CRITICAL_MATTER_DENSITY)
    tr = inputs.tracers(ic.N, 64, 7)
    n = 8
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=prec, scheme=B.DKD)
    try:
        sim.set_state(ic.x, ic.v)
        assert sim.vjp_plan()["kind"] == "vjp_sym_f32"
        sim.adjoint_forward(TAU, n, k)
        xT, vT, t, aT = sim.state()
        gvT, gmT = tracer_loss_grads(xT, vT, ic.m, aT, tr)
        g = sim.adjoint_backward(None, gvT, gmT)
    finally:
        sim.close()
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "dkd")
    gvO, gmO = tracer_loss_grads(r["x"], r["v"], ic.m, r["schedule"]["a"][-1], tr)
    ref = oracle.adjoint_run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n,
                             np.zeros_like(ic.x), gvO, gmO, scheme="dkd")
    for key, got, want in zip(("gx", "gv", "gm"), g, ref):
        assert rel(got, want) < 1e-4, key


# ---- the pair-once VJP under periodic boundaries (the real-space term of the
# Ewald sum as its pair policy: minimum image, then b and c of the erfc form;
# from 8 tiles of 1024 bodies)

def periodic_force_vjp(x, m, w, eps, L, prec, shape=-1, a=1.0, G=1.0):
    sim = B.Simulation(m, eps, LCDM_D, a, prec=prec, G=G)
    try:
        sim.set_state(x)
        sim.set_tuning(shape)
        sim.set_periodic(L)
        gx, gm = sim.force_vjp(w)
        return gx, gm, sim.vjp_plan()["kind"]
    finally:
        sim.close()


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP])
@pytest.mark.parametrize("N,equal", [(8192, True), (8192, False), (9001, False)])
def test_periodic_force_vjp_pair_once_matches_oracle(N, equal, prec):
    rng = np.random.default_rng(960 + N)
    L = 2.5
    x = inputs.f32(L * rng.random((N, 3)))
    m = inputs.f32(np.full(N, 1.0 / N) if equal else rng.lognormal(0.0, 0.5, N) / N)
    w = inputs.f32(rng.standard_normal((N, 3)))
    eps, a, G = 0.01, 0.5, 1.3
    gx, gm, kind = periodic_force_vjp(x, m, w, eps, L, prec, a=a, G=G)
    assert kind == "ewald_vjp_sym_f32"
    rows = np.sort(np.random.default_rng(N + 1).choice(N, 512, replace=False))
    rx, rm = oracle.ewald_vjp(x, m, w, eps, L, G, rows=rows)
    s = 1.0 / a ** 3
    ex, em = rel(gx[rows], s * rx), rel(gm[rows], s * rm)
    assert ex < 1e-5 and em < 1e-5, (ex, em)
    # the per-ordered-pair real-space VJP (any tuning shape but 3): the two
    # differ in the order of the pair sums and in how u' rounds
    gx0, gm0, kind0 = periodic_force_vjp(x, m, w, eps, L, prec, shape=2, a=a, G=G)
    assert kind0 == "ewald_vjp_f32"
    dx, dm = rel(gx, gx0), rel(gm, gm0)
    assert dx < 5e-6 and dm < 5e-6, (dx, dm)


def test_periodic_vjp_plan_kinds():
    x, m = system(8192, False, 6)
    for kw, shape, kind in ((dict(), -1, "ewald_vjp_sym_f32"), (dict(scheme=B.DKD), 3, "ewald_vjp_sym_f32"),
                            (dict(), 0, "ewald_vjp_f32"), (dict(prec=B.FP64), -1, "ewald_vjp_f64")):
        sim = B.Simulation(m, 0.01, LCDM_D, 1.0, **{"prec": B.FP32, **kw})
        try:
            sim.set_state(x)
            sim.set_tuning(shape)
            sim.set_periodic(1.0)
            assert sim.vjp_plan()["kind"] == kind, (kw, shape)
        finally:
            sim.close()
    x, m = system(7168, False, 6)   # 7 tiles
    sim = B.Simulation(m, 0.01, LCDM_D, 1.0, prec=B.FP32)
    try:
        sim.set_state(x)
        sim.set_periodic(1.0)
        assert sim.vjp_plan()["kind"] == "ewald_vjp_f32"
    finally:
        sim.close()


@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
def test_periodic_adjoint_pair_once_matches_per_pair_kernel(scheme):
    # 8192 bodies of the 32^3 recipe in the periodic unit box, 6 steps with
    # checkpoints every 4, then the adjoint of a tracer loss: with the
    # pair-once real-space force and VJP against the per-ordered-pair ones
    # (both are checked against the oracle above and in the periodic tests)
    ic = inputs.perturbed_grid(21, 0.1, 0.02, 43, zeldovich=True, count=8192,
                               total_mass=inputs.CRITICAL_MATTER_DENSITY)
    tr = inputs.tracers(ic.N, 64, 7)
    out = []
    for shape in (3, 2):
        sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32_COMP,
                           scheme=B.KDK if scheme == "kdk" else B.DKD)
        try:
            sim.set_state(ic.x, ic.v)
            sim.set_tuning(shape)
            sim.set_periodic(1.0)
            kind = sim.vjp_plan()["kind"]
            sim.adjoint_forward(TAU, 6, 4)
            xT, vT, t, aT = sim.state()
            gvT, gmT = tracer_loss_grads(xT, vT, ic.m, aT, tr)
            out.append((kind,) + tuple(sim.adjoint_backward(None, gvT, gmT)))
        finally:
            sim.close()
    (k3, *g3), (k2, *g2) = out
    assert k3 == "ewald_vjp_sym_f32" and k2 == "ewald_vjp_f32"
    for key, a, b in zip(("gx", "gv", "gm"), g3, g2):
        e = rel(a, b)
        assert e < 2e-5, (key, e)
