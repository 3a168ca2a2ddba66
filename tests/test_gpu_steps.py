"""GPU parity of the leapfrog with Hubble drag (Eqs. 3-5, KDK) and the FP64
Friedmann schedule (Eq. 2) against the FP64 oracle.

Positions are compared element by element (maximum over bodies <= 1e-5 box
units in FP32, 1e-9 in FP64) for as long as the dynamics do not amplify
rounding: 10 steps for boxes at the background (critical) matter density, and
the steps before collapse for the m = 1/N boxes (3 for 16^3, 2 for 32^3 with its
infall velocities), which are ~28x overdense and collapse within a few steps (the FP64 oracle itself then amplifies a 6e-8
perturbation to 1e-3; see tests/test_oracle_chaos.py).  Beyond that, exact
discrete invariants apply.
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
POS_TOL = {B.FP32: 1e-5, B.FP32_COMP: 1e-5, B.FP64: 1e-9}
# Velocities: RMS over bodies relative to RMS |v|, and the worst body relative
# to max |v|.  A body in a close encounter (separation ~ eps) receives kicks of
# ~10^3 whose relative accuracy is limited by the float32 positions
# (ulp / eps ~ 1e-4), hence the looser worst-body bound in FP32.
VEL_RMS_TOL = {B.FP32: 1e-5, B.FP32_COMP: 1e-5, B.FP64: 1e-11}
VEL_MAX_TOL = {B.FP32: 1e-3, B.FP32_COMP: 1e-3, B.FP64: 1e-9}
PRE_COLLAPSE = {"grid16": 3, "grid32": 2}
SCHEME = {"kdk": B.KDK, "dkd": B.DKD}


def run_gpu(ic, prec, scheme, nsteps, tracers=None, chunks=None, a_start=inputs.A_START, G=1.0,
            cosmo=LCDM_D, tau=TAU):
    sim = B.Simulation(ic.m, ic.eps, cosmo, a_start, prec=prec, scheme=SCHEME[scheme], G=G)
    try:
        sim.set_state(ic.x, ic.v)
        if tracers is not None:
            sim.record_tracers(tracers, nsteps)
        for n in (chunks or [nsteps]):
            sim.step(tau, n)
        x, v, t, a = sim.state()
        rec = sim.read_tracers() if tracers is not None else None
        diag = sim.diagnostics()
        return dict(x=x, v=v, t=t, a=a, tracers=rec, diag=diag, stats=sim.stats())
    finally:
        sim.close()


def check_state(g, r, prec, n):
    assert np.abs(g["x"] - r["x"]).max() < POS_TOL[prec]
    dv = np.linalg.norm(g["v"] - r["v"], axis=1)
    vn = np.linalg.norm(r["v"], axis=1)
    assert np.sqrt(np.mean(dv ** 2)) < VEL_RMS_TOL[prec] * np.sqrt(np.mean(vn ** 2))
    assert dv.max() < VEL_MAX_TOL[prec] * vn.max()
    assert g["a"] == pytest.approx(r["schedule"]["a"][-1], rel=1e-13)
    assert g["t"] == pytest.approx(n * TAU, rel=1e-13)


@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP, B.FP64])
def test_grid16_ten_steps_critical_density(prec, scheme):
    ic = inputs.grid16(critical=True)
    n = 10
    g = run_gpu(ic, prec, scheme, n)
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, scheme)
    check_state(g, r, prec, n)


@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP, B.FP64])
def test_grid16_before_collapse(prec, scheme):
    ic = inputs.grid16()
    n = PRE_COLLAPSE["grid16"]
    g = run_gpu(ic, prec, scheme, n)
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, scheme)
    check_state(g, r, prec, n)


def test_grid16_twenty_steps_fp64():
    # the oracle-checkable workload: 16^3 bodies, 20 KDK steps in FP64; the
    # collapse after step 4 multiplies rounding-order differences by ~1e6
    # (tests/test_oracle_chaos.py), so 1e-7 is ~10x the expected difference
    ic = inputs.grid16()
    g = run_gpu(ic, B.FP64, "kdk", 20)
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, 20, "kdk")
    assert np.abs(g["x"] - r["x"]).max() < 1e-7
    assert g["a"] == pytest.approx(r["schedule"]["a"][-1], rel=1e-13)


@pytest.mark.parametrize("critical,n", [(False, PRE_COLLAPSE["grid32"]), (True, 10)])
def test_grid32_with_tracers(critical, n):
    # the 32^3 paper-scale workload: growing-mode velocities, FP32 compensated
    # force, FP64 a(t), 64 tracers recorded every step
    ic = inputs.grid32(critical=critical)
    tr = inputs.tracers(ic.N, 64, 7)
    g = run_gpu(ic, B.FP32_COMP, "kdk", n, tracers=tr)
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "kdk", tracers=tr)
    check_state(g, r, B.FP32_COMP, n)
    assert g["tracers"].shape == (n, 64, 6)
    np.testing.assert_allclose(g["tracers"][:, :, :3], r["tracers"][:, :, :3], atol=1e-5)
    vs = np.abs(r["tracers"][:, :, 3:]).max()
    np.testing.assert_allclose(g["tracers"][:, :, 3:], r["tracers"][:, :, 3:],
                               atol=VEL_MAX_TOL[B.FP32_COMP] * vs)


def test_split_calls_equal_one_call():
    ic = inputs.grid16(critical=True)
    one = run_gpu(ic, B.FP32, "kdk", 12)
    split = run_gpu(ic, B.FP32, "kdk", 12, chunks=[5, 1, 6])
    assert np.array_equal(one["x"], split["x"]) and np.array_equal(one["v"], split["v"])


def test_more_steps_than_one_schedule_chunk():
    # 1100 steps cross the 1024-step schedule chunk; small weakly bound system
    rng = np.random.default_rng(21)
    N = 64
    x = inputs.f32(rng.random((N, 3)))
    v = inputs.f32(0.01 * rng.standard_normal((N, 3)))
    m = inputs.f32(np.full(N, 0.01 / N))
    ic = inputs.ICs(x=x, v=v, m=m, eps=0.05, name="weak")
    tau = 1e-3
    g = run_gpu(ic, B.FP64, "kdk", 1100, a_start=0.5, tau=tau)
    r = oracle.run(x, v, m, 0.05, 1.0, LCDM, 0.5, tau, 1100, "kdk")
    assert np.abs(g["x"] - r["x"]).max() < 1e-9
    assert g["a"] == pytest.approx(r["schedule"]["a"][-1], rel=1e-12)


def test_diagnostics_match_oracle():
    ic = inputs.grid16(critical=True)
    g = run_gpu(ic, B.FP64, "kdk", 5)
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, 5, "kdk")
    d = oracle.diagnostics(r["x"], r["v"], ic.m, r["schedule"]["a"][-1], ic.eps, 1.0, LCDM)
    gd = g["diag"]
    assert gd["K"] == pytest.approx(d["K"], rel=1e-9)
    assert gd["W"] == pytest.approx(d["W"], rel=1e-9)
    assert gd["H"] == pytest.approx(d["H"], rel=1e-12)
    np.testing.assert_allclose([gd["Cx"], gd["Cy"], gd["Cz"]], d["COM"], rtol=1e-12)
    pscale = abs(d["K"]) ** 0.5
    np.testing.assert_allclose([gd["Px"], gd["Py"], gd["Pz"]], d["P"], atol=1e-12 * pscale + 1e-15)
    # |x| <= ~1, so |L| is bounded by the same scale as |P|
    np.testing.assert_allclose([gd["Lx"], gd["Ly"], gd["Lz"]], d["L"], atol=1e-12 * pscale + 1e-15)
    assert gd["step"] == 5


@pytest.mark.parametrize("prec", [B.FP64, B.FP32_COMP])
def test_diagnostics_of_a_rotating_boosted_box_match_oracle(prec):
    # a box with a rigid rotation, a bulk velocity and random motions, so that
    # every moment (P, L, COM) is far from zero; compared element by element
    ic = inputs.grid16(critical=True)
    rng = np.random.default_rng(8)
    c = ic.x.mean(0)
    w = np.array([0.4, -0.9, 1.3])
    ic.v = inputs.f32(np.cross(w, ic.x - c) + np.array([0.3, 0.1, -0.2])
                      + 0.05 * rng.standard_normal(ic.x.shape))
    n = 3
    g = run_gpu(ic, prec, "kdk", n)
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "kdk")
    d = oracle.diagnostics(g["x"], g["v"], ic.m, g["a"], ic.eps, 1.0, LCDM)
    gd = g["diag"]
    tol = 1e-12 if prec == B.FP64 else 1e-6
    # same state on both sides: the GPU's moments of its own state
    for key, names in (("P", ("Px", "Py", "Pz")), ("L", ("Lx", "Ly", "Lz")),
                       ("COM", ("Cx", "Cy", "Cz"))):
        got = np.array([gd[k] for k in names])
        np.testing.assert_allclose(got, d[key], atol=tol * np.abs(d[key]).max())
        assert np.abs(d[key]).max() > 1e-3 * (1.0 if key == "COM" else ic.m.sum() * g["a"] ** 2)
    assert gd["K"] == pytest.approx(d["K"], rel=tol)
    assert gd["W"] == pytest.approx(d["W"], rel=tol)
    # and the oracle's own trajectory gives the same moments (before collapse)
    dr = oracle.diagnostics(r["x"], r["v"], ic.m, r["schedule"]["a"][-1], ic.eps, 1.0, LCDM)
    np.testing.assert_allclose([gd["Lx"], gd["Ly"], gd["Lz"]], dr["L"],
                               atol=1e-5 * np.abs(dr["L"]).max())


def test_fp32_diagnostics_close_to_oracle():
    ic = inputs.grid16(critical=True)
    g = run_gpu(ic, B.FP32, "kdk", 3)
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, 3, "kdk")
    d = oracle.diagnostics(r["x"], r["v"], ic.m, r["schedule"]["a"][-1], ic.eps, 1.0, LCDM)
    assert g["diag"]["W"] == pytest.approx(d["W"], rel=1e-6)
    assert g["diag"]["K"] == pytest.approx(d["K"], rel=1e-4)


def test_momentum_and_angular_momentum_invariants_fp64():
    # sum m F = 0 and sum m x cross F = 0 make sum m v and sum m x cross v
    # scale exactly by the product of the drag factors
    ic = inputs.grid16()
    rng = np.random.default_rng(5)
    ic.v = inputs.f32(0.05 * rng.standard_normal(ic.x.shape))
    n = 30
    g = run_gpu(ic, B.FP64, "kdk", n)
    sch = oracle.schedule(LCDM, inputs.A_START, TAU, n, "kdk")
    fac = np.prod(sch["c1"] * sch["c2"])
    P0 = np.sum(ic.m[:, None] * ic.v, axis=0)
    P1 = np.sum(ic.m[:, None] * g["v"], axis=0)
    np.testing.assert_allclose(P1, fac * P0, atol=1e-12 * np.abs(P0).max())


def test_error_paths():
    ic = inputs.grid16()
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START)
    try:
        with pytest.raises(B.ColatusError) as e:
            sim.step(TAU, 1)
        assert e.value.status == B.E_STATE
        bad = ic.x.copy()
        bad[7, 1] = np.nan
        with pytest.raises(B.ColatusError) as e:
            sim.set_state(bad)
        assert e.value.status == B.E_NONFINITE
        sim.set_state(ic.x)
        with pytest.raises(B.ColatusError) as e:
            sim.step(-1.0, 1)
        assert e.value.status == B.E_ARG
    finally:
        sim.close()


def test_recollapse_reports_friedmann_error():
    # closed matter universe (Omega_M = 2, Omega_K = -1) turns around at a = 2
    ic = inputs.grid16()
    sim = B.Simulation(ic.m, ic.eps, dict(Omega_R=0.0, Omega_M=2.0, Omega_K=-1.0, Omega_L=0.0, H0=1.0),
                       1.9, prec=B.FP64)
    try:
        sim.set_state(ic.x)
        sim.step(0.05, 40)
        with pytest.raises(B.ColatusError) as e:
            sim.synchronize()
        assert e.value.status == B.E_FRIEDMANN
    finally:
        sim.close()


@pytest.mark.parametrize("prec,tol", [(B.FP64, 1e-9), (B.FP32_COMP, 1e-4)])
def test_layzer_irvine_residual_follows_the_oracle(prec, tol):
    # 50 KDK steps of the 16^3 box at the background density, diagnostics
    # (FP64 reductions on the GPU) after every step: the residual of
    # d(K+W)/dt = -H (2K+W) is the leapfrog's own O(tau^2) error (~2e-3 of
    # |W0| here) and must follow the oracle's residual for the same run
    ic = inputs.grid16(critical=True)
    n = 50
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=prec, scheme=B.KDK)
    try:
        sim.set_state(ic.x, ic.v)
        diags = [sim.diagnostics()]
        for _ in range(n):
            sim.step(TAU, 1)
            diags.append(sim.diagnostics())
    finally:
        sim.close()
    t = np.array([d["t"] for d in diags])
    res_gpu = oracle.layzer_irvine(diags, t)
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "kdk", diag_every=1)
    res_ref = oracle.layzer_irvine([d[1] for d in r["diagnostics"]], TAU * np.arange(n + 1))
    assert 1e-3 < np.abs(res_ref).max() < 1e-2            # the discretisation error is resolved
    np.testing.assert_allclose(res_gpu, res_ref, rtol=0, atol=tol)


@pytest.mark.parametrize("scheme", [B.KDK, B.KDK_CANONICAL])
def test_long_calls_match_single_steps_and_the_schedule(scheme):
    # One call of 300 steps runs while the FP64 schedule is still being
    # extended (in pieces of tens of entries on a side stream); it must give
    # the same states, bit for bit, as 300 calls of one step, and the
    # oracle's a(t).
    ic = inputs.grid8()
    n = 300
    out = []
    for calls in ([n], [1] * n):
        sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32, scheme=scheme)
        try:
            sim.set_state(ic.x, ic.v)
            for c in calls:
                sim.step(TAU, c)
            out.append(sim.state())
        finally:
            sim.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    kind = "canonical" if scheme == B.KDK_CANONICAL else "kdk"
    sch = oracle.schedule(LCDM, inputs.A_START, TAU, n, kind)
    assert out[0][3] == pytest.approx(sch["a"][-1], rel=1e-13)
    assert out[0][2] == pytest.approx(n * TAU, rel=1e-13)


@pytest.mark.parametrize("scheme,prec", [(B.KDK, B.FP32_COMP), (B.DKD, B.FP32), (B.KDK_CANONICAL, B.FP32),
                                         (B.KDK, B.FP64)])
def test_resume_from_a_saved_state_is_bitwise(scheme, prec):
    # Checkpoint and resume: a new context started at the saved scale factor
    # with the saved positions and velocities continues the run bit for bit
    # (the schedule depends only on a, and the step opening is recomputed
    # from the same forces).  Time restarts at 0 in the new context.
    ic = inputs.grid8()
    n1, n2 = 7, 9
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=prec, scheme=scheme)
    try:
        sim.set_state(ic.x, ic.v)
        sim.step(TAU, n1 + n2)
        x_ref, v_ref, t_ref, a_ref = sim.state()
    finally:
        sim.close()
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=prec, scheme=scheme)
    try:
        sim.set_state(ic.x, ic.v)
        sim.step(TAU, n1)
        x1, v1, t1, a1 = sim.state()
    finally:
        sim.close()
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, a1, prec=prec, scheme=scheme)
    try:
        sim.set_state(x1, v1)
        sim.step(TAU, n2)
        x2, v2, t2, a2 = sim.state()
    finally:
        sim.close()
    assert np.array_equal(x2, x_ref) and np.array_equal(v2, v_ref)
    assert a2 == a_ref
    assert t1 + t2 == pytest.approx(t_ref, rel=1e-14)
