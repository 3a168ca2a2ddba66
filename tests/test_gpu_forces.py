"""GPU parity of the all-pairs force (Eq. 1) against the FP64 oracle.

Tolerances (RMS over bodies of |acc_gpu - acc_oracle|, relative to the mean
|acc_oracle|): 1e-5 for FP32, 1e-6 for FP32 with compensated accumulation,
1e-11 for FP64.  Inputs are float32-representable, so both sides see the same
values; the oracle runs in double precision.
"""
import numpy as np
import pytest

import oracle
from paper_1208_3444_b300 import binding as B
from paper_1208_3444_b300 import inputs

pytestmark = pytest.mark.gpu

LCDM = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
TOL = {B.FP32: 1e-5, B.FP32_COMP: 1e-6, B.FP64: 1e-11}
PRECS = [B.FP32, B.FP32_COMP, B.FP64]


def rel_rms(a, b):
    return float(np.sqrt(np.mean(np.sum((a - b) ** 2, axis=1))) /
                 np.mean(np.linalg.norm(b, axis=1)))


def gpu_forces(x, m, eps, prec, a=1.0, G=1.0):
    sim = B.Simulation(m, eps, LCDM, a, prec=prec, G=G)
    try:
        sim.set_state(x)
        return sim.forces()
    finally:
        sim.close()


def random_system(N, seed):
    rng = np.random.default_rng(seed)
    x = inputs.f32(rng.random((N, 3)))
    m = inputs.f32(rng.lognormal(0.0, 0.5, N) / N)
    return x, m


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [1, 2, 3, 31, 33, 255, 257, 1023, 1025, 3000])
def test_small_and_ragged_sizes(N, prec):
    x, m = random_system(N, 100 + N)
    eps = 0.01
    got = gpu_forces(x, m, eps, prec)
    ref = oracle.forces(x, m, eps)
    if N == 1:
        assert np.all(got == 0.0)
        return
    assert rel_rms(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_grid16(prec):
    ic = inputs.grid16()
    got = gpu_forces(ic.x, ic.m, ic.eps, prec)
    ref = oracle.forces(ic.x, ic.m, ic.eps)
    assert rel_rms(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP])
def test_clustered_plummer_lognormal_masses(prec):
    ic = inputs.plummer_clusters(20000, 9)
    got = gpu_forces(ic.x, ic.m, ic.eps, prec)
    ref = oracle.forces(ic.x, ic.m, ic.eps)
    assert rel_rms(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP])
def test_grid32_every_body(prec):
    # the 32^3 workload, all bodies, in the launch configuration the benchmark uses
    ic = inputs.grid32()
    got = gpu_forces(ic.x, ic.m, ic.eps, prec)
    ref = oracle.forces(ic.x, ic.m, ic.eps)
    assert rel_rms(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP])
def test_128cubed_sampled_rows(prec):
    # N = 2^21 = 128^3 uniform bodies; 384 seeded rows checked against the oracle
    ic = inputs.uniform(1 << 21, 11)
    got = gpu_forces(ic.x, ic.m, ic.eps, prec)
    rows = np.sort(np.random.default_rng(12).choice(ic.N, 384, replace=False))
    ref = oracle.forces(ic.x, ic.m, ic.eps, rows=rows)
    assert rel_rms(got[rows], ref) < TOL[prec]
    assert np.all(np.isfinite(got))


def test_scale_factor_and_G():
    x, m = random_system(500, 3)
    base = gpu_forces(x, m, 0.02, B.FP64, a=1.0, G=1.0)
    np.testing.assert_allclose(gpu_forces(x, m, 0.02, B.FP64, a=0.5, G=1.0), 8.0 * base, rtol=1e-13)
    np.testing.assert_allclose(gpu_forces(x, m, 0.02, B.FP64, a=1.0, G=2.5), 2.5 * base, rtol=1e-13)


def test_device_tensors_in_and_out():
    import torch
    x, m = random_system(5000, 4)
    sim = B.Simulation(m, 0.01, LCDM, 1.0, prec=B.FP32)
    try:
        xt = torch.tensor(x, dtype=torch.float32, device="cuda")
        sim.set_state(xt)
        out = torch.empty((5000, 3), dtype=torch.float32, device="cuda")
        sim.forces(out)
        sim.synchronize()
        host = sim.forces()
    finally:
        sim.close()
    np.testing.assert_allclose(out.cpu().numpy(), host, rtol=1e-6, atol=1e-6 * np.abs(host).max())
    assert rel_rms(host, oracle.forces(x, m, 0.01)) < TOL[B.FP32]


def test_deterministic_repeat():
    x, m = random_system(4096, 5)
    a = gpu_forces(x, m, 0.01, B.FP32)
    b = gpu_forces(x, m, 0.01, B.FP32)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
@pytest.mark.parametrize("prec", [B.FP32, B.FP32_COMP])
@pytest.mark.parametrize("workload", ["grid32", "plummer"])
def test_every_tile_shape(shape, prec, workload):
    ic = inputs.grid32() if workload == "grid32" else inputs.plummer_clusters(30000, 9)
    sim = B.Simulation(ic.m, ic.eps, LCDM, 1.0, prec=prec)
    try:
        sim.set_state(ic.x)
        sim.set_tuning(shape)
        got = sim.forces()
    finally:
        sim.close()
    ref = oracle.forces(ic.x, ic.m, ic.eps)
    assert rel_rms(got, ref) < TOL[prec]


def test_autotune_and_cache(tmp_path):
    from paper_1208_3444_b300 import tuning
    ic = inputs.grid32()
    sim = B.Simulation(ic.m, ic.eps, LCDM, 1.0, prec=B.FP32_COMP)
    try:
        sim.set_state(ic.x)
        shape, ms = sim.autotune(2)
        assert shape in (0, 1, 2, 3) and len(ms) == 4 and ms[shape] == min(m for m in ms if m > 0)
        got = sim.forces()
        path = str(tmp_path / "tune.json")
        rec = tuning.tuned(sim, path, ic.m, "gpu")
        again = tuning.tuned(sim, path, ic.m, "gpu")
        assert rec == again and tuning.load(path)
        with pytest.raises(B.ColatusError):
            sim.set_tuning(7)
        sim.set_tuning(-1)
    finally:
        sim.close()
    assert rel_rms(got, oracle.forces(ic.x, ic.m, ic.eps)) < TOL[B.FP32_COMP]


def test_force_plan_names_the_launched_kernel():
    # the 32^3 equal-mass bodies take shape 3 (every pair once, 512 x 4 on
    # 2048-body tiles, the 136 tile pairs it <= jt) with the equal-mass form;
    # shape 0 (512 x 4, 512-body j-tiles, every 1/s^2 from the rsqrt) on request
    ic = inputs.grid32()
    for prec, comp in ((B.FP32, False), (B.FP32_COMP, True)):
        sim = B.Simulation(ic.m, ic.eps, LCDM, 1.0, prec=prec)
        try:
            sim.set_state(ic.x)
            p = sim.force_plan()
            sim.set_tuning(0)
            p0 = sim.force_plan()
        finally:
            sim.close()
        assert p["kind"] == "force_sym_f32" and p["comp"] == comp and p["eqm"]
        assert (p["threads"], p["ipt"], p["jt"], p["nrcp"]) == (512, 4, 2048, 0)
        assert p["units"] == 16 * 17 // 2
        assert p0["kind"] == "force_f32" and p0["comp"] == comp and p0["eqm"]
        assert (p0["threads"], p0["ipt"], p0["jt"], p0["nrcp"]) == (512, 4, 512, 0)
        assert p0["units"] == (ic.N // 2048) * (ic.N // 512)
