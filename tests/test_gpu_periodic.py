"""GPU parity of periodic boundaries (Ewald summation) against the oracle's
converged Ewald sum: forces in every precision (unwrapped positions too), the
lattice and large-box limits, KDK and DKD trajectories, and the API rules."""
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
PRECS = [B.FP32, B.FP32_COMP, B.FP64]


def rel_rms(a, b):
    return float(np.sqrt(np.mean(np.sum((a - b) ** 2, axis=1))) /
                 np.mean(np.linalg.norm(b, axis=1)))


def periodic_forces(x, m, eps, L, prec, a=1.0, G=1.0, **kw):
    sim = B.Simulation(m, eps, LCDM_D, a, prec=prec, G=G)
    try:
        sim.set_state(x)
        sim.set_periodic(L, **kw)
        return sim.forces(), sim.periodic_params()
    finally:
        sim.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [2, 257, 3000])
def test_forces_match_the_converged_ewald_sum(N, prec):
    rng = np.random.default_rng(800 + N)
    L = 2.5
    x = inputs.f32(L * rng.random((N, 3)))
    m = inputs.f32(rng.lognormal(0.0, 0.5, N) / N)
    eps, a, G = 0.01, 0.5, 1.3
    got, _ = periodic_forces(x, m, eps, L, prec, a=a, G=G)
    ref = oracle.ewald_forces(x, m, eps, L, G) / a ** 3
    assert rel_rms(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_clustered_bodies(prec):
    ic = inputs.plummer_clusters(2000, 9)
    got, _ = periodic_forces(ic.x, ic.m, 0.005, 1.0, prec)
    assert rel_rms(got, oracle.ewald_forces(ic.x, ic.m, 0.005, 1.0)) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_unwrapped_positions(prec):
    # bodies moved by whole boxes: the minimum image is taken per pair.  In
    # FP32 the difference of two positions a few boxes apart rounds at
    # ~ulp(3) = 2.4e-7, which bounds the agreement for any FP32 mode.
    rng = np.random.default_rng(810)
    x = rng.random((2000, 3))
    m = inputs.f32(rng.random(2000) / 2000)
    xs = inputs.f32(x + rng.integers(-2, 3, size=x.shape))
    got, _ = periodic_forces(xs, m, 0.01, 1.0, prec)
    ref = oracle.ewald_forces(xs, m, 0.01, 1.0)
    assert rel_rms(got, ref) < (1e-11 if prec == B.FP64 else 1e-5)


def test_parameters_follow_the_precision():
    x, m = inputs.f32(np.random.default_rng(811).random((300, 3))), np.full(300, 1.0 / 300)
    _, p32 = periodic_forces(x, m, 0.01, 1.0, B.FP32)
    _, p64 = periodic_forces(x, m, 0.01, 1.0, B.FP64)
    assert 8.5 < p32["alpha"] < 9.5 and p32["nk"] == 13
    assert 11.5 < p64["alpha"] < 13.0 and 22 <= p64["nk"] <= 24
    assert p64["nkv"] > p32["nkv"] > 4000
    got, p = periodic_forces(x, m, 0.01, 1.0, B.FP64, alpha=12.5, nk=25)
    assert p["alpha"] == 12.5 and p["nk"] == 25
    assert rel_rms(got, oracle.ewald_forces(x, m, 0.01, 1.0)) < 1e-11


@pytest.mark.parametrize("prec", [B.FP32, B.FP64])
def test_lattice_feels_no_force(prec):
    # 5^3 bodies at spacing 1 in a box of side 5: every position is exact in
    # float, and with an odd count no pair is exactly half a box apart (where
    # the nearest image is not unique)
    n, L = 5, 5.0
    q = np.arange(n) + 0.75
    x = np.stack(np.meshgrid(q, q, q, indexing="ij"), axis=-1).reshape(-1, 3)
    m = np.full(len(x), 1.0 / len(x))
    got, _ = periodic_forces(x, m, 0.01, L, prec)
    one_neighbour = m[0]
    assert np.abs(got).max() < (1e-5 if prec == B.FP32 else 1e-12) * one_neighbour


def test_a_large_box_reproduces_isolated_forces():
    rng = np.random.default_rng(812)
    x = inputs.f32(rng.random((2000, 3)))
    m = inputs.f32(rng.random(2000) / 2000)
    iso = oracle.forces(x, m, 0.01)
    got, _ = periodic_forces(x, m, 0.01, 1000.0, B.FP64)
    # what remains is the background term -(4 pi/3V) sum_j m_j d_j ~ 1e-9
    assert rel_rms(got, iso) < 1e-7


def test_switching_periodic_off_restores_the_isolated_force():
    rng = np.random.default_rng(813)
    x, m = inputs.f32(rng.random((1000, 3))), inputs.f32(rng.random(1000) / 1000)
    sim = B.Simulation(m, 0.01, LCDM_D, 1.0, prec=B.FP32)
    try:
        sim.set_state(x)
        iso = sim.forces()
        sim.set_periodic(1.0)
        per = sim.forces()
        sim.set_periodic(0.0)
        back = sim.forces()
    finally:
        sim.close()
    assert np.array_equal(iso, back) and not np.array_equal(iso, per)


@pytest.mark.parametrize("scheme", ["kdk", "dkd"])
@pytest.mark.parametrize("prec", PRECS)
def test_ten_periodic_steps(prec, scheme):
    ic = inputs.perturbed_grid(8, 0.1, 0.02, 4, zeldovich=True, total_mass=inputs.CRITICAL_MATTER_DENSITY)
    n = 10
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=prec,
                       scheme={"kdk": B.KDK, "dkd": B.DKD}[scheme])
    try:
        sim.set_state(ic.x, ic.v)
        sim.set_periodic(1.0)
        sim.step(TAU, 4)
        sim.step(TAU, n - 4)
        x, v, t, a = sim.state()
    finally:
        sim.close()
    r = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, scheme, box=1.0)
    r_iso = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, scheme)
    tol = 1e-9 if prec == B.FP64 else 1e-5
    assert np.abs(r["v"] - r_iso["v"]).max() > 100 * tol * np.abs(r["v"]).max()
    assert np.abs(x - r["x"]).max() < tol
    dv = np.linalg.norm(v - r["v"], axis=1)
    vt = 1e-11 if prec == B.FP64 else 1e-5
    assert np.sqrt(np.mean(dv ** 2)) < vt * np.sqrt(np.mean(np.sum(r["v"] ** 2, axis=1)))


def test_paths_not_built_for_periodic_boundaries_refuse():
    ic = inputs.grid8()
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32)
    try:
        sim.set_state(ic.x, ic.v)
        sim.set_periodic(1.0)
        for call in (lambda: sim.autotune(1),
                     lambda: sim.set_deformation(0.1, (0.5, 0.5, 0.5))):
            with pytest.raises(B.ColatusError):
                call()
        with pytest.raises(B.ColatusError):
            sim.set_periodic(-1.0)
        sim.set_periodic(0.0)
        sim.set_deformation(0.1, (0.5, 0.5, 0.5))
        with pytest.raises(B.ColatusError):
            sim.set_periodic(1.0)
        with pytest.raises(B.ColatusError):
            sim.periodic_params()
    finally:
        sim.close()


@pytest.mark.parametrize("prec", PRECS)
def test_periodic_forces_are_deterministic(prec):
    # the structure factors are summed over body splits in a fixed order
    rng = np.random.default_rng(814)
    x, m = inputs.f32(rng.random((5000, 3))), inputs.f32(rng.random(5000) / 5000)
    sim = B.Simulation(m, 0.01, LCDM_D, 1.0, prec=prec)
    try:
        sim.set_state(x)
        sim.set_periodic(1.0)
        first = sim.forces()
        assert all(np.array_equal(first, sim.forces()) for _ in range(3))
    finally:
        sim.close()


def test_extreme_k_space_sizes():
    # nk = 63 is the largest the k-space kernels' shared memory allows (a
    # superset of the converged sum, so the result matches the oracle); nk = 1
    # leaves a single shell of k-vectors (a truncated sum: finite, and different).
    rng = np.random.default_rng(815)
    x, m = inputs.f32(rng.random((3000, 3))), inputs.f32(rng.random(3000) / 3000)
    ref = oracle.ewald_forces(x, m, 0.01, 1.0)
    big, p = periodic_forces(x, m, 0.01, 1.0, B.FP32, alpha=9.0, nk=63)
    assert p["nk"] == 63 and p["nkv"] > 500000
    assert rel_rms(big, ref) < 1e-5
    small, p = periodic_forces(x, m, 0.01, 1.0, B.FP32, alpha=9.0, nk=1)
    assert p["nkv"] == 3 and np.all(np.isfinite(small))
    assert rel_rms(small, ref) > 1e-3
    with pytest.raises(B.ColatusError):
        periodic_forces(x, m, 0.01, 1.0, B.FP32, alpha=9.0, nk=64)
