"""GPU parity of the batched ensemble (many uneven-N realisations stepped in
one persistent launch per step, 16 steps per captured CUDA graph) against the
FP64 oracle run realisation by realisation."""
import numpy as np
import pytest

import oracle
from paper_1208_3444_b300 import binding as B
from paper_1208_3444_b300 import inputs

pytestmark = pytest.mark.gpu

LCDM_D = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
LCDM = oracle.Cosmology(0.0, 0.3, 0.0, 0.7, 1.0)
TAU = inputs.lcdm_tau(2000)


def rel_rms(a, b):
    return float(np.sqrt(np.mean(np.sum((a - b) ** 2, axis=1))) /
                 np.mean(np.linalg.norm(b, axis=1)))


def concat(ics):
    return (np.concatenate([ic.x for ic in ics]), np.concatenate([ic.v for ic in ics]),
            np.concatenate([ic.m for ic in ics]), np.array([ic.eps for ic in ics]),
            np.array([ic.N for ic in ics]))


@pytest.mark.parametrize("masses", ["lognormal", "equal"])
def test_forces_of_uneven_realisations(masses):
    # "equal": every realisation has its own equal masses, so the ensemble
    # takes the equal-mass kernel, whose padding bodies must contribute nothing
    rng = np.random.default_rng(40)
    ics = []
    for N, eps in ((1, 0.02), (7, 0.01), (300, 0.005), (1025, 0.01), (2000, 0.003), (4096, 0.01)):
        x = inputs.f32(rng.random((N, 3)))
        if masses == "equal":
            m = inputs.f32(np.full(N, rng.lognormal(0.0, 0.5) / N))
        else:
            m = inputs.f32(rng.lognormal(0.0, 0.5, N) / N)
        ics.append(inputs.ICs(x=x, v=np.zeros_like(x), m=m, eps=eps, name=f"r{N}"))
    x, v, m, eps, Ns = concat(ics)
    ens = B.Ensemble(Ns, m, eps, LCDM_D, 0.8, G=1.1)
    try:
        ens.set_state(x, v)
        acc = ens.forces()
    finally:
        ens.close()
    off = np.concatenate([[0], np.cumsum(Ns)])
    for r, ic in enumerate(ics):
        got = acc[off[r]:off[r + 1]]
        if ic.N == 1:
            assert np.all(got == 0)
            continue
        ref = oracle.forces(ic.x, ic.m, ic.eps, 1.1) / 0.8 ** 3
        assert rel_rms(got, ref) < 1e-5, ic.name


def critical_ensemble(counts, seed=6):
    out = []
    for r, N in enumerate(counts):
        n = int(np.ceil(round(N ** (1.0 / 3.0), 9)))
        while n ** 3 < N:
            n += 1
        out.append(inputs.perturbed_grid(n, 0.1, 0.02, seed * 100 + r, zeldovich=True, count=N,
                                         total_mass=inputs.CRITICAL_MATTER_DENSITY))
    return out


def test_steps_match_oracle_per_realisation():
    ics = critical_ensemble([512, 1000, 1729, 3000])
    x, v, m, eps, Ns = concat(ics)
    n = 20   # one 16-step graph replay and 4 direct steps
    ens = B.Ensemble(Ns, m, eps, LCDM_D, inputs.A_START)
    try:
        ens.set_state(x, v)
        ens.step(TAU, n)
        gx, gv, t, a = ens.state()
    finally:
        ens.close()
    off = np.concatenate([[0], np.cumsum(Ns)])
    rng = np.random.default_rng(0)
    for r, ic in enumerate(ics):
        ref = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "kdk")
        # the dynamics' own response to rounding-sized (6e-8) input changes,
        # measured with the oracle: a close encounter can amplify it past 1e-5
        xp = ic.x * (1.0 + 6e-8 * rng.standard_normal(ic.x.shape))
        pert = oracle.run(xp, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "kdk")
        chaos_x = np.abs(pert["x"] - ref["x"]).max()
        assert np.abs(gx[off[r]:off[r + 1]] - ref["x"]).max() < max(1e-5, 10.0 * chaos_x), r
        rms = lambda d: float(np.sqrt(np.mean(np.sum(d ** 2, axis=1))))
        chaos_v = rms(pert["v"] - ref["v"])
        tol_v = max(1e-5 * rms(ref["v"]), 10.0 * chaos_v)
        assert rms(gv[off[r]:off[r + 1]] - ref["v"]) < tol_v, r
        assert a == pytest.approx(ref["schedule"]["a"][-1], rel=1e-13)
    assert t == pytest.approx(n * TAU, rel=1e-13)


def test_graph_replays_are_deterministic_and_split_calls_agree():
    ics = critical_ensemble([700, 1300])
    x, v, m, eps, Ns = concat(ics)
    res = []
    for chunks in ([32], [16, 16], [5, 27]):
        ens = B.Ensemble(Ns, m, eps, LCDM_D, inputs.A_START)
        try:
            ens.set_state(x, v)
            for c in chunks:
                ens.step(TAU, c)
            res.append(ens.state()[:2])
        finally:
            ens.close()
    for r in res[1:]:
        assert np.array_equal(r[0], res[0][0]) and np.array_equal(r[1], res[0][1])


def test_ensemble_workload_momentum_invariant():
    # the 64-realisation workload (log-uniform N in [1024, 32768]), 3 steps:
    # sum m v of each realisation scales by the product of its drag factors
    ics = inputs.ensemble(64, seed=5)
    x, v, m, eps, Ns = concat(ics)
    ens = B.Ensemble(Ns, m, eps, LCDM_D, inputs.A_START)
    try:
        ens.set_state(x, v)
        ens.step(TAU, 3)
        gx, gv, t, a = ens.state()
        st = ens.stats()
    finally:
        ens.close()
    assert np.all(np.isfinite(gx)) and np.all(np.isfinite(gv))
    sch = oracle.schedule(LCDM, inputs.A_START, TAU, 3, "kdk")
    fac = float(np.prod(sch["c1"] * sch["c2"]))
    off = np.concatenate([[0], np.cumsum(Ns)])
    for r in range(len(ics)):
        s = slice(off[r], off[r + 1])
        P0 = np.sum(m[s, None] * v[s], axis=0)
        P1 = np.sum(m[s, None] * gv[s], axis=0)
        scale = np.sum(m[s, None] * np.abs(gv[s]), axis=0)
        assert np.all(np.abs(P1 - fac * P0) < 1e-5 * scale), r
    assert st["pairs_per_step"] == pytest.approx(float(np.sum(Ns.astype(float) ** 2)))


@pytest.mark.parametrize("masses", ["lognormal", "equal"])
def test_autotune_and_every_shape(masses):
    rng = np.random.default_rng(41)
    ics = []
    for N, eps in ((5, 0.02), (700, 0.01), (1300, 0.005), (2500, 0.01)):
        x = inputs.f32(rng.random((N, 3)))
        m = (np.full(N, rng.lognormal(0.0, 0.5) / N) if masses == "equal"
             else rng.lognormal(0.0, 0.5, N) / N)
        ics.append(inputs.ICs(x=x, v=inputs.f32(0.1 * rng.standard_normal((N, 3))), m=inputs.f32(m),
                              eps=eps, name=f"r{N}"))
    x, v, m, eps, Ns = concat(ics)
    off = np.concatenate([[0], np.cumsum(Ns)])
    refs = [oracle.forces(ic.x, ic.m, ic.eps) for ic in ics]
    ens = B.Ensemble(Ns, m, eps, LCDM_D, 1.0)
    try:
        ens.set_state(x, v)
        ms, chosen = ens.autotune(2)
        assert len(ms) == 4 and np.all(ms > 0) and chosen == int(np.argmin(ms))
        for shape in range(4):
            ens.set_tuning(shape)
            ens.set_state(x, v)                              # back to the initial positions
            a = ens.state()[3]                               # the clock has moved on
            acc = ens.forces()
            assert np.array_equal(acc, ens.forces())          # deterministic per shape
            for r, ref in enumerate(refs):
                assert rel_rms(acc[off[r]:off[r + 1]], ref / a ** 3) < 1e-5, (shape, r)
            ens.step(TAU, 17)                                # a fresh graph per shape
            assert np.all(np.isfinite(ens.state()[1]))
        with pytest.raises(B.ColatusError):
            ens.set_tuning(4)
    finally:
        ens.close()


def test_tracers_match_oracle_per_realisation():
    # tracers in every realisation, at its first and last body among others;
    # 20 steps: one 16-step graph replay and 4 direct steps
    ics = critical_ensemble([512, 1000, 1729, 3000])
    x, v, m, eps, Ns = concat(ics)
    off = np.concatenate([[0], np.cumsum(Ns)])
    local = {0: [0, 511, 100], 1: [3, 999], 2: [0, 864], 3: [2999, 1500, 7]}
    idx = np.array([off[r] + k for r in local for k in local[r]])
    n = 20
    ens = B.Ensemble(Ns, m, eps, LCDM_D, inputs.A_START)
    try:
        ens.set_state(x, v)
        ens.record_tracers(idx, 25)
        ens.step(TAU, n)
        rec = ens.read_tracers()
        gx, gv, _, _ = ens.state()
    finally:
        ens.close()
    assert rec.shape == (n, len(idx), 6)
    # the last record is the state itself, bit for bit
    assert np.array_equal(rec[-1, :, :3], gx[idx].astype(np.float32))
    assert np.array_equal(rec[-1, :, 3:], gv[idx].astype(np.float32))
    col = 0
    rng = np.random.default_rng(1)
    for r, ks in local.items():
        ic = ics[r]
        ref = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "kdk", tracers=ks)
        xp = ic.x * (1.0 + 6e-8 * rng.standard_normal(ic.x.shape))
        pert = oracle.run(xp, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "kdk", tracers=ks)
        got = rec[:, col:col + len(ks)]
        chaos = np.abs(pert["tracers"] - ref["tracers"]).max(axis=(0, 1))
        scale = np.abs(ref["tracers"]).max(axis=(0, 1))
        err = np.abs(got - ref["tracers"]).max(axis=(0, 1))
        assert np.all(err[:3] < np.maximum(1e-5, 10 * chaos[:3])), (r, err)
        assert np.all(err[3:] < np.maximum(1e-5 * scale[3:], 10 * chaos[3:])), (r, err)
        col += len(ks)


def test_tracer_ring_and_rerecording_with_graphs():
    ics = critical_ensemble([700, 1300])
    x, v, m, eps, Ns = concat(ics)
    ens = B.Ensemble(Ns, m, eps, LCDM_D, inputs.A_START)
    try:
        ens.set_state(x, v)
        ens.record_tracers([5, 1999], 7)             # a ring shorter than the run
        ens.step(TAU, 16)
        ens.step(TAU, 4)
        rec = ens.read_tracers()
        gx, gv, _, _ = ens.state()
        assert rec.shape == (7, 2, 6)                # the last 7 of 20 steps
        assert np.array_equal(rec[-1, :, :3], gx[[5, 1999]].astype(np.float32))
        # new tracers: the graphs captured with the old buffers are replaced
        ens.record_tracers([700, 3], 40)
        ens.step(TAU, 16)
        rec2 = ens.read_tracers()
        gx2, gv2, _, _ = ens.state()
        assert rec2.shape == (16, 2, 6)
        assert np.array_equal(rec2[-1, :, :3], gx2[[700, 3]].astype(np.float32))
        assert np.array_equal(rec2[-1, :, 3:], gv2[[700, 3]].astype(np.float32))
        ens.record_tracers([], 1)                    # stop recording
        ens.step(TAU, 2)
        assert ens.read_tracers().shape[0] == 0
        with pytest.raises(B.ColatusError):
            ens.record_tracers([3, 3], 5)
        with pytest.raises(B.ColatusError):
            ens.record_tracers([2000], 5)
    finally:
        ens.close()


@pytest.mark.parametrize("scheme", ["dkd", "canonical"])
def test_schemes_match_oracle_per_realisation(scheme):
    # the paper's DKD (force at the half-drift positions) and the canonical
    # KDK of Sec. II through the same graph replay and direct steps
    ics = critical_ensemble([512, 1000, 1729])
    x, v, m, eps, Ns = concat(ics)
    n = 20
    ens = B.Ensemble(Ns, m, eps, LCDM_D, inputs.A_START,
                     scheme=B.DKD if scheme == "dkd" else B.KDK_CANONICAL)
    try:
        ens.set_state(x, v)
        ens.step(TAU, 16)
        ens.step(TAU, 4)
        gx, gv, t, a = ens.state()
    finally:
        ens.close()
    off = np.concatenate([[0], np.cumsum(Ns)])
    rng = np.random.default_rng(2)
    rms = lambda d: float(np.sqrt(np.mean(np.sum(d ** 2, axis=1))))
    for r, ic in enumerate(ics):
        ref = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, scheme)
        # the oracle's own response to rounding-sized input changes (three
        # samples): a close pair (two bodies of the 1729-body DKD run) can
        # amplify it a hundredfold past the other bodies'
        chaos_x = chaos_v = 0.0
        for _ in range(3):
            xp = ic.x * (1.0 + 6e-8 * rng.standard_normal(ic.x.shape))
            pert = oracle.run(xp, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, scheme)
            chaos_x = max(chaos_x, np.abs(pert["x"] - ref["x"]).max())
            chaos_v = max(chaos_v, rms(pert["v"] - ref["v"]))
        err = np.abs(gx[off[r]:off[r + 1]] - ref["x"]).max(axis=1)
        assert np.mean(err < 1e-5) > 0.99, r                  # all but the encounters
        assert err.max() < max(1e-5, 10.0 * chaos_x), r
        tol_v = max(1e-5 * rms(ref["v"]), 10.0 * chaos_v)
        assert rms(gv[off[r]:off[r + 1]] - ref["v"]) < tol_v, r
        assert a == pytest.approx(ref["schedule"]["a"][-1], rel=1e-13)


def test_scheme_change_between_calls():
    # 16 KDK steps, then 16 DKD steps, against the oracle's two legs; the
    # change drops the KDK graph and re-opens from the state
    ics = critical_ensemble([700, 1300])
    x, v, m, eps, Ns = concat(ics)
    ens = B.Ensemble(Ns, m, eps, LCDM_D, inputs.A_START)
    try:
        ens.set_state(x, v)
        ens.step(TAU, 16)
        a16 = ens.state()[3]
        ens.set_scheme(B.DKD)
        ens.step(TAU, 16)
        gx, gv, _, _ = ens.state()
        with pytest.raises(B.ColatusError):
            ens.set_scheme(7)
    finally:
        ens.close()
    off = np.concatenate([[0], np.cumsum(Ns)])
    rng = np.random.default_rng(3)

    def two_legs(x0, ic):
        r1 = oracle.run(x0, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, 16, "kdk")
        return r1, oracle.run(r1["x"], r1["v"], ic.m, ic.eps, 1.0, LCDM, r1["schedule"]["a"][-1], TAU, 16,
                              "dkd")

    for r, ic in enumerate(ics):
        r1, r2 = two_legs(ic.x, ic)
        assert r1["schedule"]["a"][-1] == pytest.approx(a16, rel=1e-13)
        _, p2 = two_legs(ic.x * (1.0 + 6e-8 * rng.standard_normal(ic.x.shape)), ic)
        chaos = np.abs(p2["x"] - r2["x"]).max()
        assert np.abs(gx[off[r]:off[r + 1]] - r2["x"]).max() < max(1e-5, 10.0 * chaos), r
