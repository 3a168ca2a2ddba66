"""GPU parity of the tracer velocity energy spectrum against the oracle's
direct DFT (both in FP64; the GPU sums in another order).

The library takes a mixed-radix FFT for T <= 6144 whose prime factors are
all <= 64 and the direct sum otherwise; the lengths below cover both, the
boundaries between them (6144, 6145, 6400; a radix-61 stage, a prime 67)
and the paper's record length of 2000 steps for 64 tracers."""
import numpy as np
import pytest

import oracle
from paper_1208_3444_b300 import binding as B
from paper_1208_3444_b300 import inputs

pytestmark = pytest.mark.gpu

LCDM_D = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
TAU = inputs.lcdm_tau(2000)


def close(got, ref):
    # per tracer: 1e-10 of the tracer's peak, and 1e-9 relative where resolved
    scale = np.abs(ref).max(axis=1, keepdims=True)
    return np.all(np.abs(got - ref) <= 1e-9 * np.abs(ref) + 1e-10 * scale)


def series(T, ntr, seed, dtype):
    rng = np.random.default_rng(seed)
    t = np.arange(T)[:, None, None]
    v = rng.standard_normal((T, ntr, 3)) + 3.0 * np.sin(2 * np.pi * 5 * t / T + rng.random((1, ntr, 3)))
    return (v + rng.standard_normal((1, ntr, 3))).astype(dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("window", ["rect", "hann"])
@pytest.mark.parametrize("T,ntr", [(2, 1), (3, 5), (257, 64), (500, 7), (1041, 3), (4113, 2),
                                   (2000, 64), (4096, 3), (6144, 2), (6145, 1), (6400, 1),
                                   (122, 4), (134, 3)])
def test_random_series(T, ntr, window, dtype):
    v = series(T, ntr, T + ntr, dtype)
    for detrend in (True, False):
        got = B.colatus_velocity_spectrum(v, 0.013, window, detrend)
        ref = oracle.velocity_spectrum(v.astype(np.float64), 0.013, window, detrend)
        assert got.shape == ref.shape == (ntr, T // 2 + 1)
        assert close(got, ref), (detrend, np.abs(got - ref).max())


def test_device_tensors_and_record_layout():
    import torch
    v = series(300, 9, 1, np.float32)
    rec = np.zeros((300, 9, 6), dtype=np.float32)
    rec[:, :, 3:] = v
    rec[:, :, :3] = 7.0                     # positions must be ignored
    ref = oracle.velocity_spectrum(v.astype(np.float64), 0.5, "hann")
    vt = torch.tensor(rec[:, :, 3:].copy(), device="cuda")
    out = torch.empty((9, 151), dtype=torch.float64, device="cuda")
    B.colatus_velocity_spectrum(vt, 0.5, "hann", True, out=out)
    torch.cuda.synchronize()
    assert close(out.cpu().numpy(), ref)
    # the same numbers from the interleaved (x, v) record with stride 6
    r6 = B.colatus_velocity_spectrum(rec, 0.5, "hann", offset=3)
    assert close(r6, ref)


@pytest.mark.parametrize("cap", [24, 23])
def test_recorded_tracers_in_the_ring(cap):
    # 24 records take the FFT, 23 (prime) the direct sum
    ic = inputs.grid16(critical=True)
    tr = inputs.tracers(ic.N, 64, 3)
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32)
    try:
        sim.set_state(ic.x, ic.v)
        sim.record_tracers(tr, cap)         # 40 steps: the ring wraps, the last cap are kept
        sim.step(TAU, 15)
        sim.step(TAU, 25)
        rec = sim.read_tracers()
        E = sim.tracer_spectrum(TAU, "hann")
        E_rect = sim.tracer_spectrum(TAU, "rect", detrend=False)
    finally:
        sim.close()
    assert rec.shape == (cap, 64, 6)
    v = rec[:, :, 3:].astype(np.float64)
    assert close(E, oracle.velocity_spectrum(v, TAU, "hann"))
    assert close(E_rect, oracle.velocity_spectrum(v, TAU, "rect", detrend=False))


def test_argument_checks():
    with pytest.raises(B.ColatusError):
        B.colatus_velocity_spectrum(np.zeros((1, 2, 3)), 0.1)         # T < 2
    with pytest.raises(B.ColatusError):
        B.colatus_velocity_spectrum(np.zeros((8, 2, 3)), -1.0)        # dt <= 0
    ic = inputs.grid8()
    sim = B.Simulation(ic.m, ic.eps, LCDM_D, inputs.A_START, prec=B.FP32)
    try:
        sim.set_state(ic.x, ic.v)
        with pytest.raises(B.ColatusError):
            sim.tracer_spectrum(TAU)                                 # nothing recorded
    finally:
        sim.close()
