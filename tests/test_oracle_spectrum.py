"""Pins of the oracle's tracer velocity energy spectrum."""
import numpy as np
import pytest

import oracle


def test_pure_sinusoid_peak_height_and_zero_elsewhere():
    T, dt, k0, A = 256, 0.01, 17, 0.7
    n = np.arange(T)
    v = np.zeros((T, 1, 3))
    v[:, 0, 1] = A * np.cos(2 * np.pi * k0 * n / T + 0.3)
    E = oracle.velocity_spectrum(v, dt, "rect")[0]
    # |DFT| at k0 is A T / 2; one-sided doubles it; the (1/2) of the energy
    assert E[k0] == pytest.approx(2 * 0.5 * dt / T * (A * T / 2) ** 2, rel=1e-12)
    others = np.delete(E, k0)
    assert np.all(np.abs(others) < 1e-20 * E[k0] + 1e-24)


def test_hann_side_lobes_are_a_quarter_of_the_peak():
    T, dt, k0 = 200, 0.5, 30
    n = np.arange(T)
    v = np.zeros((T, 2, 3))
    v[:, 1, 0] = np.sin(2 * np.pi * k0 * n / T)
    E = oracle.velocity_spectrum(v, dt, "hann")[1]
    # the periodic Hann window turns a bin-centred line into amplitudes (1/4, 1/2, 1/4)
    assert E[k0 - 1] / E[k0] == pytest.approx(0.25, rel=1e-10)
    assert E[k0 + 1] / E[k0] == pytest.approx(0.25, rel=1e-10)
    assert np.all(np.delete(E, [k0 - 1, k0, k0 + 1]) < 1e-20)


@pytest.mark.parametrize("T", [2, 3, 64, 101, 250])
@pytest.mark.parametrize("window", ["rect", "hann"])
def test_parseval(T, window):
    rng = np.random.default_rng(T)
    dt = 0.037
    v = rng.standard_normal((T, 5, 3)) + rng.standard_normal((1, 5, 3))
    E = oracle.velocity_spectrum(v, dt, window)
    u = v - v.mean(axis=0)
    n = np.arange(T)
    w = np.ones(T) if window == "rect" else 0.5 * (1 - np.cos(2 * np.pi * n / T))
    if np.sum(w * w) == 0:
        pytest.skip("window vanishes")
    lhs = E.sum(axis=1) / (T * dt)
    rhs = np.sum(w[:, None] ** 2 * 0.5 * np.sum(u ** 2, axis=2), axis=0) / np.sum(w * w)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


@pytest.mark.parametrize("T", [63, 64])
def test_matches_numpy_fft(T):
    rng = np.random.default_rng(80 + T)
    v = rng.standard_normal((T, 4, 3))
    dt = 2.0
    E = oracle.velocity_spectrum(v, dt, "rect", detrend=False)
    F = np.fft.rfft(v, axis=0)                       # [nf, 4, 3]
    P = 0.5 * np.sum(np.abs(F) ** 2, axis=2).T       # [4, nf]
    c = np.full(T // 2 + 1, 2.0)
    c[0] = 1.0
    if T % 2 == 0:
        c[-1] = 1.0
    np.testing.assert_allclose(E, c * dt / T * P, rtol=1e-11, atol=1e-12 * P.max())


def test_constant_series():
    T, dt = 40, 0.1
    v = np.tile(np.array([1.0, -2.0, 0.5]), (T, 3, 1))
    assert np.all(np.abs(oracle.velocity_spectrum(v, dt)) < 1e-25)
    E = oracle.velocity_spectrum(v, dt, detrend=False)
    assert E[0, 0] == pytest.approx(dt * T * 0.5 * (1 + 4 + 0.25), rel=1e-14)
    assert np.all(np.abs(E[:, 1:]) < 1e-20)
