"""Pins of the oracle's Friedmann solver (Eq. 2) against closed forms.

Each universe below has a textbook closed-form a(t); the oracle integrates
da/dt = a H(a) numerically, so agreement checks the RK4 stepping, the radicand
of Eq. 2 and the time convention (t = 0 at a_start) at once.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import Cosmology

A0 = 1.0 / 51.0


def _integrate(c, a0, T, nsteps, nsub=8):
    sch = oracle.schedule(c, a0, T / nsteps, nsteps, "kdk", nsub)
    return sch["t"], sch["a"]


def test_hubble_today_is_H0():
    c = Cosmology(0.0, 0.3, 0.0, 0.7, 2.5)
    assert oracle.hubble(1.0, c) == pytest.approx(2.5, rel=1e-15)


def test_hubble_terms():
    # each density term scales with its own power of a
    for i, p in enumerate((-4, -3, -2, 0)):
        om = [0.0, 0.0, 0.0, 0.0]
        om[i] = 1.0
        c = Cosmology(*om, 1.0)
        assert oracle.hubble(0.25, c) == pytest.approx(math.sqrt(0.25 ** p), rel=1e-15)


def test_einstein_de_sitter_closed_form():
    # Omega_M = 1: a^{3/2} = a0^{3/2} + (3/2) H0 t
    c = Cosmology(0.0, 1.0, 0.0, 0.0, 1.0)
    t, a = _integrate(c, A0, 0.05, 200)
    exact = (A0 ** 1.5 + 1.5 * t) ** (2.0 / 3.0)
    assert np.max(np.abs(a / exact - 1.0)) < 1e-12


def test_flat_lcdm_sinh_form():
    c = Cosmology(0.0, 0.3, 0.0, 0.7, 1.0)

    def age(a):
        return 2.0 / (3.0 * math.sqrt(0.7)) * math.asinh(math.sqrt(0.7 / 0.3) * a ** 1.5)

    def a_of(tabs):
        return (0.3 / 0.7) ** (1.0 / 3.0) * math.sinh(1.5 * math.sqrt(0.7) * tabs) ** (2.0 / 3.0)

    T = age(1.0) - age(A0)
    t, a = _integrate(c, A0, T, 2000)
    exact = np.array([a_of(age(A0) + ti) for ti in t])
    assert abs(a[-1] - 1.0) < 1e-11
    assert np.max(np.abs(a / exact - 1.0)) < 1e-11


def test_milne_linear():
    c = Cosmology(0.0, 0.0, 1.0, 0.0, 1.3)
    t, a = _integrate(c, 0.2, 2.0, 50)
    assert np.max(np.abs(a / (0.2 + 1.3 * t) - 1.0)) < 1e-14


def test_radiation():
    c = Cosmology(1.0, 0.0, 0.0, 0.0, 1.0)
    t, a = _integrate(c, 0.1, 0.3, 1000)
    assert np.max(np.abs(a / np.sqrt(0.01 + 2.0 * t) - 1.0)) < 1e-12


def test_de_sitter():
    c = Cosmology(0.0, 0.0, 0.0, 1.0, 0.7)
    t, a = _integrate(c, 0.5, 3.0, 200)
    assert np.max(np.abs(a / (0.5 * np.exp(0.7 * t)) - 1.0)) < 1e-12


def test_rk4_fourth_order():
    c = Cosmology(0.0, 1.0, 0.0, 0.0, 1.0)
    exact = (A0 ** 1.5 + 1.5 * 0.002) ** (2.0 / 3.0)
    e1 = abs(oracle.friedmann_advance(A0, 0.002, c, 4) - exact)
    e2 = abs(oracle.friedmann_advance(A0, 0.002, c, 8) - exact)
    assert 12.0 < e1 / e2 < 20.0


def test_recollapse_raises():
    # closed matter universe: E^2 = 2 a^-3 - a^-2 < 0 beyond a = 2
    c = Cosmology(0.0, 2.0, -1.0, 0.0, 1.0)
    with pytest.raises(oracle.FriedmannError):
        oracle.hubble(2.5, c)
