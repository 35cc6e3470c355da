"""Pins of the oracle's complete elliptic integrals K, E (Gauss AGM)."""
import math
import os

import numpy as np
import scipy.special as sp

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "special_values.txt")


def golden():
    out = {}
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()[:2]
            out[k] = float(v)
    return out


def test_zero_parameter():
    K, E = oracle.ellipke(np.array([0.0]))
    assert abs(K[0] - math.pi / 2) < 1e-15 and abs(E[0] - math.pi / 2) < 1e-15


def test_half_parameter_closed_form():
    g = golden()
    K, E = oracle.ellipke(np.array([0.5]))
    assert abs(K[0] - g["K_half"]) < 1e-14
    assert abs(E[0] - g["E_half"]) < 1e-14
    # Gamma-function closed form of the lemniscate case
    assert abs(K[0] - math.gamma(0.25) ** 2 / (4 * math.sqrt(math.pi))) < 1e-14


def test_legendre_relation():
    m = np.linspace(0.01, 0.99, 99)
    K, E = oracle.ellipke(m)
    Kc, Ec = oracle.ellipke(1.0 - m)
    assert np.max(np.abs(E * Kc + Ec * K - K * Kc - math.pi / 2)) < 1e-13


def test_against_scipy_including_near_one():
    m = np.concatenate([np.linspace(0.0, 0.999, 500), 1.0 - np.logspace(-3, -12, 40)])
    mc = np.concatenate([1.0 - m[:500], np.logspace(-3, -12, 40)])
    K, E = oracle.ellipke(m, mc)
    Ks = sp.ellipkm1(mc)
    Es = sp.ellipe(m)
    assert np.max(np.abs(K / Ks - 1)) < 1e-14
    assert np.max(np.abs(E / Es - 1)) < 1e-14
