"""Pins of the oracle's Jc(B, T, eps) and E-J law (reduced special cases)."""
import math

import numpy as np

import oracle
from paper_2403_07666_b300.workloads import MATERIAL

P = dict(MATERIAL)


def jc(B, T, eps=0.0, f=1.0):
    return oracle.critical_current(np.array([B]), np.array([T]), np.array([eps]),
                                   np.array([f]), np.array([1]), P)[0]


def test_jc_reduced_cases():
    base = jc(0.0, 0.0)
    assert abs(base - P["Jc0"] / math.sqrt(0.1)) < 1e-6 * base      # every factor is 1
    # temperature factor alone at B = 0: (1 - 0.75)^1.5 = 1/8
    assert abs(jc(0.0, 13.5) / base - 0.125) < 1e-14
    # field factor alone at T = 0: (1 - 7/28)^2 * sqrt(0.1 / 7.1)
    assert abs(jc(7.0, 0.0) / base - 0.5625 * math.sqrt(0.1 / 7.1)) < 1e-14
    # Bc2(T) = Bc2(0) (1 - t^2): at T = Tc/2, Bc2 = 21 T; at B = 10.5 the field factor is 1/4
    assert abs(jc(10.5, 9.0) / (base * 0.5 ** 1.5 * 0.25 * math.sqrt(0.1 / 10.6)) - 1) < 1e-13
    assert jc(21.0, 9.0) == 0.0 and jc(0.0, 18.0) == 0.0 and jc(30.0, 4.2) == 0.0
    # strain factor 1 - C |eps|^p equals 1/2 at |eps| = (1/1800)^(1/1.7)
    e_half = (0.5 / 900.0) ** (1 / 1.7)
    assert abs(jc(0.0, 0.0, -e_half) / base - 0.5) < 1e-13
    assert jc(0.0, 0.0, -0.02) == 0.0                                  # clamped at 0
    assert abs(jc(0.0, 0.0, f=1.3) / base - 1.3) < 1e-14


def ej(I, Jc, mat=1, r=0.02, a=4e-8, p=P):
    return oracle.ej_terms(np.array([I]), np.array([Jc]), np.array([mat]), np.array([r]),
                           np.array([a]), p)


def test_power_law_regime():
    a, Jc = 4e-8, 1e11
    for x in (0.3, 0.6, 0.9):
        t = ej(x * Jc * a, Jc, a=a)
        # s << 1: E = E0 (J/Jc)^n to relative O(s)
        assert abs(t["E"][0] / (P["E0"] * x ** P["n"]) - 1) < 1e-5


def test_parallel_law_limits():
    a = 4e-8
    t = ej(2.0, 0.0, a=a)                       # Jc = 0: normal state
    assert abs(t["rho"][0] - P["rho_n"]) < 1e-24 and abs(t["E"][0] - P["rho_n"] * 2.0 / a) < 1e-12
    t = ej(0.0, 1e11, a=a)                      # J = 0: no field, no loss
    assert t["E"][0] == 0.0 and t["G"][0] == 0.0 and t["q"][0] == 0.0
    # s = 1 when J = Jc and E0 = Jc rho_n: rho = rho_n / 2
    p2 = dict(P, E0=1e11 * P["rho_n"])
    t = ej(1e11 * a, 1e11, a=a, p=p2)
    assert abs(t["rho"][0] / P["rho_n"] - 0.5) < 1e-14
    # deep flux flow, s >> 1: rho -> rho_n
    t = ej(10 * 1e11 * a, 1e11, a=a)
    assert abs(t["rho"][0] / P["rho_n"] - 1) < 1e-12
    t = ej(3.0, 5e10, mat=0, a=a)               # Cu element: ohmic
    assert abs(t["E"][0] / (P["rho_n"] * 3.0 / a) - 1) < 1e-15


def test_loop_derivative_against_finite_difference():
    a, r = 4e-8, 0.021
    for Jc, x in ((1e11, 0.95), (1e11, 1.02), (1e11, 1.6), (2e9, 3.0), (1e11, 0.5)):
        I = x * Jc * a
        t = ej(I, Jc, a=a, r=r)
        hI = 1e-7 * I
        Ep = ej(I + hI, Jc, a=a, r=r)["E"][0]
        Em = ej(I - hI, Jc, a=a, r=r)["E"][0]
        fd = 2 * math.pi * r * (Ep - Em) / (2 * hI)
        assert abs(t["G"][0] / fd - 1) < 1e-6
        assert t["q"][0] >= 0.0
