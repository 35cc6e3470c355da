"""Pins of the oracle's loop inductances and dense operator."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle.inductance import MU0, near_average, mutual_point, self_inductance, GMD_SQUARE


def test_far_field_dipole_limit():
    a, b = 0.02, 0.03
    # the closed form cancels like 16/k^4 for distant loops, so d stays moderate
    for d in (0.3, 1.0, 3.0):
        M = mutual_point(a, 0.0, b, d)
        dip = MU0 * math.pi * a * a * b * b / (2 * d ** 3)
        # leading correction is O((a^2 + b^2) / d^2)
        assert abs(M / dip - 1) < 5 * (a * a + b * b) / d ** 2


def test_near_field_log_limit():
    a = 0.02
    for delta in (1e-5, 1e-6):
        M = mutual_point(a, 0.0, a, delta)
        ref = MU0 * a * (math.log(8 * a / delta) - 2)
        assert abs(M / ref - 1) < 1e-6


def test_symmetry_of_point_formula():
    rng = np.random.default_rng(1)
    r1, r2 = rng.uniform(0.01, 0.1, (2, 50))
    z1, z2 = rng.uniform(-0.05, 0.05, (2, 50))
    assert np.max(np.abs(mutual_point(r1, z1, r2, z2) / mutual_point(r2, z2, r1, z1) - 1)) < 1e-14


def test_loop_field_on_axis_closed_form():
    a, I = 0.03, 7.0
    z = np.linspace(-0.1, 0.1, 21)
    Br, Bz = oracle.loop_field(a, 0.01, I, np.zeros_like(z), z)
    ref = MU0 * I * a * a / (2 * (a * a + (z - 0.01) ** 2) ** 1.5)
    assert np.max(np.abs(Bz / ref - 1)) < 1e-13
    assert np.max(np.abs(Br)) == 0.0


def test_loop_field_against_biot_savart_quadrature():
    a, I, z0 = 0.025, 3.0, 0.004
    for (r, z) in ((0.01, 0.0), (0.04, 0.02), (0.024, 0.003)):
        def dB(phi, comp):
            # current element a dphi (-sin, cos, 0) at (a cos, a sin, z0); field point (r, 0, z)
            rx, ry, rz = r - a * math.cos(phi), -a * math.sin(phi), z - z0
            d3 = (rx * rx + ry * ry + rz * rz) ** 1.5
            dlx, dly = -a * math.sin(phi), a * math.cos(phi)
            cx = dly * rz
            cz = dlx * ry - dly * rx
            return (cx if comp == 0 else cz) / d3
        Bx = MU0 * I / (4 * math.pi) * integrate.quad(dB, 0, 2 * math.pi, args=(0,), epsabs=0, epsrel=1e-13, limit=200)[0]
        Bzq = MU0 * I / (4 * math.pi) * integrate.quad(dB, 0, 2 * math.pi, args=(1,), epsabs=0, epsrel=1e-13, limit=200)[0]
        Br, Bz = oracle.loop_field(a, z0, I, np.array([r]), np.array([z]))
        assert abs(Br[0] - Bx) < 1e-10 * abs(Bzq) and abs(Bz[0] / Bzq - 1) < 1e-10


def test_mutual_equals_flux_of_point_field():
    """M_12 = (1/I) * flux of loop 1's field through the disk of loop 2."""
    a, b, dz = 0.02, 0.031, 0.007
    I = 1.0
    flux = integrate.quad(lambda rho: oracle.loop_field(a, 0.0, I, np.array([rho]), np.array([dz]))[1][0]
                          * 2 * math.pi * rho, 0.0, b, epsabs=0, epsrel=1e-12, limit=200)[0]
    assert abs(mutual_point(a, 0.0, b, dz) / flux - 1) < 1e-10


def test_gmd_square_constant():
    """exp(mean of ln|x - y|) over two uniform points of the unit square."""
    f = lambda v, u: 4 * (1 - u) * (1 - v) * 0.5 * math.log(u * u + v * v)
    val = integrate.dblquad(f, 0, 1, 0, 1, epsabs=1e-13, epsrel=1e-13)[0]
    assert abs(math.exp(val) - GMD_SQUARE) < 2e-6


def test_near_average_tends_to_point_formula_far_away():
    h = 1e-4
    M = near_average(np.array([0.02]), np.array([0.0]), np.array([h]),
                     np.array([0.021]), np.array([0.004]), np.array([h]))
    P = mutual_point(0.02, 0.0, 0.021, 0.004)
    assert abs(M[0] / P - 1) < 1e-5          # O((h/d)^2) averaging correction


def test_self_term_is_mean_of_point_formula_over_square():
    """Self term vs a quasi-Monte-Carlo mean of the point formula over point
    pairs of one square (the self term is the flux-averaged mutual term)."""
    from scipy.stats import qmc
    r, h = 0.03, 2e-4
    pts = qmc.Sobol(4, seed=3).random(2 ** 18)
    M = mutual_point(r + h * (pts[:, 0] - 0.5), h * (pts[:, 1] - 0.5),
                     r + h * (pts[:, 2] - 0.5), h * (pts[:, 3] - 0.5))
    assert abs(np.mean(M) / self_inductance(r, h) - 1) < 3e-4


def test_near_average_adjacent_squares_against_qmc():
    from scipy.stats import qmc
    r, h = 0.025, 2e-4
    pts = qmc.Sobol(4, seed=5).random(2 ** 16)
    M = mutual_point(r + h * (pts[:, 0] - 0.5), h * (pts[:, 1] - 0.5),
                     r + h + h * (pts[:, 2] - 0.5), h * (pts[:, 3] - 0.5))
    G = near_average(np.array([r]), np.array([0.0]), np.array([h]),
                     np.array([r + h]), np.array([0.0]), np.array([h]))
    assert abs(np.mean(M) / G[0] - 1) < 2e-4


def test_full_operator_symmetric_positive_definite():
    geo = oracle.solenoid_elements(3, 4, 4, 0.02, 0.9e-3, 0.8e-3)
    M = oracle.assemble_M(geo["r"], geo["z"], geo["h"])
    assert np.array_equal(M, M.T)
    ev = np.linalg.eigvalsh(M)
    assert ev.min() > 0
    assert np.all(np.diag(M) > 0) and np.all(M > 0)


def test_operator_rows_equal_assembled_rows():
    from oracle.inductance import operator_rows
    geo = oracle.solenoid_elements(3, 4, 4, 0.02, 0.9e-3, 0.8e-3)
    M = oracle.assemble_M(geo["r"], geo["z"], geo["h"])
    rows = np.array([0, 17, 95, 191])
    R = operator_rows(geo["r"], geo["z"], geo["h"], rows)
    assert np.array_equal(R, M[rows])
