"""Pins of the oracle's field stencil and coil geometry."""
import math

import numpy as np

import oracle
from oracle.inductance import MU0, mutual_point


def _geo(NL=3, NT=4, n=4):
    return oracle.solenoid_elements(NL, NT, n, 0.02, 0.9e-3, 0.8e-3)


def test_geometry_element_order_and_positions():
    geo = _geo(2, 3, 2)
    # element e = (t*NL + l)*n^2 + b*n + a: wire (l=1, t=2), a=1, b=0
    e = (2 * 2 + 1) * 4 + 0 * 2 + 1
    h = 0.4e-3
    assert abs(geo["r"][e] - (0.02 + 0.05e-3 + 0.9e-3 + 1.5 * h)) < 1e-15
    assert abs(geo["z"][e] - (-1.5 * 0.9e-3 + 0.05e-3 + 2 * 0.9e-3 + 0.5 * h)) < 1e-15
    # the coil is symmetric about z = 0
    assert abs(geo["z"].min() + geo["z"].max()) < 1e-15


def test_uniform_applied_field_exact():
    geo = _geo()
    Ba = 0.37
    Br, Bz = oracle.field_from_flux(geo, math.pi * geo["r"] ** 2 * Ba)
    assert np.max(np.abs(Bz - Ba)) < 1e-13 and np.max(np.abs(Br)) < 1e-13


def test_stencil_of_external_loop_flux_matches_point_field():
    """Flux of a distant loop sampled at the element centres, differentiated by
    the stencil, vs the loop's elliptic point field at those centres."""
    geo = _geo(4, 6, 4)
    a, z0, I = 0.018, 0.006, 50.0
    phi = mutual_point(geo["r"], geo["z"], a, z0) * I
    Br, Bz = oracle.field_from_flux(geo, phi)
    Brr, Bzr = oracle.loop_field(a, z0, I, geo["r"], geo["z"])
    scale = np.max(np.hypot(Brr, Bzr))
    assert np.max(np.abs(Bz - Bzr)) < 2e-3 * scale
    assert np.max(np.abs(Br - Brr)) < 2e-3 * scale


def test_thick_solenoid_on_axis_closed_form():
    """Sum of the element point loops vs the closed-form axial field of
    uniformly-filled rectangular windings (each wire square)."""
    geo = _geo(4, 8, 4)
    J = 1e7
    I = J * geo["area"]
    zs = np.linspace(-0.01, 0.01, 9)
    Bloops = np.zeros_like(zs)
    for e in range(geo["N"]):
        Bloops += oracle.loop_field(geo["r"][e], geo["z"][e], I[e], np.zeros_like(zs), zs)[1]
    Bref = np.zeros_like(zs)
    d, p, g = 0.8e-3, 0.9e-3, 0.1e-3
    for l in range(4):
        r1 = 0.02 + g / 2 + l * p
        r2 = r1 + d
        for t in range(8):
            z1 = -4 * p + g / 2 + t * p
            z2 = z1 + d
            def F(u):
                return u * np.log((r2 + np.sqrt(r2 * r2 + u * u)) / (r1 + np.sqrt(r1 * r1 + u * u)))
            Bref += MU0 * J / 2 * (F(zs - z1) - F(zs - z2))
    assert np.max(np.abs(Bloops / Bref - 1)) < 2e-3       # O((h / r)^2) midpoint error
