"""Pins of the oracle's Lorentz hoop strain (Flux Jumps Propagation section:
the electromagnetic strain produced by the Lorentz force enters Jc(eps)).

eps_e = eps0_e + r_e J_e B_z,e / Y_eff is checked against the magnetic pressure
on a long thin solenoid (Maxwell stress: the outward force per unit bore area
is B_in^2 / (2 mu0)), against the mirror symmetry of a coil whose drive is
reversed, and against the static-strain limit."""
import math

import numpy as np

import oracle
from oracle.field import field_from_flux
from oracle.geometry import solenoid_elements
from oracle.inductance import operator_rows
from oracle.step import OracleCoil
from paper_2403_07666_b300.workloads import MATERIAL, random_coil

MU0 = 4e-7 * math.pi


def test_hoop_strain_sums_to_magnetic_pressure():
    """A single-layer 1000-turn solenoid with a uniform J in every wire: over
    the midplane turn, sum_e a_e (eps_e - eps0_e) Y / r_e = sum J B_z a is the
    radial force of one pitch of winding per unit circumference, p B_in^2/(2 mu0),
    B_in = mu0 J d^2 / p times the finite-length factor (L/2)/sqrt((L/2)^2 + R^2)."""
    NT, n = 1000, 4
    r_in, pitch, d = 0.020, 0.9e-3, 0.8e-3
    geo = solenoid_elements(1, NT, n, r_in, pitch, d)
    Y = 5e10
    p = dict(MATERIAL, thermal=0, Y_eff=Y)
    N = geo["N"]
    eps0 = np.full(N, -0.002)
    c = OracleCoil(geo, p, np.ones(N), eps0, np.ones(N, dtype=np.int64), M=np.zeros((0, 0)))
    J = 3e8
    c.I = J * geo["area"]
    t = NT // 2
    rows = np.arange(t * n * n, (t + 1) * n * n)
    phi = np.zeros(N)          # the r-stencil of a one-layer turn only reads that turn
    phi[rows] = operator_rows(geo["r"], geo["z"], geo["h"], rows) @ c.I
    _, Bz = field_from_flux(geo, phi)
    eps = c.strain_now(Bz)
    force = np.sum(geo["area"][rows] * (eps[rows] - eps0[rows]) * Y / geo["r"][rows])
    L = NT * pitch
    R = r_in + 0.5 * (pitch - d) + 0.5 * d
    B_in = MU0 * J * d * d / pitch * (0.5 * L) / math.hypot(0.5 * L, R)
    expect = pitch * B_in ** 2 / (2.0 * MU0)
    assert abs(force / expect - 1.0) < 2e-3, force / expect
    # tension at the bore side of the winding (B_z > 0 there, J > 0)
    assert np.all(eps[rows] - eps0[rows] > 0.0)


def _run(w, steps, drive):
    c = oracle.build(w.geometry, w.material, w.jc_factor, w.strain, w.mat)
    for _ in range(steps):
        c.step(drive)
    return c


def test_reversed_drive_mirrors_the_trajectory():
    """r J B_z is even under I -> -I (B_z changes sign with the currents): a coil
    ramped the other way follows -I exactly, also with the Lorentz strain."""
    w = random_coil(41, 2, 3, 4, ramp_rate=5e5, material=dict(MATERIAL, Jc0=2e7, Y_eff=2e8))
    rev = dict(w.drive, ramp_rate=-w.drive["ramp_rate"], I_max=w.drive["I_max"])
    a = _run(w, 25, w.drive)
    b = _run(w, 25, rev)
    assert np.max(np.abs(a.I + b.I)) <= 1e-12 * np.max(np.abs(a.I))
    assert np.max(np.abs(a.u_T - b.u_T)) <= 1e-12 * np.max(a.u_T)


def test_lorentz_strain_changes_jc_in_the_expected_direction():
    """Compressive static strain relaxed by the tensile hoop strain of the
    inner layer raises Jc there; Y_eff -> infinity gives the static strain."""
    mtl = dict(MATERIAL, Jc0=2e7)
    w = random_coil(42, 3, 4, 4, ramp_rate=5e5, material=mtl)
    w.strain[:] = -0.003
    wl = random_coil(42, 3, 4, 4, ramp_rate=5e5, material=dict(mtl, Y_eff=2e8))
    wl.strain[:] = -0.003
    ws = random_coil(42, 3, 4, 4, ramp_rate=5e5, material=dict(mtl, Y_eff=1e300))
    ws.strain[:] = -0.003
    a, b, s = _run(w, 12, w.drive), _run(wl, 12, wl.drive), _run(ws, 12, ws.drive)
    assert np.array_equal(a.I, s.I)
    pa = a.pointwise(0.0)
    pb = b.pointwise(0.0)
    geo = b.geo
    inner = (geo["i_r"] < geo["n"]) & (pb["Bz"] > 0) & (b.I > 0) & (b.mat == 1)
    assert inner.sum() > 4
    assert np.all(pb["eps"][inner] > -0.003)
    assert np.all(np.abs(pb["eps"][inner]) < 0.003)
    # Jc of the same state with and without the hoop strain
    from oracle.constitutive import critical_current
    jc_static = critical_current(pb["Bmag"], pb["T"], b.strain, b.jc_factor, b.mat, b.p)
    assert np.all(pb["Jc"][inner] > jc_static[inner])
    # and the coupled run departs from the static-strain run
    assert np.max(np.abs(b.I - a.I)) > 1e-6 * np.max(np.abs(a.I))
    assert pa["eps"] is a.strain
