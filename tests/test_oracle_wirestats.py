"""Pins of the oracle's per-wire statistics (Flux Jumps Propagation and
Quenches Propagation sections: per-wire maximum temperature, maximum Joule
power density, Joule heat from an onset): closed forms of an ohmic loop and
the consistency of the per-wire heat with the step diagnostics."""
import math

import numpy as np

import oracle
from paper_2403_07666_b300.workloads import MATERIAL, solenoid

P = dict(MATERIAL)
NODRIVE = {"dt": 1e-5, "ramp_rate": 0.0, "I_max": 0.0, "Ba_rate": 0.0, "Ba_max": 0.0, "Ba_waveform": 0}


def _one_loop(r=0.02, h=5e-4, **over):
    p = dict(P, thermal=0, jc_model=1)
    p.update(over)
    geom = {"kind": "list", "r": np.array([r]), "z": np.array([0.0]), "h": np.array([h]), "block": 1}
    return oracle.build(geom, p, np.ones(1), np.zeros(1), np.array([0]), np.array([False]))


def test_ohmic_loop_heat_is_geometric_sum():
    """A free Cu loop decays as I_{k+1} = I_k L / (L + dt R) under the
    linearly-implicit step, so its heat by the rectangle rule is
    dt R I0^2 (1 - g^(2n)) / (1 - g^2), g = L / (L + dt R)."""
    r, h = 0.02, 5e-4
    c = _one_loop(r, h)
    I0 = 7.0
    c.I = np.array([I0])
    a = h * h
    R = 2 * math.pi * r * P["rho_n"] / a
    L = c.M[0, 0]
    dt = NODRIVE["dt"]
    g = L / (L + dt * R)
    n = 40
    for _ in range(n):
        c.step(NODRIVE)
    Q = dt * R * I0 ** 2 * (1 - g ** (2 * n)) / (1 - g * g)
    st = c.wire_stats()
    assert abs(st[0, 0] - Q) <= 1e-12 * Q
    # maximum power density: the first step's rho_n J^2; T stays at the bath (no thermal model)
    assert abs(st[2, 0] - P["rho_n"] * (I0 / a) ** 2) <= 1e-12 * st[2, 0]
    assert st[1, 0] == P["T_bath"]
    # a Cu loop never meets the filament criteria
    assert np.all(st[3:7, 0] == -1.0)


def test_wire_heat_sums_to_diagnostic_joule_power():
    """Sum over wires of Q_total = sum over steps of dt x the diagnostic Joule
    power (computed separately, over all elements, for the record)."""
    w = solenoid("ws", 3, 5, 4, 21, ramp_rate=2e4, material=dict(MATERIAL, Jc0=2e8))
    c = oracle.build(w.geometry, w.material, w.jc_factor, w.strain, w.mat)
    recs = [c.step(w.drive) for _ in range(60)]
    dt = w.drive["dt"]
    total = sum(dt * rec[4] for rec in recs)
    st = c.wire_stats()
    assert total > 0
    assert abs(st[0].sum() - total) <= 1e-12 * total
    # running maxima over start-of-step states: the start state of step k + 1 is the
    # end state of step k, whose maximum temperature the record holds
    assert np.all(st[1] >= P["T_bath"] - 1e-12)
    expect = max(P["T_bath"], max(rec[5] for rec in recs[:-1]))
    assert abs(st[1].max() - expect) <= 1e-12 * expect
    assert np.all(st[0] >= 0)


def test_onset_heat_is_recorded_before_the_onset_step():
    """A wire driven past |J/Jc| = 1: Q_at_jump equals the heat accumulated over
    the steps before first_jump, and later heat only adds to Q_total."""
    mtl = dict(MATERIAL, Jc0=2e7, thermal=0)
    w = solenoid("jump", 2, 3, 4, 23, ramp_rate=5e5, material=mtl)
    c = oracle.build(w.geometry, w.material, w.jc_factor, w.strain, w.mat)
    snap = []
    for _ in range(40):
        snap.append(c.Q_total.copy())
        c.step(w.drive)
    st = c.wire_stats()
    jumped = np.nonzero(c.first_jump >= 0)[0]
    assert len(jumped) > 0
    for wi in jumped:
        k = c.first_jump[wi]
        assert st[3, wi] == snap[k][wi]
        assert st[0, wi] >= st[3, wi]
    never = np.nonzero(c.first_jump < 0)[0]
    assert np.all(st[3, never] == -1.0)
