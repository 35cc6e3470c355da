"""Pins of the oracle's coupled step: KKT solve, brute-force loops, Bean's
critical state and the circuit energy balance."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from paper_2403_07666_b300.workloads import MATERIAL, solenoid

P = dict(MATERIAL)
NODRIVE = {"dt": 1e-5, "ramp_rate": 0.0, "I_max": 0.0, "Ba_rate": 0.0, "Ba_max": 0.0, "Ba_waveform": 0}


def _list_coil(r, z, h, block, constrained, mat, **over):
    p = dict(P, thermal=0, jc_model=1)
    p.update(over)
    geom = {"kind": "list", "r": np.array(r), "z": np.array(z), "h": np.array(h), "block": block}
    N = len(r)
    return oracle.build(geom, p, np.ones(N), np.zeros(N), np.array(mat), np.array(constrained, bool))


def test_kkt_residual_and_constraint():
    w = solenoid("t", 3, 4, 4, 11, ramp_rate=1e4)
    c = oracle.build(w.geometry, w.material, w.jc_factor, w.strain, w.mat)
    for _ in range(3):
        c.step(w.drive)
    L = c.last
    B = c.geo["block"]
    Pu = np.repeat(L["u"], B)
    res = L["A"] @ L["Idot"] - Pu + L["R"]
    scale = np.abs(L["A"]).max() * np.abs(L["Idot"]).max() + np.abs(L["R"]).max()
    assert np.max(np.abs(res)) < 1e-12 * scale
    sums = L["Idot"].reshape(-1, B).sum(axis=1)
    assert np.max(np.abs(sums - L["c"])) < 1e-10 * np.abs(L["c"]).max()
    # the step keeps every turn's current on the ramp
    assert np.max(np.abs(c.I.reshape(-1, B).sum(axis=1) - 3e-5 * 1e4)) < 1e-12


def test_two_free_ohmic_loops_closed_form():
    c = _list_coil([0.020, 0.0215], [0.0, 0.0007], [5e-4, 5e-4], 1, [0, 0], [0, 0])
    I0 = np.array([3.0, -1.0])
    c.I = I0.copy()
    M = c.M
    Rd = 2 * math.pi * np.array([0.020, 0.0215]) * P["rho_n"] / 2.5e-7
    dt = NODRIVE["dt"]
    # explicit 2 x 2 inverse of (M + dt R)
    a, b, cc, d = M[0, 0] + dt * Rd[0], M[0, 1], M[1, 0], M[1, 1] + dt * Rd[1]
    inv = np.array([[d, -b], [-cc, a]]) / (a * d - b * cc)
    step = np.eye(2) - dt * inv @ np.diag(Rd)
    I = I0.copy()
    for k in range(60):
        c.step(NODRIVE)
        I = step @ I
    assert np.max(np.abs(c.I - I)) < 1e-13 * np.abs(I0).max()
    # continuous solution exp(-M^-1 R t): first-order agreement
    errs = []
    for dtk in (2e-6, 1e-6):
        cc2 = _list_coil([0.020, 0.0215], [0.0, 0.0007], [5e-4, 5e-4], 1, [0, 0], [0, 0])
        cc2.I = I0.copy()
        dr = dict(NODRIVE, dt=dtk)
        n = int(round(2e-4 / dtk))
        for _ in range(n):
            cc2.step(dr)
        exact = expm(-np.linalg.solve(M, np.diag(Rd)) * 2e-4) @ I0
        errs.append(np.max(np.abs(cc2.I - exact)) / np.abs(I0).max())
    assert errs[1] < 0.05 and 1.7 < errs[0] / errs[1] < 2.3


def _four_loops(mat):
    r = [0.020, 0.0205, 0.020, 0.0205]
    z = [0.0, 0.0, 0.0008, 0.0008]
    return _list_coil(r, z, [4e-4] * 4, 2, [1, 1], mat, Jc0=2e8)


def test_four_loops_two_turns_dense_kkt():
    """2 turns x 2 elements on a transport ramp: the 6 x 6 KKT solved by
    numpy.linalg.solve every step (all-Cu: linear, written out by hand)."""
    c = _four_loops([0, 0, 0, 0])
    drive = dict(NODRIVE, ramp_rate=1e4, I_max=1e9)
    r = np.array([0.020, 0.0205, 0.020, 0.0205])
    Rd = 2 * math.pi * r * P["rho_n"] / 1.6e-7
    Pm = np.array([[1, 0], [1, 0], [0, 1], [0, 1]], float)
    M = c.M
    I = np.zeros(4)
    t = 0.0
    dt = drive["dt"]
    for k in range(40):
        K = np.zeros((6, 6))
        K[:4, :4] = M + dt * np.diag(Rd)
        K[:4, 4:] = -Pm
        K[4:, :4] = Pm.T
        It1 = 1e4 * (t + dt)
        rhs = np.concatenate([-Rd * I, (It1 - Pm.T @ I) / dt])
        sol = np.linalg.solve(K, rhs)
        I = I + dt * sol[:4]
        t += dt
        rec = c.step(drive)
        assert abs(rec[2] - sol[4:].sum()) < 1e-11 * abs(sol[4:]).max()
    assert np.max(np.abs(c.I - I)) < 1e-12 * np.abs(I).max()


def test_four_loops_superconducting_dense_kkt():
    """Same with one filament element per turn: E and G from the (separately
    pinned) E-J law, the KKT assembled and solved densely here."""
    mat = np.array([1, 0, 1, 0])
    c = _four_loops(mat)
    drive = dict(NODRIVE, ramp_rate=3e5, I_max=1e9)
    r = np.array([0.020, 0.0205, 0.020, 0.0205])
    Pm = np.array([[1, 0], [1, 0], [0, 1], [0, 1]], float)
    I = np.zeros(4)
    t, dt = 0.0, drive["dt"]
    p = dict(c.p)
    for k in range(60):
        Jc = np.where(mat == 1, p["Jc0"], 0.0)
        tm = oracle.ej_terms(I, Jc, mat, r, np.full(4, 1.6e-7), p)
        K = np.zeros((6, 6))
        K[:4, :4] = c.M + dt * np.diag(tm["G"])
        K[:4, 4:] = -Pm
        K[4:, :4] = Pm.T
        rhs = np.concatenate([-2 * math.pi * r * tm["E"], (3e5 * (t + dt) - Pm.T @ I) / dt])
        sol = np.linalg.solve(K, rhs)
        I = I + dt * sol[:4]
        t += dt
        c.step(drive)
    assert np.max(np.abs(c.I - I)) < 1e-10 * np.abs(I).max()
    assert np.max(np.abs(I[[0, 2]])) > 1.0        # the filament elements carry the ramp


def test_bean_tube_full_penetration_moment():
    """Thick tube of free loops (r in [a1, a2], length 4 mm), constant Jc,
    n = 500, axial field ramped beyond full penetration.  Bean's critical
    state has J = -Jc everywhere, so m = -pi Jc L (a2^3 - a1^3) / 3 at any
    length: m / V -> -Jc (a2^3 - a1^3) / (3 (a2^2 - a1^2)), up to the
    creep factor (E/E0)^(1/n) ~ 1.005 at the ramp's electric field."""
    a1, a2 = 2e-3, 3e-3
    geom = {"kind": "solenoid", "n_layers": 1, "n_turns": 4, "n_sub": 5, "r_in": a1,
            "pitch": a2 - a1, "wire_d": a2 - a1, "transport": 0}
    Jc0 = 1e9
    p = dict(P, thermal=0, jc_model=1, Jc0=Jc0, n=500.0)
    N = 100
    c = oracle.build(geom, p, np.ones(N), np.zeros(N), np.ones(N, int))
    # the per-step field increment (5e-4 T) stays below mu0 h Jc / n
    drive = dict(NODRIVE, dt=5e-4, Ba_rate=1.0, Ba_max=10.0, Ba_waveform=1)
    for _ in range(2400):
        rec = c.step(drive)
    V = math.pi * (a2 * a2 - a1 * a1) * 4 * (a2 - a1)
    bean = -Jc0 * (a2 ** 3 - a1 ** 3) / (3 * (a2 * a2 - a1 * a1))
    assert abs((rec[3] / V) / bean - 1) < 0.01
    J = c.I / c.geo["area"]
    assert np.all(np.abs(J / -Jc0 - 1) < 0.01)        # fully penetrated critical state


def test_energy_balance_first_order():
    """Work of the transport source and of the applied field equals Joule heat
    plus magnetic energy 1/2 I^T M I, to first order in dt."""
    imb = []
    for dt in (2e-5, 1e-5):
        w = solenoid("e", 2, 3, 4, 5, ramp_rate=2e4, dt=dt, Ba_rate=20.0, Ba_max=10.0, Ba_waveform=1)
        c = oracle.build(w.geometry, dict(w.material, thermal=0), w.jc_factor, w.strain, w.mat)
        n = int(round(2e-3 / dt))
        Ein = Ejoule = 0.0
        m_prev = It_prev = 0.0
        for _ in range(n):
            rec = c.step(w.drive)
            # the current is linear inside a step: midpoint current times the step's voltage
            Ein += dt * (0.5 * (It_prev + rec[1]) * rec[2] - w.drive["Ba_rate"] * 0.5 * (m_prev + rec[3]))
            Ejoule += dt * rec[4]
            m_prev, It_prev = rec[3], rec[1]
        Emag = 0.5 * c.I @ c.M @ c.I
        assert Ejoule > 0.02 * Ein
        imb.append((Ein - Ejoule - Emag) / Ein)
    assert abs(imb[1]) < 2e-2
    assert 1.6 < imb[0] / imb[1] < 2.4


def test_triangle_field_drive_values():
    """Waveform 2 of the applied field (Numerical Algorithm section: ramping
    external field): a triangle 0 -> +Ba_max -> -Ba_max -> 0 of slope Ba_rate,
    period P = 4 Ba_max / Ba_rate, repeated.  Values at the corners, at the
    quarter points of each leg, across a period boundary, and the sign of the
    slope on each leg."""
    amp, rate = 0.1, 4.0
    d = {"dt": 1e-4, "ramp_rate": 0.0, "I_max": 0.0, "Ba_rate": rate, "Ba_max": amp, "Ba_waveform": 2}
    per = 4 * amp / rate
    expect = {0.0: 0.0, per / 8: amp / 2, per / 4: amp, 3 * per / 8: amp / 2, per / 2: 0.0,
              5 * per / 8: -amp / 2, 3 * per / 4: -amp, 7 * per / 8: -amp / 2,
              per: 0.0, per + per / 8: amp / 2, 2 * per + 3 * per / 4: -amp}
    for t, want in expect.items():
        It, Ba = oracle.drive_values(t, d)
        assert It == 0.0
        assert abs(Ba - want) < 1e-12 * amp, (t, Ba, want)
    eps = 1e-6 * per
    for t0, slope in ((per / 8, rate), (per / 2, -rate), (7 * per / 8, rate), (per + per / 16, rate)):
        s = (oracle.drive_values(t0 + eps, d)[1] - oracle.drive_values(t0 - eps, d)[1]) / (2 * eps)
        assert abs(s - slope) < 1e-6 * rate, (t0, s, slope)
    # the ramp waveform caps at Ba_max and the transport ramp at I_max
    d1 = dict(d, Ba_waveform=1, ramp_rate=10.0, I_max=3.0)
    assert oracle.drive_values(0.01, d1) == (0.1, 0.04)
    assert oracle.drive_values(1.0, d1) == (3.0, amp)
