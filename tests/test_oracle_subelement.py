"""Pins of the oracle's subelement decoupling (Numerical Algorithm section: the
field-driven part J_H has zero net current in every subelement, the transport
part J_I is shared by the coupled subelements of the whole wire through the
A-V formulation).

The constrained solve with one group per turn is checked against the
single-constraint solve, the bordered system against numpy's dense solver, the
transport shares of two loops in parallel against the parallel-inductor
division (L2 - M) : (L1 - M), and a field ramp on turns without transport
current against the zero-net invariant of every subelement."""
import numpy as np

import oracle
from oracle.step import kkt_solve, subelement_kkt_solve, transport_shares
from paper_2403_07666_b300.workloads import MATERIAL, random_coil


def _spd(rng, n):
    X = rng.standard_normal((n, n))
    return X @ X.T + n * np.eye(n)


def test_one_group_per_turn_is_the_turn_constraint():
    rng = np.random.default_rng(1)
    B, W = 5, 4
    A = _spd(rng, B * W)
    R = rng.standard_normal(B * W)
    c = rng.standard_normal(W)
    con = np.array([True, False, True, True])
    groups = np.zeros(B, dtype=np.int64)
    _, d = transport_shares(A, R, c, B, con, groups)
    assert np.allclose(d[con, 0], c[con], rtol=1e-13, atol=0)
    x1, u1 = kkt_solve(A, R, c, B, con)
    x2, u2, v = subelement_kkt_solve(A, R, d, B, con, groups)
    assert np.max(np.abs(x1 - x2)) <= 1e-12 * np.max(np.abs(x1))
    assert np.max(np.abs(u1 - u2)) <= 1e-12 * np.max(np.abs(u1))


def test_bordered_system_matches_dense_solve():
    """[[A, -Q], [Q^T, 0]] [x; v] = [-R; d] assembled and solved directly."""
    rng = np.random.default_rng(2)
    B, W = 6, 3
    groups = np.array([0, 0, 1, 1, 2, 2])
    S = 3
    con = np.array([True, True, False])
    A = _spd(rng, B * W)
    R = rng.standard_normal(B * W)
    d = rng.standard_normal((W, S))
    x, u, v = subelement_kkt_solve(A, R, d, B, con, groups)
    N = B * W
    cols = [(w, g) for w in range(W) if con[w] for g in range(S)]
    Q = np.zeros((N, len(cols)))
    for k, (w, g) in enumerate(cols):
        Q[w * B + np.nonzero(groups == g)[0], k] = 1.0
    K = np.block([[A, -Q], [Q.T, np.zeros((len(cols), len(cols)))]])
    rhs = np.concatenate([-R, [d[w, g] for (w, g) in cols]])
    sol = np.linalg.solve(K, rhs)
    assert np.max(np.abs(x - sol[:N])) <= 1e-11 * np.max(np.abs(sol[:N]))
    vv = np.array([v[w, g] for (w, g) in cols])
    assert np.max(np.abs(vv - sol[N:])) <= 1e-11 * np.max(np.abs(sol[N:]))
    # the free turn is unconstrained and reports no voltage
    assert np.all(v[2] == 0.0) and u[2] == 0.0
    assert abs(u[0] - np.mean(v[0])) <= 1e-15 * abs(u[0]) + 1e-300


def _two_turns(groups, neighbour_ramp=True):
    """Two turns of two coaxial loops each (radially adjacent), superconducting
    (E negligible): the first ramps, the second ramps too or is held at 0."""
    p = dict(MATERIAL, thermal=0, jc_model=1, Jc0=1e16)
    geom = {"kind": "list", "r": np.array([0.0200, 0.0204, 0.0200, 0.0204]),
            "z": np.array([0.0, 0.0, 0.0009, 0.0009]), "h": np.full(4, 4e-4), "block": 2,
            "groups": groups}
    c = oracle.build(geom, p, np.ones(4), np.zeros(4), np.ones(4, dtype=np.int64),
                     np.array([True, True]))
    drive = {"dt": 1e-5, "ramp_rate": 3e5, "I_max": 1e9, "Ba_rate": 0.0, "Ba_max": 0.0, "Ba_waveform": 0}
    return c, drive


def test_parallel_loops_share_by_their_own_inductances():
    """Decoupled subelements: each loop of a turn is its own subelement, so the
    turn's transport current divides as in two inductors in parallel,
    I1 : I2 = (L2 - M) : (L1 - M), whatever the neighbouring turn does.  With
    one coupled group the neighbour's flux shifts the division."""
    c, drive = _two_turns(np.array([0, 1]))
    for _ in range(20):
        c.step(drive)
    L1, L2, M = c.M[0, 0], c.M[1, 1], c.M[0, 1]
    ratio = c.I[0] / c.I[1]
    assert abs(ratio / ((L2 - M) / (L1 - M)) - 1.0) < 1e-9
    assert abs(c.I[0] + c.I[1] - 20 * 1e-5 * 3e5) < 1e-9
    cc, _ = _two_turns(None)
    for _ in range(20):
        cc.step(drive)
    assert abs(cc.I[0] / cc.I[1] / ratio - 1.0) > 1e-3


def test_field_ramp_keeps_every_subelement_net_zero():
    """Turns with no transport current in a ramping applied field: the induced
    currents circulate inside every subelement (zero net each); one coupled
    group per turn lets the net of a quadrant drift."""
    mtl = dict(MATERIAL, Jc0=2e8)
    quad = np.array([(b // 2) * 2 + (a // 2) for b in range(4) for a in range(4)])
    w = random_coil(61, 2, 3, 4, ramp_rate=0.0, I_max=0.0, material=mtl, dt=1e-4,
                    Ba_rate=40.0, Ba_max=0.05, Ba_waveform=1)
    w.geometry["groups"] = quad
    c = oracle.build(w.geometry, w.material, w.jc_factor, w.strain, w.mat)
    w0 = random_coil(61, 2, 3, 4, ramp_rate=0.0, I_max=0.0, material=mtl, dt=1e-4,
                     Ba_rate=40.0, Ba_max=0.05, Ba_waveform=1)
    c0 = oracle.build(w0.geometry, w0.material, w0.jc_factor, w0.strain, w0.mat)
    scale = net = net0 = 0.0
    for _ in range(30):                # 12.5 steps of ramp, then the currents decay
        c.step(w.drive)
        c0.step(w0.drive)
        I = c.I.reshape(-1, 16)
        I0 = c0.I.reshape(-1, 16)
        scale = max(scale, np.max(np.abs(I)))
        net = max(net, max(np.max(np.abs(I[:, quad == g].sum(axis=1))) for g in range(4)))
        net0 = max(net0, np.max(np.abs(I0[:, quad == 0].sum(axis=1))) / np.max(np.abs(I0)))
    assert scale > 0
    assert net <= 1e-11 * scale
    assert np.all(c.I_tr == 0.0) or np.max(np.abs(c.I_tr)) <= 1e-11 * scale
    assert net0 > 1e-3


def test_transport_fills_the_outer_subelements_first():
    """A superconducting turn under a current ramp: the ring of outer elements
    takes more than its element share of the transport current, the inner
    2 x 2 subelement less (the self-field screens the inside)."""
    ring = np.array([0 if (a in (1, 2) and b in (1, 2)) else 1 for b in range(4) for a in range(4)])
    w = random_coil(62, 1, 3, 4, ramp_rate=2e4, material=dict(MATERIAL, Jc0=1e12, thermal=0))
    w.geometry["groups"] = ring
    c = oracle.build(w.geometry, w.material, w.jc_factor, w.strain, w.mat)
    for _ in range(10):
        c.step(w.drive)
    I = c.I.reshape(-1, 16)
    inner = I[:, ring == 0].sum(axis=1) / I.sum(axis=1)
    assert np.all(inner < 4 / 16)
    assert np.all(np.abs(I.sum(axis=1) - 10 * 1e-5 * 2e4) < 1e-9)


def test_transport_relaxes_to_the_resistive_division():
    """Ohmic (Cu) loops of one turn in two subelements, a current ramp then a
    long hold: the transport part settles where the loop voltages 2 pi r rho J
    are equal (loops in parallel: I_k proportional to 1 / R_k = a / (2 pi r_k
    rho_n)), and the field-driven part decays, so I_k -> I_t (1/r_k) / sum 1/r_j.
    Without the resistive voltage of the transport part it would keep the
    inductive division of the ramp."""
    p = dict(MATERIAL, thermal=0, jc_model=1)
    r = np.array([0.0200, 0.0204, 0.0200, 0.0204])
    geom = {"kind": "list", "r": r, "z": np.array([0.0, 0.0, 4e-4, 4e-4]), "h": np.full(4, 4e-4),
            "block": 4, "groups": np.array([0, 0, 1, 1])}
    c = oracle.build(geom, p, np.ones(4), np.zeros(4), np.zeros(4, dtype=np.int64), np.array([True]))
    drive = {"dt": 1e-5, "ramp_rate": 2e5, "I_max": 10.0, "Ba_rate": 0.0, "Ba_max": 0.0, "Ba_waveform": 0}
    for _ in range(50):
        c.step(drive)
    early = c.I / 10.0
    for _ in range(1200):
        c.step(drive)
    share = (1.0 / r) / np.sum(1.0 / r)
    assert np.max(np.abs(c.I / 10.0 - share)) < 1e-6
    assert np.max(np.abs(early - share)) > 1e-3
    assert np.max(np.abs(c.I_tr - c.I)) < 1e-6 * 10.0
