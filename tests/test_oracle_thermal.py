"""Pins of the oracle's heat-diffusion step (T^3 laws, bath sink, ADI)."""
import math

import numpy as np
import pytest

import oracle
from oracle.thermal import ThermalGrid
from paper_2403_07666_b300.workloads import MATERIAL

P = dict(MATERIAL)


def test_isolated_element_relaxation():
    """One element, all four faces on the bath, q = 0: the T^3 laws cancel and
    T - T_bath decays as exp(-lambda t), lambda = 4 h0 / (rho_m c0 h T_ref^3)."""
    h = 0.8e-3
    geo = oracle.solenoid_elements(1, 1, 1, 0.02, 0.9e-3, h)
    lam = 4 * P["h0"] / (P["rho_m"] * P["c0"] * h * P["T_ref"] ** 3)
    assert abs(lam - 37.9) < 0.1
    T0, Tb, tend = 6.0, P["T_bath"], 0.02
    errs = []
    for dt in (2e-5, 1e-5):
        th = ThermalGrid(geo, P)
        u = np.full((1, 1), T0 ** 4)
        for _ in range(int(round(tend / dt))):
            u = th.adi_step(u, np.zeros((1, 1)), dt)
        T = u[0, 0] ** 0.25
        exact = Tb + (T0 - Tb) * math.exp(-lam * tend)
        errs.append(abs(T - exact) / (T0 - Tb))
    assert errs[1] < 2 * lam * 1e-5                 # O(lambda dt)
    assert 1.8 < errs[0] / errs[1] < 2.2             # first order: halves with dt


def test_energy_conservation_without_bath():
    geo = oracle.solenoid_elements(3, 4, 4, 0.02, 0.9e-3, 0.8e-3)
    p = dict(P, h0=0.0)
    th = ThermalGrid(geo, p)
    rng = np.random.default_rng(0)
    u = (4.2 + rng.uniform(0, 3, (geo["Gz"], geo["Gr"]))) ** 4
    q = rng.uniform(0, 1e6, u.shape)
    dt = 1e-5
    un = th.adi_step(u, q, dt)
    gain = dt * np.sum(4.0 / (p["rho_m"] * p["c0"]) * q)
    assert abs((un.sum() - u.sum()) - gain) < 1e-12 * u.sum()
    # a uniform state without source is a fixed point
    uu = np.full_like(u, 5.0 ** 4)
    assert np.max(np.abs(th.adi_step(uu, 0 * q, dt) - uu)) < 1e-12 * uu.max()


def test_peaceman_rachford_cosine_mode_amplification():
    """Uniform grid (no epoxy gaps): a separable cosine mode is an eigenvector;
    one PR step multiplies it by (1+a_z)(1+a_r)/((1-a_r)(1-a_z)), a = dt/2 lambda."""
    geo = oracle.solenoid_elements(3, 5, 4, 0.02, 0.8e-3, 0.8e-3)     # pitch = side: no gap
    p = dict(P, h0=0.0)
    th = ThermalGrid(geo, p)
    Gr, Gz = geo["Gr"], geo["Gz"]
    K, C = th.K_in, th.C
    dt = 2e-6
    for kr, kz in ((1, 2), (3, 1), (5, 7)):
        mode = np.outer(np.cos(math.pi * kz * (np.arange(Gz) + 0.5) / Gz),
                        np.cos(math.pi * kr * (np.arange(Gr) + 0.5) / Gr))
        lr = -4 * K / C * math.sin(math.pi * kr / (2 * Gr)) ** 2
        lz = -4 * K / C * math.sin(math.pi * kz / (2 * Gz)) ** 2
        ar, az = 0.5 * dt * lr, 0.5 * dt * lz
        g = (1 + az) * (1 + ar) / ((1 - ar) * (1 - az))
        base = 5.0 ** 4                        # uniform state: a fixed point
        out = th.adi_step(base + 100.0 * mode, np.zeros_like(mode), dt)
        assert np.max(np.abs((out - base) / 100.0 - g * mode)) < 1e-11


def test_adi_step_against_dense_half_step_solves():
    geo = oracle.solenoid_elements(2, 3, 3, 0.02, 0.9e-3, 0.8e-3)
    th = ThermalGrid(geo, P)
    Gr, Gz = geo["Gr"], geo["Gz"]
    n = Gr * Gz
    Ar = np.zeros((n, n))
    Az = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        Ar[:, k] = th.apply_axis(e.reshape(Gz, Gr), th.Kr, axis=1).ravel()
        Az[:, k] = th.apply_axis(e.reshape(Gz, Gr), th.Kz, axis=0).ravel()
    rng = np.random.default_rng(2)
    u = ((4.2 + rng.uniform(0, 2, n)) ** 4)
    q = rng.uniform(0, 1e7, n)
    dt = 1e-5
    s = th.source(u.reshape(Gz, Gr), q.reshape(Gz, Gr)).ravel()
    I = np.eye(n)
    ustar = np.linalg.solve(I - dt / 2 * Ar, u + dt / 2 * Az @ u + dt / 2 * s)
    unew = np.linalg.solve(I - dt / 2 * Az, ustar + dt / 2 * Ar @ ustar + dt / 2 * s)
    out = th.adi_step(u.reshape(Gz, Gr), q.reshape(Gz, Gr), dt).ravel()
    assert np.max(np.abs(out - unew)) < 1e-13 * np.max(np.abs(unew))


def _fine_grid_conductance(segments, face_height, slices=4000):
    """Brute-force 1-D steady conduction between two cell centres.

    ``segments`` lists (length, conductivity) of the materials in series; each
    is cut into equal slices, node temperatures solved with u = 1 at one end
    and u = 0 at the other by a dense linear solve of the nodal balance (not
    a series-resistance formula).  Returns the heat flow per unit depth
    through a face of height ``face_height`` per unit of u difference."""
    k_links, dx_links = [], []
    for length, kappa in segments:
        n = max(1, int(round(slices * length / sum(s[0] for s in segments))))
        k_links += [kappa] * n
        dx_links += [length / n] * n
    cond = np.array(k_links) / np.array(dx_links)          # per link
    m = cond.size + 1                                        # nodes
    A = np.zeros((m, m))
    b = np.zeros(m)
    for i, g in enumerate(cond):
        A[i, i] += g
        A[i + 1, i + 1] += g
        A[i, i + 1] -= g
        A[i + 1, i] -= g
    A[0, :] = 0.0
    A[0, 0] = 1.0
    b[0] = 1.0
    A[-1, :] = 0.0
    A[-1, -1] = 1.0
    u = np.linalg.solve(A, b)
    return cond[0] * (u[0] - u[1]) * face_height


@pytest.mark.parametrize("layers,turns,axis", [(2, 1, 1), (1, 2, 0)])
def test_epoxy_gap_conductance_against_fine_grid_conduction(layers, turns, axis):
    """Two one-element wires side by side (radially, then axially), no bath,
    no source.  In u = T^4 the heat flux is -(kappa_ref / (4 T_ref^3)) du/dx
    in both Cu and epoxy (both follow the T^3 law), so the conductance between
    the two cell centres is that of half a Cu cell, the epoxy gap and half a
    Cu cell in series.  One Peaceman-Rachford step multiplies the difference
    mode u1 - u2 by (1 - dt K / C) / (1 + dt K / C); K read off the oracle's
    step must equal the brute-force fine-grid conduction across Cu | epoxy |
    Cu (Methods, heat-diffusion paragraph: the composite section)."""
    d, pitch = 0.8e-3, 0.9e-3
    geo = oracle.solenoid_elements(layers, turns, 1, 0.02, pitch, d)
    p = dict(P, h0=0.0)
    th = ThermalGrid(geo, p)
    T3 = 4.0 * p["T_ref"] ** 3
    gap = pitch - d
    K_fine = _fine_grid_conductance(
        [(d / 2, p["kappa_cu"] / T3), (gap, p["kappa_ep"] / T3), (d / 2, p["kappa_cu"] / T3)], d)
    C = p["rho_m"] * p["c0"] * d * d / 4.0                 # cell capacity per unit depth
    dt = 1e-5
    base, amp = 5.0 ** 4, 40.0
    u = np.full((geo["Gz"], geo["Gr"]), base)
    if axis == 1:
        u[0, 0] += amp
        u[0, 1] -= amp
    else:
        u[0, 0] += amp
        u[1, 0] -= amp
    out = th.adi_step(u, np.zeros_like(u), dt)
    diff = (out.ravel()[0] - out.ravel()[1]) / (2 * amp)
    K_step = C * (1.0 - diff) / (dt * (1.0 + diff))
    assert abs(K_step - K_fine) < 1e-9 * K_fine
    # the epoxy dominates: swapping the two conductivities or dropping the gap
    # would move K by orders of magnitude
    K_swapped = _fine_grid_conductance(
        [(d / 2, p["kappa_ep"] / T3), (gap, p["kappa_cu"] / T3), (d / 2, p["kappa_ep"] / T3)], d)
    assert abs(K_step - K_swapped) > 0.5 * K_fine
    assert abs(K_step - p["kappa_cu"] / T3) > 0.5 * K_fine
