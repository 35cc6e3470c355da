"""Parity at the benchmark's full size: the 96,000-element real-size coil in
the configurations bench.py times (tensor-core Toeplitz and dense operators,
PCG rtol 1e-9).  The oracle cannot solve this coil directly, so it checks
outputs it can compute one at a time: operator columns, the field at sampled
elements, the stationarity of the step's constrained solve on sampled wires,
the whole heat step and the step's diagnostics."""
import numpy as np
import pytest

import oracle
from oracle.field import lagrange3_weights
from oracle.inductance import operator_rows
from oracle.thermal import ThermalGrid
from paper_2403_07666_b300 import build as B
from paper_2403_07666_b300 import workloads as wl
from tests.gpu_common import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _stencil_B(geo, I, e):
    """(B_r, B_z) at element e from oracle rows of the flux (B_a = 0)."""
    Gr, Gz = geo["Gr"], geo["Gz"]
    grid = np.full((Gz, Gr), -1)
    grid[geo["i_z"], geo["i_r"]] = np.arange(geo["N"])
    iz, ir = geo["i_z"][e], geo["i_r"][e]
    jr = min(max(ir - 1, 0), Gr - 3)
    jz = min(max(iz - 1, 0), Gz - 3)
    er = grid[iz, jr:jr + 3]
    ez = grid[jz:jz + 3, ir]
    rows = operator_rows(geo["r"], geo["z"], geo["h"], np.concatenate([er, ez]))
    phi = rows @ I
    ax_r, ax_z = geo["r_axis"], geo["z_axis"]
    wr = lagrange3_weights(ax_r[jr], ax_r[jr + 1], ax_r[jr + 2], ax_r[ir])
    wz = lagrange3_weights(ax_z[jz], ax_z[jz + 1], ax_z[jz + 2], ax_z[iz])
    dr = sum(wk * p for wk, p in zip(wr, phi[:3]))
    dz = sum(wk * p for wk, p in zip(wz, phi[3:]))
    r = geo["r"][e]
    return -dz / (2 * np.pi * r), dr / (2 * np.pi * r)


# FP32 storage rounds every operator entry by up to 2^-24; the flux carries that
# rounding and the 3-point stencil differentiates it across one element, which
# amplifies it about 10^3-fold in B (measured 1.7e-4 after 5 steps).
# The tensor-core Toeplitz form stores each entry as an FP16 hi + lo pair
# (about 2^-22 relative) and is the operator format bench.py times.
@pytest.mark.parametrize("precision,fmt,tol_op,tol,tol_B", [("fp32", "dense", 2e-7, 2e-5, 5e-4),
                                                             ("fp32", "toeplitz_tc", 3e-7, 2e-5, 5e-4),
                                                             ("fp64", "dense", 1e-11, 1e-6, 1e-6)])
def test_real_coil_sampled_parity(precision, fmt, tol_op, tol, tol_B):
    from paper_2403_07666_b300.coil import Coil
    w = wl.real_coil()
    g = w.geometry
    geo = oracle.solenoid_elements(g["n_layers"], g["n_turns"], g["n_sub"], g["r_in"], g["pitch"],
                                   g["wire_d"])
    N, Bk = geo["N"], geo["block"]
    assert N == 96000
    drive = dict(w.drive, ramp_rate=1e4)                 # non-trivial currents within a few steps
    p = w.material
    with Coil.from_workload(w, precision=precision, format=fmt, rtol=1e-9) as c:
        # operator columns (M symmetric: column j = row j)
        for j in (0, 12345, 48017, N - 1):
            e = np.zeros(N)
            e[j] = 1.0
            col = c.apply_operator(e)
            assert rel(col, operator_rows(geo["r"], geo["z"], geo["h"], [j])[0]) < tol_op
        c.step(5, drive)
        Ik = c.currents()
        sk = c.read(drive)
        c.step(1, drive)
        Ik1 = c.currents()
        sk1 = c.read(drive)
        rec = c.diag(5, 1)[0]
    dt = drive["dt"]
    t1 = 6 * dt
    It1 = drive["ramp_rate"] * t1
    # transport constraint on every turn
    assert np.max(np.abs(Ik1.reshape(-1, Bk).sum(axis=1) - It1)) < 1e-9 * It1
    # field at sampled elements from oracle flux rows and the GPU's currents
    rng = np.random.default_rng(17)
    samples = np.concatenate([[0, N - 1, 47 * Bk + 5], rng.integers(0, N, 5)])
    Bref = np.array([_stencil_B(geo, Ik, e) for e in samples])
    Bgpu = np.stack([sk["Br"][samples], sk["Bz"][samples]], axis=1)
    assert np.max(np.abs(Bgpu - Bref)) < tol_B * np.max(np.abs(Bref))
    # pointwise state k from the GPU's B and T (oracle law)
    Bm = np.hypot(sk["Br"], sk["Bz"])
    Jc = oracle.critical_current(Bm, sk["T"], w.strain, w.jc_factor, w.mat, p)
    tm = oracle.ej_terms(Ik, Jc, w.mat, geo["r"], geo["area"], p)
    # stationarity of the constrained solve on sampled wires: (M Idot + dt G Idot + R) is the
    # wire's loop voltage, the same on every element of the wire
    Idot = (Ik1 - Ik) / dt
    for wi in (0, 2999, 5999, int(rng.integers(0, N // Bk))):
        el = np.arange(wi * Bk, (wi + 1) * Bk)
        MI = operator_rows(geo["r"], geo["z"], geo["h"], el) @ Idot
        R = 2 * np.pi * geo["r"][el] * tm["E"][el]
        gvec = MI + dt * tm["G"][el] * Idot[el] + R
        scale = max(np.max(np.abs(MI)), np.max(np.abs(R)))
        assert np.ptp(gvec) < tol * scale, (wi, np.ptp(gvec) / scale)
    # whole heat step on the full grid from the GPU's state k
    th = ThermalGrid(geo, p)
    u1 = th.adi_step(th.to_grid(sk["T"] ** 4), th.to_grid(tm["q"]), dt)
    T1 = th.to_elem(u1) ** 0.25
    dT = max(np.max(np.abs(T1 - p["T_bath"])), 1e-6 * p["T_bath"])
    assert np.max(np.abs(sk1["T"] - T1)) < tol * dT
    # diagnostics of the step
    Pj = np.sum(tm["q"] * 2 * np.pi * geo["r"] * geo["area"])
    assert abs(rec[4] - Pj) <= tol * abs(Pj)
    assert abs(rec[3] - np.sum(np.pi * geo["r"] ** 2 * Ik1)) <= 1e-12 * abs(rec[3])
    assert abs(rec[1] - It1) <= 1e-12 * It1
