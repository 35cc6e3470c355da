"""Forward-mode derivatives of the oracle's step series (tangent-linear
oracle).  TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``.

The calibration of the paper fits its E-J and Jc laws to a measured
magnetization loop (Methods); the library differentiates its discrete steps
in reverse (adjoint).  This module gives the same derivatives in forward
mode, directly from the oracle's definition of the step: for a direction
v = (v_f per element, v_n, v_C) in the parameters (Jc factor f, creep
exponent n, strain coefficient C_eps) it returns, for every step k,

    dm_k = d m_k / d theta . v     (moment sum pi r^2 I after step k)
    dP_k = d P_k / d theta . v     (Joule power sum q 2 pi r a of the start
                                    state of step k, the diagnostic record)

by the complex-step method (Squire and Trapp, SIAM Review 40 (1998) 110;
Martins, Sturdza and Alonso, ACM TOMS 29 (2003) 245): every parameter
receives an imaginary perturbation i h v, the step is evaluated in complex
arithmetic with complex-analytic operations, and Im(.)/h is the directional
derivative to rounding (no difference of nearby values is taken, so h can be
1e-30).  The step is the oracle's (``step.OracleCoil.step``): the same field
stencil, Jc(B, T, eps), parallel power-law / normal E-J law, exact KKT solve
and Peaceman-Rachford ADI, restated with

  * |x| as x sign(Re x) (analytic away from 0), maxima and branch tests on the
    real part;
  * the KKT system, whose matrix M + dt diag(G) is complex symmetric (not
    Hermitian), solved by LU instead of Cholesky;
  * the linear parts (loop flux M I, field stencil, the ADI's tridiagonal
    solves and axis operators) applied to the real and imaginary parts, which
    is exact for a real linear map.

Pins (tests/test_oracle_tangent.py): against central finite differences of
the oracle's own step series for every parameter, and dP_k = 0, dm_k = 0 for
a purely ohmic (all Cu) coil, whose step does not depend on f, n or C_eps.
The subelement decoupling is not covered (the library's adjoint refuses it).
"""

import numpy as np
import scipy.linalg as sla

from .constitutive import FILAMENT
from .field import field_from_flux
from .step import build, drive_values


def _cabs(x):
    return x * np.sign(x.real)


def _linear(f, x):
    """A real linear map applied to a complex argument."""
    return f(x.real) + 1j * f(x.imag)


def _critical_current(Bm, T, eps, f, mat, p, C_eps):
    if p["jc_model"] == 1:
        Jc = f * p["Jc0"] + 0.0 * Bm
    else:
        tr = T / p["Tc"]
        Bc2 = p["Bc2_0"] * (1.0 - tr * tr)
        ok = (T.real < p["Tc"]) & (Bm.real < Bc2.real)
        with np.errstate(invalid="ignore", divide="ignore"):
            sfac = 1.0 - C_eps * _cabs(eps) ** p["p_eps"]
            sfac = np.where(sfac.real > 0.0, sfac, 0.0)
            Jc = (f * p["Jc0"] * (1.0 - tr) ** 1.5 * (1.0 - Bm / Bc2) ** 2 / np.sqrt(Bm + p["B_reg"]) * sfac)
        Jc = np.where(ok, Jc, 0.0)
    return np.where(np.asarray(mat) == FILAMENT, Jc, 0.0)


def _ej_terms(I, Jc, mat, r, area, p, n):
    J = I / area
    aJ = _cabs(J)
    fil = np.asarray(mat) == FILAMENT
    rho_n = p["rho_n"]
    sc = fil & (Jc.real > 0.0) & (aJ.real > 0.0)
    Jcs = np.where(sc, Jc, 1.0)
    aJs = np.where(sc, aJ, 1.0)
    ell = np.log(p["E0"] / (Jcs * rho_n)) + (n - 1.0) * np.log(aJs / Jcs)
    pos = ell.real > 0.0
    t = np.exp(-np.where(pos, ell, 0.0))
    s = np.exp(np.where(pos, 0.0, ell))
    frac = np.where(pos, 1.0 / (1.0 + t), s / (1.0 + s))
    dfac = np.where(pos, (1.0 + n * t) / (1.0 + t) ** 2, s * (s + n) / (1.0 + s) ** 2)
    # Jc = 0: normal; J = 0 (superconducting): rho = 0
    norm = fil & (Jc.real <= 0.0)
    zero = fil & (Jc.real > 0.0) & (aJ.real == 0.0)
    frac = np.where(norm, 1.0, np.where(zero, 0.0, frac))
    dfac = np.where(norm, 1.0, np.where(zero, 0.0, dfac))
    frac = np.where(fil, frac, 1.0)
    dfac = np.where(fil, dfac, 1.0)
    rho = rho_n * frac
    E = rho * J
    G = 2.0 * np.pi * r * rho_n * dfac / area
    return E, G, E * J


def _kkt(A, R, c, block, constrained):
    """A x - P u = -R, P^T x = c for a complex symmetric A (LU, Schur)."""
    N = A.shape[0]
    lu = sla.lu_factor(A)
    xR = sla.lu_solve(lu, R)
    wires = np.nonzero(constrained)[0]
    if wires.size == 0:
        return -xR
    P = np.zeros((N, wires.size))
    for k, w in enumerate(wires):
        P[w * block:(w + 1) * block, k] = 1.0
    Y = sla.lu_solve(lu, P.astype(A.dtype))
    S = P.T @ Y
    uc = np.linalg.solve(S, c[wires] + P.T @ xR)
    return Y @ uc - xR


def _to_grid(th, v):
    out = np.zeros((th.geo["Gz"], th.geo["Gr"]), dtype=complex)
    out[th.geo["i_z"], th.geo["i_r"]] = v
    return out


def _adi(th, u, q, dt, p):
    """ThermalGrid.adi_step with a complex u and q (source pointwise in
    complex arithmetic; the axis operators and line solves are real linear)."""
    T = np.sqrt(np.sqrt(u))
    loss = th.n_border * th.h * p["h0"] * (T / p["T_ref"]) ** 3 * (T - p["T_bath"])
    s = 4.0 / (p["rho_m"] * p["c0"]) * (q - loss / (th.h * th.h))
    hd = 0.5 * dt
    lin_z = lambda x: th.apply_axis(x, th.Kz, axis=0)      # noqa: E731
    lin_r = lambda x: th.apply_axis(x, th.Kr, axis=1)      # noqa: E731
    lo, di, up = th.tridiag(th.Kr, hd)
    from .thermal import thomas
    ustar = _linear(lambda x: thomas(lo, di, up, x), u + hd * _linear(lin_z, u) + hd * s)
    rhs2 = ustar + hd * _linear(lin_r, ustar) + hd * s
    lo, di, up = th.tridiag(th.Kz, hd)
    return _linear(lambda x: thomas(lo, di, up, x.T).T, rhs2)


def directional_derivatives(w, n_steps, v_f=None, v_n=0.0, v_C=0.0, h=1e-30):
    """(m, P, dm, dP) over n_steps oracle steps of workload w from its initial
    state: moments after each step, Joule powers of each step's start state,
    and their derivatives along (v_f, v_n, v_C)."""
    orc = build(w.geometry, w.material, w.jc_factor, w.strain, w.mat)
    if orc.groups is not None:
        raise ValueError("subelement decoupling is not differentiated")
    geo, p = orc.geo, dict(orc.p)
    N, B, W = geo["N"], geo["block"], geo["W"]
    r, area = geo["r"], geo["area"]
    f = orc.jc_factor + 1j * h * (np.zeros(N) if v_f is None else np.asarray(v_f, dtype=np.float64))
    n = p["n"] + 1j * h * v_n
    C_eps = p["C_eps"] + 1j * h * v_C
    Y = p.get("Y_eff", 0.0)
    th = orc.thermal
    I = np.zeros(N, dtype=complex)
    u = np.full(N, p["T_bath"] ** 4, dtype=complex)
    t = 0.0
    drive = w.drive
    dt = drive["dt"]
    m, P, dm, dP = [], [], [], []
    for _ in range(n_steps):
        _, Ba0 = drive_values(t, drive)
        It1, Ba1 = drive_values(t + dt, drive)
        dBa = (Ba1 - Ba0) / dt
        if geo["grid"]:
            phi = _linear(lambda x: orc.M @ x, I) + np.pi * r ** 2 * Ba0
            Br = _linear(lambda x: field_from_flux(geo, x)[0], phi)
            Bz = _linear(lambda x: field_from_flux(geo, x)[1], phi)
        else:
            Br = Bz = np.zeros(N, dtype=complex)
        Bm = np.sqrt(Br * Br + Bz * Bz)
        T = np.sqrt(np.sqrt(u))
        eps = orc.strain + (r * (I / area) * Bz / Y if Y else 0.0)
        Jc = _critical_current(Bm, T, eps, f, orc.mat, p, C_eps)
        E, G, q = _ej_terms(I, Jc, orc.mat, r, area, p, n)
        Pk = np.sum(q * 2.0 * np.pi * r * area)
        R = 2.0 * np.pi * r * E + np.pi * r * r * dBa
        c = (It1 - I.reshape(W, B).sum(axis=1)) / dt
        A = orc.M + np.diag(dt * G)
        x = _kkt(A, R, c, B, orc.constrained)
        I = I + dt * x
        if th is not None:
            u = th.to_elem(_adi(th, _to_grid(th, u), _to_grid(th, q), dt, p))
        t = t + dt
        mk = np.sum(np.pi * r * r * I)
        m.append(mk.real)
        dm.append(mk.imag / h)
        P.append(Pk.real)
        dP.append(Pk.imag / h)
    return np.array(m), np.array(P), np.array(dm), np.array(dP)
