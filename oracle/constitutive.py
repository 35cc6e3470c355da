"""E-J law with Jc(B, T, eps) and Joule heating (oracle).

Methods, E-J paragraph: E = rho(J) J with a law spanning flux creep, flux
flow and the normal state, and a Kramer-type Jc(B, T, eps) fit.  The paper
defers the explicit laws to its supplement; the forms used here are the
explicit ones of the synthetic Nb3Sn workload:

    Jc = f Jc0 (1 - T/Tc)^1.5 (1 - |B|/Bc2(T))^2 / sqrt(|B| + B_reg)
           * max(0, 1 - C_eps |eps|^p_eps),     Bc2(T) = Bc2(0) (1 - (T/Tc)^2),

Jc = 0 where T >= Tc or |B| >= Bc2(T).  ``jc_model = 1`` uses Jc = f Jc0.

Filament (superconducting) elements: the power law E0 (J/Jc)^n acts in
parallel with the normal resistivity rho_n, so rho -> rho_n as Jc -> 0 (the
0.95 rho_n quench criterion of the quench section needs that limit):

    l   = ln(E0 / (Jc rho_n)) + (n - 1) ln(|J| / Jc),   s = e^l,
    rho = rho_n s / (1 + s),  E = rho J,  q = E J,
    dE/dJ = rho_n s (s + n) / (1 + s)^2.

Cu (matrix) elements are ohmic: rho = rho_n.  The loop term of the circuit
equation is 2 pi r E; its derivative with respect to the loop current is
G = 2 pi r (dE/dJ) / a (a = element area).

Pins (tests/test_oracle_constitutive.py): hand values of Jc, the limits
Jc -> 0 and J -> 0, the pure power law where s << 1, and G against a central
finite difference of 2 pi r E(I).
"""

import numpy as np

FILAMENT = 1
COPPER = 0


def critical_current(Bmag, T, eps, f, mat, p):
    """Critical current density per element [A/m^2] (0 for Cu elements)."""
    Bmag = np.asarray(Bmag, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    if p["jc_model"] == 1:
        Jc = f * p["Jc0"] + 0.0 * Bmag
    else:
        tr = T / p["Tc"]
        Bc2 = p["Bc2_0"] * (1.0 - tr * tr)
        ok = (T < p["Tc"]) & (Bmag < Bc2)
        with np.errstate(invalid="ignore", divide="ignore"):
            strain = np.maximum(0.0, 1.0 - p["C_eps"] * np.abs(eps) ** p["p_eps"])
            Jc = (f * p["Jc0"] * (1.0 - tr) ** 1.5 * (1.0 - Bmag / Bc2) ** 2
                  / np.sqrt(Bmag + p["B_reg"]) * strain)
        Jc = np.where(ok, Jc, 0.0)
    return np.where(np.asarray(mat) == FILAMENT, Jc, 0.0)


def ej_terms(I, Jc, mat, r, area, p):
    """Per-element (J, rho, E, dE/dJ, G, q, |J|/Jc) for loop currents I."""
    I = np.asarray(I, dtype=np.float64)
    J = I / area
    absJ = np.abs(J)
    fil = np.asarray(mat) == FILAMENT
    rho_n = p["rho_n"]
    nexp = p["n"]
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        ell = np.log(p["E0"] / (Jc * rho_n)) + (nexp - 1.0) * np.log(absJ / Jc)
        ell = np.where(Jc <= 0.0, np.inf, ell)
        ell = np.where((Jc > 0.0) & (absJ == 0.0), -np.inf, ell)
        # s/(1+s) and s(s+n)/(1+s)^2 without overflow
        pos = ell > 0.0
        t = np.exp(-np.where(pos, ell, 0.0))          # e^{-l} for l > 0
        s = np.exp(np.where(pos, 0.0, ell))           # e^{l}  for l <= 0
        frac = np.where(pos, 1.0 / (1.0 + t), s / (1.0 + s))
        dfac = np.where(pos, (1.0 + nexp * t) / (1.0 + t) ** 2, s * (s + nexp) / (1.0 + s) ** 2)
        jratio = np.where(Jc > 0.0, absJ / Jc, np.where(absJ > 0.0, np.inf, 0.0))
    frac = np.where(fil, frac, 1.0)
    dfac = np.where(fil, dfac, 1.0)
    jratio = np.where(fil, jratio, 0.0)
    rho = rho_n * frac
    E = rho * J
    dEdJ = rho_n * dfac
    G = 2.0 * np.pi * r * dEdJ / area
    q = E * J
    return {"J": J, "rho": rho, "E": E, "dEdJ": dEdJ, "G": G, "q": q, "jratio": jratio}
