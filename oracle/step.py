"""One coupled electromagnetic-thermal time step, solved exactly (oracle).

Per-element circuit equation of loop e (Numerical Algorithm section: the field
on each wire from all currents plus the background field, the transport part
of J over each whole wire by the A-V formulation):

    sum_j M_ej dI_j/dt + pi r_e^2 dB_a/dt + 2 pi r_e E_e(I_e) = u_w(e),

u_w = loop voltage of turn w (the scalar-potential unknown of the A-V
formulation; free loops have u = 0), with the transport constraint
sum_{e in w} I_e = I_t(t) on every turn.  The time step is linearly-implicit
Euler: E is linearised about the start-of-step state with its exact diagonal
derivative G = d(2 pi r E)/dI (B and T frozen), giving per step

    (M + dt G) Idot - P u = -R,      P^T Idot = c,
    R_e = 2 pi r_e E_e + pi r_e^2 (B_a(t+dt) - B_a(t)) / dt,
    c_w = (I_t(t + dt) - sum_{e in w} I_e) / dt,

then I <- I + dt Idot and the heat equation advances with the Joule source
q = E J of the start-of-step state.  The paper's own inner iteration
(m = 1, 2 with 2.5 % / 0.1 % stopping thresholds) approximates the converged
step; the oracle defines the converged step and solves it directly:
Cholesky of A = M + dt G, Schur complement S = P^T A^-1 P for u, then
Idot = A^-1 (P u - R).

Pins (tests/test_oracle_step.py): constraint and KKT residual of the direct
solve, closed-form two-loop recurrence, a 4-loop KKT solved by plain
numpy.linalg.solve, Bean's critical-state moment -Jc a / 3, and the energy
balance of the stepped circuit.

Per-wire statistics (Flux Jumps Propagation and Quenches Propagation
sections: the maximum temperature and the maximum Joule power density of
each wire, the Joule heat Q_FJ of a wire from the occurrence of a flux jump to
its peak, and the Joule heat Q_q from the onset of the rapid increase of rho
to the quench), all from the start-of-step state of every step:

    Q_total[w]  += dt * P_w,  P_w = sum_{e in w} q_e 2 pi r_e a_e   (rectangle rule)
    T_max[w]     = max over steps and elements of T_e
    P_max[w]     = max over steps and elements of q_e
    Q_at_jump[w], Q_at_rise[w], Q_at_quench[w] = Q_total before the step on which
        the wire first meets |J/Jc| > 1, mean rho/rho_n > 0.05 (the onset of the
        rapid rise of rho; the threshold is this build's reading), mean
        rho/rho_n > 0.95 (-1 until then)

so Q_FJ = Q_total(t_peak) - Q_at_jump and Q_q = Q_at_quench - Q_at_rise.
Pins: Q_total of an ohmic loop is I^2 R t; the per-wire Q_total sum to the
time integral of the diagnostic Joule power.

Subelements (Numerical Algorithm section: J = J_H + J_I; the field-driven
part J_H circulates in each subelement with zero net current, the transport
part J_I spreads over the whole wire with its subelements coupled, by the A-V
formulation; both with the resistivity of the total J).  With a group id per
element position of a turn (``groups``), every transport turn tracks J_I as
state; a step first solves J_I on the turn alone (its self block of
M + dt G, the resistive voltage 2 pi r rho J_I, the transport constraint;
``transport_shares``), then the coupled system with one constraint per
subelement fixing its net rate to the J_I share (``subelement_kkt_solve``):
the fields of the other turns and of the background move current only inside
subelements.  Pins (tests/test_oracle_subelement.py): one group per turn
equals the turn-constrained solve, a dense bordered solve, the parallel
inductor division (L2 - M) : (L1 - M), the zero-net invariant under a field
ramp, the resistive division 1/r_k of a held current, outer subelements first.

Lorentz hoop strain (Flux Jumps Propagation section: thermal, pre-strain and
the electromagnetic strain of the Lorentz force set Jc(eps); Quenches
Propagation section, cases 3-5 with electromagnetic strain fields): with
Y_eff > 0 the strain entering Jc is eps = eps0 + r J B_z / Y_eff from the
start-of-step state, the hoop stress r J B_z over an effective Young's modulus
of the winding (this build's reading; the paper's mechanics model is in its
supplement).  Pins (tests/test_oracle_lorentz.py): the magnetic-pressure
closed form of a long thin solenoid, sign and evenness under current reversal,
and the static-strain limit Y_eff -> infinity.
"""

import numpy as np
import scipy.linalg as sla

from .constitutive import critical_current, ej_terms, FILAMENT
from .field import field_from_flux
from .inductance import assemble_M
from .thermal import ThermalGrid

DIAG_FIELDS = ("t", "I_t", "V_term", "moment", "P_joule", "T_max", "max_jratio", "max_rho_frac")


def drive_values(t, d):
    """Transport current I_t(t) and applied axial field B_a(t) of a drive dict.

    I_t = min(ramp_rate * t, I_max).  B_a: waveform 0 = none, 1 = linear ramp
    at Ba_rate capped at Ba_max, 2 = triangle 0 -> +Ba_max -> -Ba_max -> 0 with
    slope Ba_rate, repeated.
    """
    It = min(d["ramp_rate"] * t, d["I_max"])
    wf = d.get("Ba_waveform", 0)
    rate = d.get("Ba_rate", 0.0)
    amp = d.get("Ba_max", 0.0)
    if wf == 0 or rate == 0.0:
        Ba = 0.0
    elif wf == 1:
        Ba = min(rate * t, amp)
    else:
        period = 4.0 * amp / rate
        tau = t - period * np.floor(t / period)
        if tau < 0.25 * period:
            Ba = rate * tau
        elif tau < 0.75 * period:
            Ba = amp - rate * (tau - 0.25 * period)
        else:
            Ba = -amp + rate * (tau - 0.75 * period)
    return It, Ba


def kkt_solve(A, R, c, block, constrained):
    """Exact solution of  A x - P u = -R,  P^T x = c.

    P is the element-to-constrained-block incidence (blocks of ``block``
    consecutive elements, ``constrained`` flags per block).  Returns (x, u)
    with u = 0 on free blocks.
    """
    N = A.shape[0]
    W = N // block
    cho = sla.cho_factor(A, lower=True)
    xR = sla.cho_solve(cho, R)
    wires = np.nonzero(constrained)[0]
    u = np.zeros(W)
    if wires.size == 0:
        return -xR, u
    P = np.zeros((N, wires.size))
    for k, w in enumerate(wires):
        P[w * block:(w + 1) * block, k] = 1.0
    Y = sla.cho_solve(cho, P)
    S = P.T @ Y
    uc = np.linalg.solve(S, c[wires] + P.T @ xR)
    u[wires] = uc
    x = Y @ uc - xR
    return x, u


def transport_shares(A, R_I, c, block, constrained, groups):
    """Rate x_I of the transport part J_I and its per-subelement nets d[w, s].

    Numerical Algorithm section: J = J_H + J_I; the transport part J_I is
    distributed over the whole wire, its subelements coupled, by the A-V
    formulation; the field-driven part J_H, driven by the field of the other
    wires and the background, circulates inside each subelement with zero
    net; both use the resistivity of the total J at the start of the step.
    Reading: J_I of turn w solves the turn's own circuit, its self block
    A_w = M_ww + dt G_w, with the resistive voltage of the transport part
    R_I = 2 pi r rho J_I, under the turn's transport constraint:
        A_w x_I - 1 u = -R_I,w,   1^T x_I = c_w,
    and d[w, s] = sum of x_I over the elements of subelement s.
    """
    N = A.shape[0]
    W = N // block
    S = int(np.max(groups)) + 1
    d = np.zeros((W, S))
    xI = np.zeros(N)
    ones = np.ones(block)
    for w in np.nonzero(constrained)[0]:
        sl = slice(w * block, (w + 1) * block)
        Aw = A[sl, sl]
        y = np.linalg.solve(Aw, ones)
        t = np.linalg.solve(Aw, R_I[sl])
        u = (c[w] + t.sum()) / y.sum()
        xI[sl] = y * u - t
        for g in range(S):
            d[w, g] = xI[sl][groups == g].sum()
    return xI, d


def subelement_kkt_solve(A, R, d, block, constrained, groups):
    """Exact solution of  A x - Q v = -R,  Q^T x = d  with one constraint per
    subelement of every constrained turn (Q = element-to-subelement incidence
    of those turns; free loops stay unconstrained).  The field-driven part of
    the step cannot change a subelement's net current: only the transport
    shares d do.  Returns (x, u, v): v[w, s] the subelement loop voltages,
    u[w] their mean weighted by the subelement's element count (the turn
    voltage reported in the diagnostics; 0 on free loops)."""
    N = A.shape[0]
    W = N // block
    S = int(np.max(groups)) + 1
    wires = np.nonzero(constrained)[0]
    cho = sla.cho_factor(A, lower=True)
    xR = sla.cho_solve(cho, R)
    v = np.zeros((W, S))
    u = np.zeros(W)
    if wires.size == 0:
        return -xR, u, v
    Q = np.zeros((N, wires.size * S))
    rhs = np.zeros(wires.size * S)
    for k, w in enumerate(wires):
        for g in range(S):
            Q[w * block + np.nonzero(groups == g)[0], k * S + g] = 1.0
            rhs[k * S + g] = d[w, g]
    Y = sla.cho_solve(cho, Q)
    Sc = Q.T @ Y
    vc = np.linalg.solve(Sc, rhs + Q.T @ xR)
    x = Y @ vc - xR
    size = np.bincount(groups, minlength=S) / block
    for k, w in enumerate(wires):
        v[w] = vc[k * S:(k + 1) * S]
        u[w] = np.dot(size, v[w])
    return x, u, v


class OracleCoil:
    """State and step of one coil, every quantity in FP64."""

    def __init__(self, geo, params, jc_factor, strain, mat, constrained=None, M=None):
        self.geo = geo
        self.p = dict(params)
        N = geo["N"]
        self.jc_factor = np.asarray(jc_factor, dtype=np.float64)
        self.strain = np.asarray(strain, dtype=np.float64)
        self.mat = np.asarray(mat).astype(np.int64)
        W = geo["W"]
        if constrained is None:
            constrained = np.ones(W, dtype=bool)
        self.constrained = np.asarray(constrained, dtype=bool)
        self.M = assemble_M(geo["r"], geo["z"], geo["h"]) if M is None else M
        # subelements: group id of every element position of a turn (None: one group)
        g = geo.get("groups")
        self.groups = None if g is None or int(np.max(g)) == 0 else np.asarray(g, dtype=np.int64)
        self.I_tr = np.zeros(N)      # transport part J_I a of the element currents (with subelements)
        self.I = np.zeros(N)
        self.u_T = np.full(N, self.p["T_bath"] ** 4)
        self.t = 0.0
        self.steps = 0
        self.diag = []
        self.thermal = ThermalGrid(geo, self.p) if (geo["grid"] and self.p["thermal"]) else None
        self.first_jump = np.full(W, -1, dtype=np.int64)
        self.first_quench = np.full(W, -1, dtype=np.int64)
        self.first_rise = np.full(W, -1, dtype=np.int64)
        self.Q_total = np.zeros(W)
        self.T_max_w = np.zeros(W)
        self.P_max_w = np.zeros(W)
        self.Q_at_jump = np.full(W, -1.0)
        self.Q_at_rise = np.full(W, -1.0)
        self.Q_at_quench = np.full(W, -1.0)
        self.last = None

    # -- the state's fields ----------------------------------------------------
    def temperature(self):
        return np.sqrt(np.sqrt(self.u_T))

    def flux(self):
        return self.M @ self.I

    def field(self, Ba):
        geo = self.geo
        if not geo["grid"]:
            z = np.zeros(geo["N"])
            return z, z.copy()
        phi_tot = self.flux() + np.pi * geo["r"] ** 2 * Ba
        return field_from_flux(geo, phi_tot)

    def strain_now(self, Bz):
        """Element strain: the static strain, plus with Y_eff > 0 the Lorentz
        hoop strain r J B_z / Y_eff of the current state (Flux Jumps Propagation
        section: the electromagnetic strain produced by the Lorentz force; the
        hoop stress of a loop carrying J in the axial field B_z is r J B_z)."""
        Y = self.p.get("Y_eff", 0.0)
        if not Y:
            return self.strain
        J = self.I / self.geo["area"]
        return self.strain + self.geo["r"] * J * Bz / Y

    def pointwise(self, Ba):
        Br, Bz = self.field(Ba)
        Bmag = np.sqrt(Br * Br + Bz * Bz)
        T = self.temperature()
        eps = self.strain_now(Bz)
        Jc = critical_current(Bmag, T, eps, self.jc_factor, self.mat, self.p)
        terms = ej_terms(self.I, Jc, self.mat, self.geo["r"], self.geo["area"], self.p)
        terms.update(Br=Br, Bz=Bz, Bmag=Bmag, T=T, Jc=Jc, eps=eps)
        return terms

    # -- one step ------------------------------------------------------------
    def step(self, drive):
        geo, p = self.geo, self.p
        dt = drive["dt"]
        r, area = geo["r"], geo["area"]
        B = geo["block"]
        W = geo["W"]
        t0, t1 = self.t, self.t + dt
        _, Ba0 = drive_values(t0, drive)
        It1, Ba1 = drive_values(t1, drive)
        dBa = (Ba1 - Ba0) / dt
        pw = self.pointwise(Ba0)
        R = 2.0 * np.pi * r * pw["E"] + np.pi * r * r * dBa
        c = (It1 - self.I.reshape(W, B).sum(axis=1)) / dt
        A = self.M + np.diag(dt * pw["G"])
        if self.groups is None:
            Idot, u = kkt_solve(A, R, c, B, self.constrained)
        else:
            R_I = 2.0 * np.pi * r * pw["rho"] * self.I_tr / area
            xI, d = transport_shares(A, R_I, c, B, self.constrained, self.groups)
            Idot, u, _ = subelement_kkt_solve(A, R, d, B, self.constrained, self.groups)
            self.I_tr = self.I_tr + dt * xI
        self.last = dict(pw, Idot=Idot, u=u, R=R, c=c, A=A)
        # detectors on the start-of-step state (flux-jump |J/Jc| > 1, quench rho > 0.95 rho_n)
        fil = (self.mat == FILAMENT).reshape(W, B)
        jr = np.where(fil, pw["jratio"].reshape(W, B), 0.0)
        rho_frac = np.where(fil, pw["rho"].reshape(W, B) / p["rho_n"], 0.0)
        nfil = fil.sum(axis=1)
        mean_rho = np.where(nfil > 0, rho_frac.sum(axis=1) / np.maximum(nfil, 1), 0.0)
        wire_jr = jr.max(axis=1)
        new_jump = (self.first_jump < 0) & (wire_jr > 1.0)
        new_rise = (self.first_rise < 0) & (mean_rho > 0.05)
        new_quench = (self.first_quench < 0) & (mean_rho > 0.95)
        self.first_jump = np.where(new_jump, self.steps, self.first_jump)
        self.first_rise = np.where(new_rise, self.steps, self.first_rise)
        self.first_quench = np.where(new_quench, self.steps, self.first_quench)
        # per-wire statistics: onsets take the heat accumulated before this step
        self.Q_at_jump = np.where(new_jump, self.Q_total, self.Q_at_jump)
        self.Q_at_rise = np.where(new_rise, self.Q_total, self.Q_at_rise)
        self.Q_at_quench = np.where(new_quench, self.Q_total, self.Q_at_quench)
        P_w = (pw["q"] * 2.0 * np.pi * r * area).reshape(W, B).sum(axis=1)
        self.Q_total = self.Q_total + dt * P_w
        self.T_max_w = np.maximum(self.T_max_w, pw["T"].reshape(W, B).max(axis=1))
        self.P_max_w = np.maximum(self.P_max_w, pw["q"].reshape(W, B).max(axis=1))
        # advance
        self.I = self.I + dt * Idot
        if self.thermal is not None:
            th = self.thermal
            unew = th.adi_step(th.to_grid(self.u_T), th.to_grid(pw["q"]), dt)
            self.u_T = th.to_elem(unew)
        self.t = t1
        self.steps += 1
        rec = (t1, It1, float(u[self.constrained].sum()),
               float(np.sum(np.pi * r * r * self.I)),
               float(np.sum(pw["q"] * 2.0 * np.pi * r * area)),
               float(self.temperature().max()),
               float(wire_jr.max()), float(mean_rho.max()))
        self.diag.append(rec)
        return rec

    def wire_stats(self):
        """Rows Q_total, T_max, P_max, Q_at_jump, Q_at_rise, Q_at_quench, first_rise."""
        return np.stack([self.Q_total, self.T_max_w, self.P_max_w, self.Q_at_jump, self.Q_at_rise,
                         self.Q_at_quench, self.first_rise.astype(np.float64)])

    def read(self, drive=None):
        """J, B_r, B_z, T and moment of the current state."""
        Ba = drive_values(self.t, drive)[1] if drive is not None else 0.0
        pw = self.pointwise(Ba)
        return {"J": pw["J"], "Br": pw["Br"], "Bz": pw["Bz"], "T": pw["T"],
                "moment": float(np.sum(np.pi * self.geo["r"] ** 2 * self.I))}


def build(geometry, material, jc_factor, strain, mat, constrained=None):
    """OracleCoil from a plain geometry dict (solenoid parameters or a list)."""
    from .geometry import solenoid_elements, list_elements
    if geometry["kind"] == "solenoid":
        geo = solenoid_elements(geometry["n_layers"], geometry["n_turns"], geometry["n_sub"],
                                geometry["r_in"], geometry["pitch"], geometry["wire_d"])
        if geometry.get("groups") is not None:
            geo["groups"] = np.asarray(geometry["groups"])
        if constrained is None:
            constrained = np.full(geo["W"], bool(geometry.get("transport", 1)))
    else:
        geo = list_elements(geometry["r"], geometry["z"], geometry["h"], geometry["block"])
        if geometry.get("groups") is not None:
            geo["groups"] = np.asarray(geometry["groups"])
    return OracleCoil(geo, material, jc_factor, strain, mat, constrained)
