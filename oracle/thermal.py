"""Heat diffusion with T^3 laws, Robin bath sink and ADI (oracle).

Methods, heat-diffusion paragraph: c dT/dt = div(kappa grad T) + E.J on the
coil cross-section, -kappa grad T . n = h (T - T0) on its four borders,
c, kappa, h all proportional to T^3, solved by the alternating-direction
implicit method on the composite (superconductor / Cu / epoxy) section.

With c = c0 T^3 (per kg, density rho_m), kappa = kappa_ref (T/T_ref)^3 and
the Kirchhoff variable u = T^4 the bulk equation is linear:

    (rho_m c0 / 4) du/dt = div( kappa_ref / (4 T_ref^3) grad u ) + q.

Finite volumes on the element grid, per unit depth (planar, as the paper
writes the operator on the cross-section):
  * cell capacity            C = rho_m c0 h^2 / 4
  * face inside a wire       K_in  = kappa_cu / (4 T_ref^3)
  * face across an epoxy gap K_gap = h / (h / kappa_cu + g / kappa_ep) / (4 T_ref^3)
    (half cell of Cu, the gap of epoxy, half cell of Cu in series; the epoxy
    stores no heat)
  * each border face loses   h * h0 (T/T_ref)^3 (T - T_bath), evaluated at the
    start of the step (explicit)

Peaceman-Rachford with the source s = (4 / (rho_m c0)) (q - loss / h^2):
    (I - dt/2 A_r) u*      = (I + dt/2 A_z) u^k + dt/2 s
    (I - dt/2 A_z) u^{k+1} = (I + dt/2 A_r) u*  + dt/2 s
and T = u^{1/4}.

Pins (tests/test_oracle_thermal.py): the decay rate of one isolated element
(the T^3 laws cancel), exact conservation of sum(u) without bath, the
closed-form Peaceman-Rachford amplification of a cosine mode, and one step
against a dense solve of the two half-step systems.
"""

import numpy as np


def thomas(lower, diag, upper, rhs):
    """Solve tridiagonal systems along the last axis of ``rhs`` (same matrix)."""
    n = diag.size
    cp = np.zeros(n)
    dp = np.zeros_like(rhs)
    cp[0] = upper[0] / diag[0] if n > 1 else 0.0
    dp[..., 0] = rhs[..., 0] / diag[0]
    for i in range(1, n):
        den = diag[i] - lower[i] * cp[i - 1]
        if i < n - 1:
            cp[i] = upper[i] / den
        dp[..., i] = (rhs[..., i] - lower[i] * dp[..., i - 1]) / den
    x = np.zeros_like(rhs)
    x[..., n - 1] = dp[..., n - 1]
    for i in range(n - 2, -1, -1):
        x[..., i] = dp[..., i] - cp[i] * x[..., i + 1]
    return x


class ThermalGrid:
    """Thermal operator of a solenoid element grid."""

    def __init__(self, geo, p):
        self.geo = geo
        self.p = p
        h = geo["h_elem"]
        g = geo["gap"]
        T3 = 4.0 * p["T_ref"] ** 3
        self.K_in = p["kappa_cu"] / T3
        if g > 0.0:
            self.K_gap = h / (h / p["kappa_cu"] + g / p["kappa_ep"]) / T3
        else:
            self.K_gap = self.K_in
        self.C = p["rho_m"] * p["c0"] * h * h / 4.0
        self.h = h
        # face conductances between consecutive grid columns / rows
        self.Kr = np.where(geo["gap_r"], self.K_gap, self.K_in)
        self.Kz = np.where(geo["gap_z"], self.K_gap, self.K_in)
        Gr, Gz = geo["Gr"], geo["Gz"]
        cols = np.arange(Gr)
        rows = np.arange(Gz)
        self.n_border = ((cols[None, :] == 0).astype(float) + (cols[None, :] == Gr - 1)
                         + (rows[:, None] == 0) + (rows[:, None] == Gz - 1))

    # -- grid <-> element order -------------------------------------------
    def to_grid(self, v):
        out = np.zeros((self.geo["Gz"], self.geo["Gr"]))
        out[self.geo["i_z"], self.geo["i_r"]] = v
        return out

    def to_elem(self, grid):
        return grid[self.geo["i_z"], self.geo["i_r"]]

    # -- operators -----------------------------------------------------------
    def apply_axis(self, u, K, axis):
        """A u along one axis: (1/C) sum over the two faces of K (u_nb - u)."""
        u = np.moveaxis(u, axis, -1)
        out = np.zeros_like(u)
        flux = K * (u[..., 1:] - u[..., :-1])     # from cell i+1 into cell i
        out[..., :-1] += flux
        out[..., 1:] -= flux
        return np.moveaxis(out / self.C, -1, axis)

    def tridiag(self, K, half_dt):
        """Coefficients of (I - half_dt A) along one axis."""
        n = K.size + 1
        lower = np.zeros(n)
        upper = np.zeros(n)
        diag = np.ones(n)
        c = half_dt / self.C
        lower[1:] = -c * K
        upper[:-1] = -c * K
        diag[1:] += c * K
        diag[:-1] += c * K
        return lower, diag, upper

    def source(self, u, q):
        """s = (4/(rho_m c0)) (q - border loss / h^2), on the grid."""
        p = self.p
        T = np.sqrt(np.sqrt(u))
        loss = self.n_border * self.h * p["h0"] * (T / p["T_ref"]) ** 3 * (T - p["T_bath"])
        return 4.0 / (p["rho_m"] * p["c0"]) * (q - loss / (self.h * self.h))

    def adi_step(self, u, q, dt):
        """One Peaceman-Rachford step on grid arrays u (= T^4) and q [W/m^3]."""
        s = self.source(u, q)
        hd = 0.5 * dt
        rhs1 = u + hd * self.apply_axis(u, self.Kz, axis=0) + hd * s
        lo, di, up = self.tridiag(self.Kr, hd)
        ustar = thomas(lo, di, up, rhs1)                       # r-lines (axis 1)
        rhs2 = ustar + hd * self.apply_axis(ustar, self.Kr, axis=1) + hd * s
        lo, di, up = self.tridiag(self.Kz, hd)
        unew = thomas(lo, di, up, rhs2.T).T                    # z-lines (axis 0)
        return unew
