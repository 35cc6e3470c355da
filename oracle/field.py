"""Magnetic field at the element centres from the loop flux (oracle).

The field on each wire (H_ext in the Numerical Algorithm section) is taken
from the flux through every element loop, Phi_tot = M I + pi r^2 B_a:

    B_z = (1 / (2 pi r)) dPhi_tot/dr,    B_r = -(1 / (2 pi r)) dPhi_tot/dz.

Derivatives use the 3-point Lagrange formula on the non-uniform global
element grid (spacing h inside a wire, h + g across an epoxy gap); on the
first and last grid line the one-sided 3-point formula.  A grid line of two
nodes uses the 2-point slope; a single node gets derivative 0.

Pins (tests/test_oracle_field.py): a uniform applied field is reproduced
exactly (pi r^2 is quadratic); the stencil of an external loop's flux agrees
with the loop's elliptic point field.
"""

import numpy as np


def lagrange3_weights(x0, x1, x2, x):
    """Weights (w0, w1, w2) with f'(x) ~ w0 f(x0) + w1 f(x1) + w2 f(x2)."""
    w0 = ((x - x1) + (x - x2)) / ((x0 - x1) * (x0 - x2))
    w1 = ((x - x0) + (x - x2)) / ((x1 - x0) * (x1 - x2))
    w2 = ((x - x0) + (x - x1)) / ((x2 - x0) * (x2 - x1))
    return w0, w1, w2


def derivative_along(f, x, axis):
    """d f / d x along ``axis`` of the 2-D grid array f with node positions x."""
    f = np.moveaxis(np.asarray(f, dtype=np.float64), axis, -1)
    G = x.size
    out = np.zeros_like(f)
    if G == 1:
        return np.moveaxis(out, -1, axis)
    if G == 2:
        slope = (f[..., 1] - f[..., 0]) / (x[1] - x[0])
        out[..., 0] = slope
        out[..., 1] = slope
        return np.moveaxis(out, -1, axis)
    for k in range(G):
        j = min(max(k - 1, 0), G - 3)          # first node of the 3-node stencil
        w0, w1, w2 = lagrange3_weights(x[j], x[j + 1], x[j + 2], x[k])
        out[..., k] = w0 * f[..., j] + w1 * f[..., j + 1] + w2 * f[..., j + 2]
    return np.moveaxis(out, -1, axis)


def field_from_flux(geo, phi_tot):
    """(B_r, B_z) at every element centre from the total loop flux.

    ``phi_tot`` is in element order; the result is in element order.
    """
    Gr, Gz = geo["Gr"], geo["Gz"]
    grid = np.zeros((Gz, Gr))
    grid[geo["i_z"], geo["i_r"]] = phi_tot
    dphi_dr = derivative_along(grid, geo["r_axis"], axis=1)
    dphi_dz = derivative_along(grid, geo["z_axis"], axis=0)
    r = geo["r"]
    Bz = dphi_dr[geo["i_z"], geo["i_r"]] / (2.0 * np.pi * r)
    Br = -dphi_dz[geo["i_z"], geo["i_r"]] / (2.0 * np.pi * r)
    return Br, Bz
