"""Element tables of the axisymmetric coil cross-section (oracle).

Numerical Algorithm section and Fig. 2a: the solenoid is reduced to its
(r, z) cross-section; the wires sit on a square (not triangular) array of
N_x x N_y turns labelled (i, j).  Each wire is taken here as a square of side
d on a pitch p (epoxy gap g = p - d centred between wires), divided into
n x n square elements of side h = d / n.  Wire (l, t) (layer l radial, turn t
axial) spans r in [R_in + g/2 + l p, + d] and z in [-N_T p/2 + g/2 + t p, + d].

Element order (shared with the library ABI by definition, not by code):
    e = (t * N_L + l) * n^2 + b * n + a,
with (a, b) the radial / axial element index inside the wire.  Wire
(block) index w = t * N_L + l.  Global grid indices: i_r = l n + a,
i_z = t n + b.
"""

import numpy as np


def solenoid_elements(n_layers, n_turns, n_sub, r_in, pitch, wire_d):
    """Element table of a regular solenoid; returns a dict of arrays."""
    NL, NT, n = int(n_layers), int(n_turns), int(n_sub)
    g = pitch - wire_d
    h = wire_d / n
    N = NL * NT * n * n
    e = np.arange(N)
    a = e % n
    b = (e // n) % n
    w = e // (n * n)
    l = w % NL
    t = w // NL
    r = r_in + 0.5 * g + l * pitch + (a + 0.5) * h
    z = -0.5 * NT * pitch + 0.5 * g + t * pitch + (b + 0.5) * h
    i_r = l * n + a
    i_z = t * n + b
    # grid axes: the radius of every grid column, the height of every grid row
    Gr, Gz = NL * n, NT * n
    col = np.arange(Gr)
    row = np.arange(Gz)
    r_axis = r_in + 0.5 * g + (col // n) * pitch + (col % n + 0.5) * h
    z_axis = -0.5 * NT * pitch + 0.5 * g + (row // n) * pitch + (row % n + 0.5) * h
    return {
        "N": N, "block": n * n, "W": NL * NT, "n": n, "NL": NL, "NT": NT,
        "h_elem": h, "gap": g,
        "r": r, "z": z, "h": np.full(N, h), "area": np.full(N, h * h),
        "wire": w, "i_r": i_r, "i_z": i_z, "Gr": Gr, "Gz": Gz,
        "r_axis": r_axis, "z_axis": z_axis,
        # face kind along r between grid column c and c+1: True = epoxy gap
        "gap_r": ((col[:-1] + 1) % n) == 0,
        "gap_z": ((row[:-1] + 1) % n) == 0,
        "grid": True,
    }


def list_elements(r, z, h, block):
    """Explicit element list (free loops, brute-force pins): no grid."""
    r = np.asarray(r, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    N = r.size
    if N % block:
        raise ValueError("element count must be a multiple of the block size")
    return {
        "N": N, "block": int(block), "W": N // block,
        "r": r, "z": z, "h": h, "area": h * h,
        "wire": np.arange(N) // block, "grid": False,
    }
