"""Coaxial-loop inductances and the dense Green's operator M (oracle).

Every conductor element of the axisymmetric cross-section is a coaxial
current loop (Numerical Algorithm section: the solenoid is reduced to its
(r, z) cross-section; the field on each wire comes from the currents of all
other wires plus the background field).  M[i, j] is the flux through loop i
per ampere in loop j:

* far pairs (i != j, centre distance >= NEAR_RADIUS * max(h_i, h_j)):
  Maxwell's formula at the element centres,
      M = mu0 sqrt(r1 r2) [ (2/k - k) K(k) - (2/k) E(k) ],
      k^2 = 4 r1 r2 / ((r1 + r2)^2 + (z1 - z2)^2);
* near pairs: the same formula averaged over both element squares with a
  4 x 4-point Gauss-Legendre rule on each square (256 point pairs);
* i == j: the thin-ring self inductance with the square's geometric mean
  distance, L = mu0 r (ln(8 r / (GMD_SQUARE h)) - 2).

Pins (tests/test_oracle_inductance.py): far-field dipole limit, near-field
logarithmic limit, the flux of the loop point-field integrated over the
second loop's disk, the GMD constant against its defining 4-D integral,
symmetry and positive definiteness of M.
"""

import numpy as np

from .elliptic import ellipke

MU0 = 4.0e-7 * np.pi
GMD_SQUARE = 0.44705      # geometric mean distance of a square / its side
NEAR_RADIUS = 3.1         # near pairs: centre distance < 3.1 element sides

# 4-point Gauss-Legendre rule on [-1, 1]
_s = np.sqrt(6.0 / 5.0)
GL4_X = np.array([-np.sqrt(3.0 / 7.0 + 2.0 / 7.0 * _s), -np.sqrt(3.0 / 7.0 - 2.0 / 7.0 * _s),
                  np.sqrt(3.0 / 7.0 - 2.0 / 7.0 * _s), np.sqrt(3.0 / 7.0 + 2.0 / 7.0 * _s)])
GL4_W = np.array([(18.0 - np.sqrt(30.0)) / 36.0, (18.0 + np.sqrt(30.0)) / 36.0,
                  (18.0 + np.sqrt(30.0)) / 36.0, (18.0 - np.sqrt(30.0)) / 36.0])


def mutual_point(r1, z1, r2, z2):
    """Maxwell's mutual inductance of two coaxial filament loops [H]."""
    r1, z1, r2, z2 = (np.asarray(v, dtype=np.float64) for v in (r1, z1, r2, z2))
    dz2 = (z1 - z2) ** 2
    den = (r1 + r2) ** 2 + dz2
    m = 4.0 * r1 * r2 / den
    mc = ((r1 - r2) ** 2 + dz2) / den
    K, E = ellipke(m, mc)
    k = np.sqrt(m)
    return MU0 * np.sqrt(r1 * r2) * ((2.0 / k - k) * K - (2.0 / k) * E)


def self_inductance(r, h):
    """Self inductance of a loop of radius r with a square h x h section."""
    r = np.asarray(r, dtype=np.float64)
    return MU0 * r * (np.log(8.0 * r / (GMD_SQUARE * h)) - 2.0)


def near_average(ri, zi, hi, rj, zj, hj):
    """Mean of the point formula over both squares (4x4 GL points each).

    Arrays of pairs in, array of averaged inductances out.
    """
    ri, zi, hi, rj, zj, hj = (np.asarray(v, dtype=np.float64)[:, None]
                              for v in (ri, zi, hi, rj, zj, hj))
    # the 16 nodes and weights of the tensor rule on one square (weights sum to 1)
    xr, xz = np.meshgrid(GL4_X, GL4_X, indexing="ij")
    wq = np.outer(GL4_W, GL4_W).ravel() / 4.0
    xr, xz = xr.ravel(), xz.ravel()
    total = np.zeros(ri.shape[0])
    for p in range(16):
        r1 = ri + 0.5 * hi * xr[p]
        z1 = zi + 0.5 * hi * xz[p]
        r2 = rj + 0.5 * hj * xr[None, :]
        z2 = zj + 0.5 * hj * xz[None, :]
        vals = mutual_point(r1, z1, r2, z2)          # (pairs, 16)
        total += wq[p] * (vals @ wq)
    return total


def near_mask(r, z, h, rows, cols):
    """True where (rows[i], cols[j]) is a near pair by the centre-distance rule."""
    hmax = np.maximum(h[rows][:, None], h[cols][None, :])
    d2 = (r[rows][:, None] - r[cols][None, :]) ** 2 + (z[rows][:, None] - z[cols][None, :]) ** 2
    return d2 < (NEAR_RADIUS * hmax) ** 2


def assemble_M(r, z, h, chunk=256):
    """Dense N x N mutual-inductance operator of the element loops."""
    r = np.asarray(r, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    N = r.size
    M = np.empty((N, N))
    cols = np.arange(N)
    near_i, near_j = [], []
    for i0 in range(0, N, chunk):
        rows = np.arange(i0, min(N, i0 + chunk))
        with np.errstate(divide="ignore", invalid="ignore"):
            M[rows] = mutual_point(r[rows][:, None], z[rows][:, None], r[None, :], z[None, :])
        nm = near_mask(r, z, h, rows, cols)
        ii, jj = np.nonzero(nm)
        keep = rows[ii] < jj                      # each unordered near pair once
        near_i.append(rows[ii][keep])
        near_j.append(jj[keep])
    ni = np.concatenate(near_i)
    nj = np.concatenate(near_j)
    for s in range(0, ni.size, 4096):
        a, b = ni[s:s + 4096], nj[s:s + 4096]
        v = near_average(r[a], z[a], h[a], r[b], z[b], h[b])
        M[a, b] = v
        M[b, a] = v
    M[cols, cols] = self_inductance(r, h)
    return M


def loop_field(a, z0, I, r, z):
    """(B_r, B_z) at points (r, z) of a filament loop of radius a at height z0.

    Standard elliptic-integral form of the Biot-Savart law for a circular
    loop; on the axis (r = 0) B_r = 0 and B_z = mu0 I a^2 / (2 (a^2 + dz^2)^1.5).
    """
    r = np.asarray(r, dtype=np.float64)
    dz = np.asarray(z, dtype=np.float64) - z0
    den = (a + r) ** 2 + dz ** 2
    gap2 = (a - r) ** 2 + dz ** 2
    m = 4.0 * a * r / den
    K, E = ellipke(m, gap2 / den)
    pref = MU0 * I / (2.0 * np.pi * np.sqrt(den))
    Bz = pref * (K + (a * a - r * r - dz * dz) / gap2 * E)
    with np.errstate(divide="ignore", invalid="ignore"):
        Br = np.where(r > 0.0, pref * dz / r * (-K + (a * a + r * r + dz * dz) / gap2 * E), 0.0)
    return Br, Bz


def operator_rows(r, z, h, rows):
    """Rows `rows` of the dense operator (same definition as assemble_M),
    computed one row at a time for coils too large to assemble."""
    r = np.asarray(r, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    rows = np.asarray(rows)
    N = r.size
    out = np.empty((rows.size, N))
    for k, i in enumerate(rows):
        with np.errstate(divide="ignore", invalid="ignore"):
            out[k] = mutual_point(r[i], z[i], r, z)
        hmax = np.maximum(h[i], h)
        near = ((r[i] - r) ** 2 + (z[i] - z) ** 2) < (NEAR_RADIUS * hmax) ** 2
        near[i] = False
        j = np.nonzero(near)[0]
        # average with the lower index first, as assemble_M does for each pair
        lo = np.minimum(i, j)
        hi = np.maximum(i, j)
        out[k, j] = near_average(r[lo], z[lo], h[lo], r[hi], z[hi], h[hi])
        out[k, i] = self_inductance(r[i], h[i])
    return out
