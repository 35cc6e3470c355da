"""Complete elliptic integrals of the first and second kind (oracle).

The coaxial-loop mutual inductance that carries the field of every wire onto
every other wire (Numerical Algorithm section: H_ext,wire is generated by the
currents of all other wires) is written with K and E.  They are computed here
by Gauss's arithmetic-geometric mean: with a_0 = 1, b_0 = sqrt(1 - m),
c_0 = sqrt(m),

    a_{j+1} = (a_j + b_j)/2,  b_{j+1} = sqrt(a_j b_j),  c_{j+1} = (a_j - b_j)/2,

K(m) = pi / (2 a_inf) and E(m) = K(m) (1 - sum_j 2^{j-1} c_j^2).

Pinned in tests/test_oracle_elliptic.py (K(0) = E(0) = pi/2, the Gamma(1/4)
closed form of K(1/2), Legendre's relation, scipy.special).
"""

import numpy as np


def ellipke(m, mc=None):
    """Return (K(m), E(m)) for parameter m = k^2 in [0, 1).

    ``mc`` = 1 - m may be passed separately when it is known more accurately
    than 1 - m (nearly touching loops).
    """
    m = np.asarray(m, dtype=np.float64)
    if mc is None:
        mc = 1.0 - m
    mc = np.asarray(mc, dtype=np.float64)
    a = np.ones_like(m)
    b = np.sqrt(mc)
    # j = 0 term of the sum: 2^{-1} c_0^2 = m / 2
    acc = 0.5 * m
    weight = 0.5
    for _ in range(64):
        c = 0.5 * (a - b)
        a, b = 0.5 * (a + b), np.sqrt(a * b)
        weight *= 2.0
        acc = acc + weight * c * c
        # stop at the rounding level: a and b may then differ by one ulp forever
        if np.all(np.abs(c) <= 1e-15 * a):
            break
    K = np.pi / (2.0 * a)
    E = K * (1.0 - acc)
    return K, E
