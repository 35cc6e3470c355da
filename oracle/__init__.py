"""FP64 CPU oracle for the coupled electromagnetic-thermal coil update.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2403_07666_b300``) never imports it and
shares no code with it: the two meet only through the seeded input arrays of
``paper_2403_07666_b300.workloads``, which holds none of the method's
arithmetic.

The oracle is a plain, slow, vectorised-numpy restatement of the method of
arXiv:2403.07666 ("Holistic numerical simulation of a quenching process on a
real-size multifilamentary superconducting coil"):

* ``elliptic``     complete elliptic integrals K, E (Gauss AGM)
* ``inductance``   coaxial-loop mutual inductance, self term, dense operator
                   and the loop point-field (Numerical Algorithm section,
                   the field H_ext on each wire from all other wires)
* ``geometry``     axisymmetric cross-section, square wire array, n x n
                   elements per wire (Numerical Algorithm section, Fig. 2a)
* ``field``        B from the loop flux by a 3-point stencil
* ``constitutive`` E-J law with Jc(B,T,eps) (Methods, E-J paragraph)
* ``thermal``      heat equation with T^3 laws, Robin bath sink, ADI
                   (Methods, heat-diffusion paragraph)
* ``step``         the per-step constrained solve (A-V transport constraint)
                   solved exactly by Cholesky + Schur complement, and the
                   linearly-implicit Euler time step
* ``tangent``      forward-mode derivatives of the step series (moment and
                   Joule power) with respect to the calibration parameters,
                   by the complex step (the adjoint's reference)

Parity status: every function above is pinned by ``tests/test_oracle_*.py``
against closed forms, library special functions, brute force or invariants.
Flux-jump onset after the instability is "parity unpinned" physically (the
avalanche is chaotic); it is compared GPU-vs-oracle only.
"""

from .elliptic import ellipke  # noqa: F401
from .inductance import (MU0, mutual_point, self_inductance,  # noqa: F401
                         near_average, assemble_M, loop_field, GMD_SQUARE)
from .geometry import solenoid_elements, list_elements  # noqa: F401
from .field import field_from_flux  # noqa: F401
from .constitutive import critical_current, ej_terms  # noqa: F401
from .thermal import ThermalGrid  # noqa: F401
from .step import (OracleCoil, kkt_solve, transport_shares, subelement_kkt_solve, drive_values,  # noqa: F401
                   build, DIAG_FIELDS)
