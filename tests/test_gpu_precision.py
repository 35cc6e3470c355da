"""The mixed form against the plain FP64 form on a trajectory into flux flow.

Mixed form: the far operator as the tensor-core block-Toeplitz product (FP16
hi/lo pairs, FP32-class) and the field and constitutive chain in FP32; the
per-wire constraint solve and the accumulation of current, flux and
temperature stay FP64.  Plain form: the dense FP64 operator and the FP64
chain.  Both step the same 8 x 8-element wires (3,072 elements) from t = 0
on a fast ramp with a reduced Jc0, so that the filaments pass |J|/Jc = 1
and carry flux flow within the window.  After every step: J, B and the
heating T - T_bath within 1e-3, 1e-4 and 1e-3 of the step's maximum, the
moment within 1e-4 of the largest |m| so far (the mixed-precision bounds)."""
import numpy as np
import pytest

from paper_2403_07666_b300 import build as B
from paper_2403_07666_b300 import workloads as wl

pytestmark = pytest.mark.gpu

BOUNDS = {"J": 1e-3, "B": 1e-4, "T": 1e-3, "m": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _rel(a, b):
    sc = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / sc)


def test_mixed_form_within_bounds_of_fp64_through_flux_flow():
    from paper_2403_07666_b300.coil import Coil
    w = wl.solenoid("precision-4x12x8", 4, 12, 8, 7666101, ramp_rate=1e5, I_max=4000.0,
                    material=dict(wl.MATERIAL, Jc0=5e9))
    Tb = w.material["T_bath"]
    steps = 400
    worst = dict.fromkeys(BOUNDS, 0.0)
    m_scale = 0.0
    with Coil.from_workload(w, precision="fp64", rtol=1e-10) as c64, \
            Coil.from_workload(w, precision="fp32", format="toeplitz_tc", rtol=1e-10) as cm:
        for _ in range(steps):
            c64.step(1, w.drive)
            cm.step(1, w.drive)
            ref, got = c64.read(w.drive), cm.read(w.drive)
            m_scale = max(m_scale, abs(ref["moment"]))
            worst["J"] = max(worst["J"], _rel(got["J"], ref["J"]))
            worst["B"] = max(worst["B"], _rel(got["Br"], ref["Br"]), _rel(got["Bz"], ref["Bz"]))
            heat = max(np.max(np.abs(ref["T"] - Tb)), 1e-6 * Tb)
            worst["T"] = max(worst["T"], float(np.max(np.abs(got["T"] - ref["T"])) / heat))
            worst["m"] = max(worst["m"], abs(got["moment"] - ref["moment"]) / m_scale)
        d64 = c64.diag()
    assert np.max(d64[:, 6]) > 1.1                       # the filaments went past Jc
    assert np.max(d64[:, 5]) > Tb + 0.05                 # and heated
    for k, bound in BOUNDS.items():
        assert worst[k] <= bound, (k, worst[k], worst)
