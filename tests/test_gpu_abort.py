"""Failure path of the tensor-core apply, made on purpose without faulting
the GPU: every wait inside k_toeplitz_tc on an mbarrier is bounded, and a
wait that runs out raises the CTA's abort flag.  coil_set_wait_limit
shortens the limit of those waits to a single cycle, so the next apply stops
early; the step must then report COIL_ERR_CUDA, keep the state of the last
completed step, leave the context usable, and the coil must step on normally
once the limit is restored."""
import numpy as np
import pytest

from paper_2403_07666_b300 import build as B
from paper_2403_07666_b300 import workloads as wl
from tests.gpu_common import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


@pytest.mark.parametrize("profile", [False, True], ids=["graph", "one_by_one"])
def test_tensor_core_wait_timeout_is_reported_and_recovers(profile):
    from paper_2403_07666_b300.coil import Coil, CoilError, ERR_CUDA
    w = wl.random_coil(94, 4, 6, 4, material=dict(wl.MATERIAL, Jc0=2e8), ramp_rate=1e5)
    kw = dict(precision="fp32", format="toeplitz_tc", rtol=1e-11)
    with Coil.from_workload(w, profile=profile, **kw) as c, Coil.from_workload(w, **kw) as ref:
        c.step(3, w.drive)
        ref.step(3, w.drive)
        I3 = c.currents()
        T3 = c.read(w.drive)["T"]
        c.set_wait_limit(1)
        for _ in range(2):                      # twice: the stopped apply leaves nothing behind
            with pytest.raises(CoilError) as ei:
                c.step(1, w.drive)
            assert ei.value.status == ERR_CUDA
            assert "timed out" in str(ei.value)
            assert c.info().steps == 3
            assert np.array_equal(c.currents(), I3)
            assert np.array_equal(c.read(w.drive)["T"], T3)
        c.set_wait_limit(0)
        c.step(6, w.drive)
        ref.step(6, w.drive)
        assert c.info().steps == 9
        got, want = c.read(w.drive), ref.read(w.drive)
        # both solved to rtol 1e-11 from the same state; the warm starts differ,
        # so the FP32-class operator rounds different inputs: the tensor-core
        # form's parity bound (1e-5 of each field's maximum) applies
        assert rel(got["J"], want["J"]) < 1e-5
        assert rel(got["Bz"], want["Bz"]) < 1e-5
        assert np.max(np.abs(got["T"] - want["T"])) < 1e-5 * np.max(np.abs(want["T"] - w.material["T_bath"]))


def test_wait_limit_rejects_negative():
    from paper_2403_07666_b300.coil import Coil, CoilError, ERR_INVALID
    w = wl.random_coil(95, 2, 3, 4)
    with Coil.from_workload(w, precision="fp32", format="toeplitz_tc") as c:
        with pytest.raises(CoilError) as ei:
            c.set_wait_limit(-5)
        assert ei.value.status == ERR_INVALID
