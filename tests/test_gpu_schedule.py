"""Schedules of the tensor-core apply and their autotuner.

The apply has two kernels with the same arithmetic per product (FP16 hi/lo
splits, three products per K step, FP32 accumulation per stage): the
two-fill one (every stored tile loaded by the CTAs of both of its products)
and the one-fill one (one load serves the tile and its transpose).  Each must
match the oracle's operator and march a coil like the oracle; the autotuner
must keep the fastest candidate it timed."""
import numpy as np
import pytest

from paper_2403_07666_b300 import build as B
from paper_2403_07666_b300 import workloads as wl
from tests.gpu_common import compare_state, oracle_of, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


# (layers, turns, n): one and several channel tiles and k blocks, ragged tiles
SHAPES = [(2, 9, 4), (5, 13, 4), (9, 7, 4), (3, 20, 6)]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("L,T,n", SHAPES)
def test_both_kernels_apply_the_oracle_operator(mode, L, T, n):
    from paper_2403_07666_b300.coil import Coil
    w = wl.random_coil(131, L, T, n)
    rng = np.random.default_rng(3)
    p = rng.standard_normal(w.n_elem)
    with Coil.from_workload(w, precision="fp32", format="toeplitz_tc") as c:
        c.set_tc_schedule(mode)
        sch = c.tc_schedule()
        assert sch["mode"] == mode
        y = c.apply_operator(p)
        y2 = c.apply_operator(p * 3.0)
    M = oracle_of(w).M
    assert rel(y, M @ p) < 2e-6
    assert rel(y2, M @ (3.0 * p)) < 2e-6


@pytest.mark.parametrize("mode", [0, 1])
def test_both_kernels_march_like_the_oracle(mode):
    from paper_2403_07666_b300.coil import Coil
    w = wl.random_coil(132, 5, 9, 4, material=dict(wl.MATERIAL, Jc0=2e8), ramp_rate=5e5)
    orc = oracle_of(w)
    with Coil.from_workload(w, precision="fp32", format="toeplitz_tc", rtol=1e-11) as c:
        c.set_tc_schedule(mode)
        for _ in range(3):
            c.step(20, w.drive)
            for _ in range(20):
                orc.step(w.drive)
            compare_state(c.read(w.drive), orc, w.drive, w.material["T_bath"], 1e-5, 1e-5, 1e-5)


def test_autotuner_keeps_its_fastest_candidate_and_retunes():
    from paper_2403_07666_b300.coil import Coil
    w = wl.random_coil(133, 6, 16, 4)
    with Coil.from_workload(w, precision="fp32", format="toeplitz_tc") as c:
        sch = c.tc_schedule()
        cand = np.array(sch["candidates"])
        assert len(cand) >= 2 and set(cand[:, 0]) == {0.0, 1.0}
        best = cand[np.argmin(cand[:, 3])]
        assert (sch["mode"], sch["n_cta"], sch["stages"]) == (int(best[0]), int(best[1]), int(best[2]))
        assert sch["us"] == pytest.approx(best[3])
        c.set_tc_schedule(-1)                 # tune again: a valid schedule, candidates timed anew
        sch2 = c.tc_schedule()
        assert sch2["us"] > 0 and len(sch2["candidates"]) == len(cand)


def test_schedule_calls_reject_other_formats_and_bad_schedules():
    from paper_2403_07666_b300.coil import Coil, CoilError, ERR_INVALID
    w = wl.random_coil(134, 2, 5, 4)
    with Coil.from_workload(w, precision="fp32") as c:
        with pytest.raises(CoilError) as ei:
            c.tc_schedule()
        assert ei.value.status == ERR_INVALID
    with Coil.from_workload(w, precision="fp32", format="toeplitz_tc") as c:
        for bad in ((2, 0, 0), (0, 5, 0), (1, 0, 99)):
            with pytest.raises(CoilError) as ei:
                c.set_tc_schedule(*bad)
            assert ei.value.status == ERR_INVALID
