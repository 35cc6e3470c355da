"""GPU parity of the per-wire statistics (Flux Jumps Propagation and Quenches
Propagation sections): running Joule heat, maximum temperature and power
density, and the onsets of the flux-jump, resistivity-rise and quench criteria
with the heat accumulated before each, against the FP64 oracle.

Onset step indices are integers decided by FP64 comparisons on both sides and
must match exactly; heat and maxima within 1e-8 relative to the largest value
of their row (the FP64 step itself matches the oracle to about 1e-10)."""
import numpy as np
import pytest

from paper_2403_07666_b300 import build as B
from paper_2403_07666_b300 import workloads as wl
from tests.gpu_common import rel, oracle_of

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _coil(w, **kw):
    from paper_2403_07666_b300.coil import Coil as _C
    return _C.from_workload(w, **kw)


def _jump_coil(seed, n_sub):
    """Low Jc and a fast ramp: every wire passes all three criteria."""
    return wl.random_coil(seed, 2, 3, n_sub, ramp_rate=5e5, material=dict(wl.MATERIAL, Jc0=2e7))


CASES = {
    # 16 elements per wire: segment kernels (several wires per warp)
    "seg-all-onsets": (lambda: _jump_coil(24, 4), 80),
    # 25 elements per wire: one warp per wire
    "warp-all-onsets": (lambda: _jump_coil(25, 5), 80),
    # slower approach, jumps and rises but no quench within the run
    "seg-jump-rise": (lambda: wl.random_coil(21, 3, 4, 4, ramp_rate=5e4,
                                             material=dict(wl.MATERIAL, Jc0=2e8)), 160),
}


def _compare(gs, os_):
    # onset indices: first_rise (row 6) and the Q_at rows' sign pattern
    assert np.array_equal(gs[6], os_[6]), (gs[6], os_[6])
    for row in (0, 2, 3, 4, 5):
        assert rel(gs[row], os_[row]) <= TOL, (row, gs[row], os_[row])
    T_bath = wl.MATERIAL["T_bath"]
    dT = np.max(np.abs(os_[1] - T_bath))
    assert np.max(np.abs(gs[1] - os_[1])) <= TOL * max(dT, 1e-6 * T_bath)


@pytest.mark.parametrize("case", list(CASES))
def test_wire_stats_match_oracle(case):
    make, steps = CASES[case]
    w = make()
    orc = oracle_of(w)
    with _coil(w, rtol=1e-11) as c:
        c.step(steps, w.drive)
        for _ in range(steps):
            orc.step(w.drive)
        gs = c.wire_stats()
        fj, fq = c.onsets()
    os_ = orc.wire_stats()
    assert np.array_equal(fj, orc.first_jump), (fj, orc.first_jump)
    assert np.array_equal(fq, orc.first_quench), (fq, orc.first_quench)
    _compare(gs, os_)
    # the rows are internally consistent: heat only grows after an onset
    met = gs[3] >= 0
    assert np.all(gs[0][met] >= gs[3][met])


def test_onset_heat_tracks_the_step_by_step_heat():
    """Q_at_jump equals Q_total read after exactly first_jump steps."""
    w = _jump_coil(24, 4)
    with _coil(w, rtol=1e-11) as c:
        hist = [c.wire_stats()[0].copy()]
        for _ in range(30):
            c.step(1, w.drive)
            hist.append(c.wire_stats()[0].copy())
        gs = c.wire_stats()
        fj, _ = c.onsets()
    for wi in np.nonzero(fj >= 0)[0]:
        assert gs[3, wi] == hist[fj[wi]][wi]


def test_wire_stats_survive_state_roundtrip_and_reset():
    w = _jump_coil(24, 4)
    with _coil(w) as a, _coil(w) as b:
        a.step(15, w.drive)
        b.load_state(a.save_state())
        assert np.array_equal(a.wire_stats(), b.wire_stats())
        a.step(20, w.drive)
        b.step(20, w.drive)
        assert np.array_equal(a.wire_stats(), b.wire_stats())
        assert np.array_equal(a.onsets()[0], b.onsets()[0])
        b.reset_wire_stats()
        st = b.wire_stats()
        assert np.all(st[:3] == 0.0) and np.all(st[3:] == -1.0)
        fj, fq = b.onsets()
        assert np.all(fj == -1) and np.all(fq == -1)
        # a new window starts from the current state: heat accumulates again
        b.step(5, w.drive)
        assert np.all(b.wire_stats()[0] > 0.0)


def test_adjoint_counts_only_its_forward_steps():
    """The adjoint's checkpoint recomputations and reverse sweep leave the
    statistics as n forward steps do."""
    w = _jump_coil(24, 4)
    K = 25
    with _coil(w) as a, _coil(w) as b:
        a.step(K, w.drive)
        b.adjoint(K, w.drive, np.ones(K), ckpt_every=7)
        assert np.array_equal(a.wire_stats(), b.wire_stats())
        assert np.array_equal(a.onsets()[0], b.onsets()[0])
        # and the coil keeps accumulating after the adjoint
        a.step(3, w.drive)
        b.step(3, w.drive)
        assert np.array_equal(a.wire_stats(), b.wire_stats())
