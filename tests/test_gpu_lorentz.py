"""GPU parity of the Lorentz hoop strain (Flux Jumps Propagation section: the
electromagnetic strain of the Lorentz force entering Jc(eps)): per-step J, B,
T and diagnostics of the FP64 path with Y_eff > 0 against the oracle, for both
pointwise kernels, within the FP64 parity bound 1e-5 of the static-strain
tests; and the coupling is live (the trajectory departs from the static one)."""
import numpy as np
import pytest

from paper_2403_07666_b300 import build as B
from paper_2403_07666_b300 import workloads as wl
from tests.gpu_common import rel, oracle_of, compare_state

pytestmark = pytest.mark.gpu

TOL64 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _coil(w, **kw):
    from paper_2403_07666_b300.coil import Coil as _C
    return _C.from_workload(w, **kw)


def _lorentz_coil(seed, n_sub, Y_eff=2e8):
    return wl.random_coil(seed, 2, 3, n_sub, ramp_rate=5e5,
                          material=dict(wl.MATERIAL, Jc0=2e7, Y_eff=Y_eff))


@pytest.mark.parametrize("seed,n_sub", [(41, 4), (43, 5), (44, 8)])
def test_lorentz_steps_match_oracle(seed, n_sub):
    w = _lorentz_coil(seed, n_sub)
    orc = oracle_of(w)
    worst = np.zeros(4)
    with _coil(w, rtol=1e-11) as c:
        for k in range(50):
            c.step(1, w.drive)
            orc.step(w.drive)
            if (k + 1) % 5 == 0:
                e = compare_state(c.read(w.drive), orc, w.drive, w.material["T_bath"], TOL64, TOL64, TOL64)
                worst = np.maximum(worst, e)
        dg = c.diag()
        fj, fq = c.onsets()
    do = np.array(orc.diag)
    for j in range(8):
        scale = np.max(np.abs(do[:, j]))
        if np.isfinite(scale) and scale > 0:
            assert np.max(np.abs(dg[:, j] - do[:, j])) <= TOL64 * scale, j
    assert np.array_equal(fj, orc.first_jump)
    assert np.array_equal(fq, orc.first_quench)


def test_lorentz_coupling_is_live_and_static_limit_is_exact():
    w_on = _lorentz_coil(41, 4)
    w_off = _lorentz_coil(41, 4, Y_eff=0.0)
    w_inf = _lorentz_coil(41, 4, Y_eff=1e300)
    with _coil(w_on) as a, _coil(w_off) as b, _coil(w_inf) as s:
        for c, w in ((a, w_on), (b, w_off), (s, w_inf)):
            c.step(30, w.drive)
        Ia, Ib, Is = a.currents(), b.currents(), s.currents()
    assert np.array_equal(Ib, Is)
    assert rel(Ia, Ib) > 1e-6


def test_reversed_drive_mirrors_the_trajectory():
    w = _lorentz_coil(41, 4)
    rev = dict(w.drive, ramp_rate=-w.drive["ramp_rate"])
    with _coil(w) as a, _coil(w) as b:
        a.step(25, w.drive)
        b.step(25, rev)
        Ia, Ib = a.currents(), b.currents()
    assert np.max(np.abs(Ia + Ib)) <= 1e-9 * np.max(np.abs(Ia))


def test_negative_young_modulus_rejected():
    from paper_2403_07666_b300.coil import CoilError, ERR_INVALID
    w = _lorentz_coil(41, 4, Y_eff=-1.0)
    with pytest.raises(CoilError) as ei:
        _coil(w)
    assert ei.value.status == ERR_INVALID
