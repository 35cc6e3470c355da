"""GPU parity of the subelement decoupling (Numerical Algorithm section:
J = J_H + J_I, the field-driven part with zero net current in every
subelement, the transport part shared by the coupled subelements of the whole
wire): per-step J, B, T, diagnostics and onsets of the FP64 path against the
oracle within the FP64 parity bound 1e-5; the zero-net invariant, which the
projected solve enforces in any operator precision; state round trip of the
transport part; the refusals."""
import numpy as np
import pytest

from paper_2403_07666_b300 import build as B
from paper_2403_07666_b300 import workloads as wl
from tests.gpu_common import oracle_of, compare_state

pytestmark = pytest.mark.gpu

TOL64 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _coil(w, **kw):
    from paper_2403_07666_b300.coil import Coil as _C
    return _C.from_workload(w, **kw)


def _grouped(seed, L, T, n, tile=None, **kw):
    kw.setdefault("material", dict(wl.MATERIAL, Jc0=2e7))
    kw.setdefault("ramp_rate", 5e5)
    w = wl.random_coil(seed, L, T, n, **kw)
    w.geometry["groups"] = wl.subelement_groups(n, tile)
    return w


@pytest.mark.parametrize("seed,L,T,n,tile", [(71, 2, 3, 4, None), (72, 3, 4, 3, None), (73, 3, 3, 2, None),
                                             (74, 2, 3, 5, None), (75, 2, 3, 8, 2)])
def test_subelement_steps_match_oracle(seed, L, T, n, tile):
    """Cu ring + filament quadrants (n = 4: 5 groups of a 16-element turn;
    n = 3: 4 groups of 9, a padded segment; n = 2: single-element groups;
    n = 5: one warp per turn) and Cu ring + nine 2 x 2 subelements of a
    64-element turn (n = 8)."""
    w = _grouped(seed, L, T, n, tile)
    orc = oracle_of(w)
    with _coil(w, rtol=1e-11) as c:
        for k in range(50):
            c.step(1, w.drive)
            orc.step(w.drive)
            if (k + 1) % 5 == 0:
                compare_state(c.read(w.drive), orc, w.drive, w.material["T_bath"], TOL64, TOL64, TOL64)
        dg = c.diag()
        fj, fq = c.onsets()
        I = c.currents()
    do = np.array(orc.diag)
    for j in range(8):
        scale = np.max(np.abs(do[:, j]))
        if np.isfinite(scale) and scale > 0:
            assert np.max(np.abs(dg[:, j] - do[:, j])) <= TOL64 * scale, j
    assert np.array_equal(fj, orc.first_jump)
    assert np.array_equal(fq, orc.first_quench)
    # every turn still carries I_t
    It = 50 * w.drive["dt"] * w.drive["ramp_rate"]
    assert np.max(np.abs(I.reshape(-1, n * n).sum(axis=1) - It)) <= 1e-9 * It


@pytest.mark.parametrize("fmt,prec,n,tile", [("dense", "fp64", 4, None), ("toeplitz_tc", "fp32", 4, None),
                                             ("dense", "fp64", 8, 2)])
def test_field_ramp_keeps_every_subelement_net_zero(fmt, prec, n, tile):
    """No transport current, a ramping applied field: the nets of all
    subelements stay zero (up to rounding) in any operator precision."""
    w = _grouped(74, 3, 4, n, tile, ramp_rate=0.0, I_max=0.0, dt=1e-4, Ba_rate=40.0, Ba_max=0.05,
                 Ba_waveform=1, material=dict(wl.MATERIAL, Jc0=2e8))
    grp = w.geometry["groups"]
    peak = net = 0.0
    with _coil(w, precision=prec, format=fmt) as c:
        for _ in range(15):
            c.step(1, w.drive)
            I = c.currents().reshape(-1, n * n)
            peak = max(peak, np.max(np.abs(I)))
            net = max(net, max(np.max(np.abs(I[:, grp == g].sum(axis=1))) for g in range(grp.max() + 1)))
    assert peak > 0
    assert net <= 1e-10 * peak


def test_state_roundtrip_carries_the_transport_part():
    w = _grouped(75, 2, 3, 4)
    with _coil(w) as a, _coil(w) as b:
        a.step(20, w.drive)
        b.load_state(a.save_state())
        a.step(15, w.drive)
        b.step(15, w.drive)
        assert np.array_equal(a.currents(), b.currents())
        assert np.array_equal(a.diag()[-1], b.diag()[-1])


def test_subelement_refusals():
    from paper_2403_07666_b300.coil import CoilError, ERR_INVALID
    w = _grouped(76, 2, 3, 4)
    with _coil(w) as c:
        with pytest.raises(CoilError) as ei:
            c.adjoint(3, w.drive, np.ones(3))
        assert ei.value.status == ERR_INVALID
    w5 = wl.random_coil(77, 2, 3, 5)
    w5.geometry["groups"] = np.arange(25) % 17         # more than 16 subelements
    with pytest.raises(CoilError):
        _coil(w5)
    w7 = wl.random_coil(78, 2, 3, 4)
    w7.geometry["groups"] = np.arange(16) % 7          # more than 6 subelements of a 16-element turn
    with pytest.raises(CoilError):
        _coil(w7)
    we = wl.random_coil(79, 2, 3, 4)
    g = np.zeros(16, dtype=np.int32)
    g[0] = 2                                           # group 1 empty
    we.geometry["groups"] = g
    with pytest.raises(CoilError):
        _coil(we)
