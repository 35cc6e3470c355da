"""Batched stepping of coils of uneven size: every kernel launched once for
the whole batch must give each coil exactly what stepping it alone gives,
and that must match the oracle."""
import numpy as np
import pytest

from paper_2403_07666_b300 import build as B
from paper_2403_07666_b300 import workloads as wl
from tests.gpu_common import oracle_of, compare_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _coils():
    mtl_a = dict(wl.MATERIAL, Jc0=2e8)
    mtl_b = dict(wl.MATERIAL, Jc0=3e8, T_bath=3.1)
    return [wl.random_coil(61, 3, 4, 4, ramp_rate=4e4, material=mtl_a),
            wl.random_coil(62, 5, 7, 4, ramp_rate=1e4, material=mtl_b),
            wl.random_coil(63, 2, 3, 6, ramp_rate=6e4, material=mtl_a),
            wl.random_coil(64, 1, 2, 8, ramp_rate=2e4, material=mtl_b)]


def test_batch_equals_single_coil_runs_bitwise():
    from paper_2403_07666_b300.coil import Coil, batch_step
    ws = _coils()
    batch = [Coil.from_workload(w, rtol=1e-11) for w in ws]
    alone = [Coil.from_workload(w, rtol=1e-11) for w in ws]
    try:
        for _ in range(3):
            batch_step(batch, 15, [w.drive for w in ws])
        for c, w in zip(alone, ws):
            c.step(45, w.drive)
        for b, a, w in zip(batch, alone, ws):
            assert b.info().steps == 45
            assert np.array_equal(b.currents(), a.currents())
            ra, rb = a.read(w.drive), b.read(w.drive)
            assert np.array_equal(ra["T"], rb["T"]) and np.array_equal(ra["Bz"], rb["Bz"])
            assert np.array_equal(b.diag(), a.diag())
    finally:
        for c in batch + alone:
            c.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_matches_oracle(precision):
    from paper_2403_07666_b300.coil import Coil, batch_step
    ws = _coils()
    orcs = [oracle_of(w) for w in ws]
    cs = [Coil.from_workload(w, precision=precision, rtol=1e-11 if precision == "fp64" else 1e-9)
          for w in ws]
    tol = 1e-5
    try:
        for k in range(4):
            batch_step(cs, 20, [w.drive for w in ws])
            for o, w in zip(orcs, ws):
                for _ in range(20):
                    o.step(w.drive)
            for c, o, w in zip(cs, orcs, ws):
                compare_state(c.read(w.drive), o, w.drive, w.material["T_bath"], tol, tol, tol)
    finally:
        for c in cs:
            c.close()


def test_batch_rejects_mixed_precision():
    from paper_2403_07666_b300.coil import Coil, CoilError, batch_step, ERR_INVALID
    ws = _coils()[:2]
    a = Coil.from_workload(ws[0], precision="fp64")
    b = Coil.from_workload(ws[1], precision="fp32")
    try:
        with pytest.raises(CoilError) as ei:
            batch_step([a, b], 1, [ws[0].drive, ws[1].drive])
        assert ei.value.status == ERR_INVALID
        assert a.info().steps == 0 and b.info().steps == 0
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("fmt,prec", [("dense", "fp64"), ("toeplitz_tc", "fp32")])
def test_batch_graph_follows_the_coil_set(fmt, prec):
    """A batched step runs as a graph kept by the batch's first coil: a call
    with another set of coils behind the same first coil, or with a coil
    replaced by a new one, must rebuild it; every coil still gets exactly what
    stepping it alone gives."""
    from paper_2403_07666_b300.coil import Coil, batch_step
    ws = _coils()[:3]
    kw = dict(precision=prec, format=fmt, rtol=1e-11)
    a, b, c = (Coil.from_workload(w, **kw) for w in ws)
    alone = [Coil.from_workload(w, **kw) for w in ws]
    if fmt == "toeplitz_tc":
        # batched applies take the two-fill schedule with its step floor; alone
        # with the same schedule a coil gets the same bits
        for x in alone:
            x.set_tc_schedule(0)
    d = None
    try:
        batch_step([a, b], 4, [ws[0].drive, ws[1].drive])
        batch_step([a, c], 4, [ws[0].drive, ws[2].drive])
        batch_step([a, b, c], 4, [w.drive for w in ws])
        b.close()
        d = Coil.from_workload(ws[1], **kw)             # a new coil, possibly at the old one's address
        batch_step([a, d], 4, [ws[0].drive, ws[1].drive])
        alone[0].step(16, ws[0].drive)
        alone[1].step(4, ws[1].drive)
        alone[2].step(8, ws[2].drive)
        assert np.array_equal(a.currents(), alone[0].currents())
        assert np.array_equal(c.currents(), alone[2].currents())
        assert np.array_equal(d.currents(), alone[1].currents())
        assert a.info().steps == 16 and c.info().steps == 8 and d.info().steps == 4
    finally:
        for x in (a, c, d, *alone):
            if x is not None:
                x.close()
