"""Graph-launched steps and adjoint solves against the same kernels launched
one by one (profile mode).  A graph-launched step is one CUDA graph: the
prologue, a while node over PCG iterations whose condition the device sets
(the last CTA of the shared-warp update kernel, or k_loop_cond for wires of
more than 16 elements), and the epilogue.  The graph changes how the kernels
are launched, not their arithmetic or its order, so the results agree bit for
bit: currents, diagnostics (iteration counts and residuals included), onsets
and adjoint gradients."""
import numpy as np
import pytest

from paper_2403_07666_b300 import build as B
from paper_2403_07666_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _coil(w, **kw):
    from paper_2403_07666_b300.coil import Coil
    return Coil.from_workload(w, **kw)


# n_sub 4 and 3: wires of 16 and 9 elements (shared-warp kernels); n_sub 5:
# 25-element wires (one warp per wire)
CASES = [("toeplitz_tc", "fp32", 4), ("toeplitz", "fp32", 3), ("dense", "fp64", 4), ("dense", "fp64", 5)]


@pytest.mark.parametrize("fmt,prec,n", CASES)
def test_graph_steps_match_one_by_one_launches(fmt, prec, n):
    w = wl.random_coil(91, 3, 4, n, material=dict(wl.MATERIAL, Jc0=2e7), ramp_rate=5e5)
    with _coil(w, precision=prec, format=fmt) as g, _coil(w, precision=prec, format=fmt, profile=True) as p:
        for _ in range(3):
            g.step(4, w.drive)
            p.step(4, w.drive)
            assert np.array_equal(g.currents(), p.currents())
        assert g.info().step_graph == 1
        assert p.info().step_graph == 0
        assert np.array_equal(g.diag(), p.diag(), equal_nan=True)
        fg, qg = g.onsets()
        fp, qp = p.onsets()
        assert np.array_equal(fg, fp) and np.array_equal(qg, qp)
        assert g.info().pcg_iterations == p.info().pcg_iterations > 0


def test_graph_adjoint_matches_one_by_one_launches():
    mtl = dict(wl.MATERIAL, Jc0=2e8)
    w = wl.random_coil(92, 3, 4, 4, ramp_rate=0.0, I_max=1e9, dt=1e-4, Ba_rate=4.0, Ba_max=0.02, Ba_waveform=2,
                       material=mtl)
    w.geometry["transport"] = 0
    K = 20
    dm = np.linspace(-1.0, 1.0, K)
    out = []
    for profile in (False, True):
        with _coil(w, rtol=1e-11, profile=profile) as c:
            s0 = c.save_state()
            c.step(K, w.drive)
            m = c.diag(0, K)[:, 3]
            c.load_state(s0)
            out.append((m, c.adjoint(K, w.drive, dm * np.max(np.abs(m)), ckpt_every=7)))
    (mg, (fg, ng, cg)), (mp, (fp, npr, cp)) = out
    assert np.array_equal(mg, mp)
    assert np.array_equal(fg, fp) and ng == npr and cg == cp
    assert np.any(fg != 0.0)
