"""Pins of the tangent-linear oracle (complex-step forward-mode derivatives
of the oracle's step series with respect to the calibration parameters)."""
import numpy as np
import pytest

import oracle
from oracle.tangent import directional_derivatives
from paper_2403_07666_b300 import workloads as wl

K = 20


def _coil(thermal=1, transport=0, Y_eff=0.0):
    mtl = dict(wl.MATERIAL, Jc0=2e8, thermal=thermal, Y_eff=Y_eff)
    w = wl.random_coil(81, 3, 4, 4, ramp_rate=2e4 if transport else 0.0, I_max=1e9, dt=1e-4,
                       Ba_rate=4.0, Ba_max=0.02, Ba_waveform=2, material=mtl)
    w.geometry["transport"] = transport
    return w


def _series(w, f=None, n=None, ce=None):
    o = oracle.build(w.geometry, w.material, w.jc_factor if f is None else f, w.strain, w.mat)
    if n is not None:
        o.p["n"] = n
    if ce is not None:
        o.p["C_eps"] = ce
    recs = [o.step(w.drive) for _ in range(K)]
    return np.array([r[3] for r in recs]), np.array([r[4] for r in recs])


def _check(got, fd):
    """The derivatives grow by orders of magnitude over the window; central
    differences resolve them only well above their noise floor (the oracle's
    solve rounding over 2h).  The last step (the largest derivative) to 1e-4,
    every step within a tenth of it to 1e-3."""
    assert abs(got[-1] - fd[-1]) <= 1e-4 * abs(fd[-1]), (got[-1], fd[-1])
    keep = np.abs(fd) > 0.1 * np.max(np.abs(fd))
    err = np.max(np.abs(got[keep] - fd[keep]) / np.abs(fd[keep]))
    assert err < 1e-3, err


@pytest.mark.parametrize("thermal,transport,Y_eff", [(1, 0, 0.0), (0, 1, 0.0), (1, 1, 5e7)])
def test_tangent_matches_oracle_central_differences(thermal, transport, Y_eff):
    w = _coil(thermal, transport, Y_eff)
    m0, P0 = _series(w)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(w.n_elem)
    cases = [({"v_n": 1.0}, lambda s: _series(w, n=w.material["n"] + s)),
             ({"v_C": 1.0}, lambda s: _series(w, ce=w.material["C_eps"] + s)),
             ({"v_f": v * w.jc_factor}, lambda s: _series(w, f=w.jc_factor * (1 + s * v)))]
    scales = [w.material["n"], w.material["C_eps"], 1.0]
    for (kw, run), sc in zip(cases, scales):
        m, P, dm, dP = directional_derivatives(w, K, **kw)
        assert np.max(np.abs(m - m0)) <= 1e-12 * np.max(np.abs(m0))     # the same step series
        assert np.max(np.abs(P - P0)) <= 1e-12 * np.max(np.abs(P0))
        h = 1e-4 * sc
        mp, Pp = run(h)
        mm, Pm = run(-h)
        _check(dm, (mp - mm) / (2 * h))
        _check(dP, (Pp - Pm) / (2 * h))


def test_tangent_of_an_ohmic_coil_is_zero():
    """All-Cu elements: the E-J law is ohmic, nothing depends on f, n or C_eps."""
    w = _coil(1, 1)
    w.mat = np.zeros_like(w.mat)
    m, P, dm, dP = directional_derivatives(w, 8, v_f=np.ones(w.n_elem), v_n=1.0, v_C=1.0)
    assert np.max(np.abs(m)) > 0 and np.max(np.abs(P)) > 0
    assert np.all(dm == 0.0) and np.all(dP == 0.0)
