"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

FP64 mode must match within 1e-5 relative (to the field's maximum) on J, B
and T per step; mixed precision within the bounds stated per result.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2403_07666_b300 import build as B
from paper_2403_07666_b300 import workloads as wl
from tests.gpu_common import rel, oracle_of, compare_state

pytestmark = pytest.mark.gpu

TOL64 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def Coil(*a, **k):
    from paper_2403_07666_b300.coil import Coil as _C
    return _C(*a, **k)


def _coil(w, **kw):
    from paper_2403_07666_b300.coil import Coil as _C
    return _C.from_workload(w, **kw)


# ----------------------------------------------------------------- operator

@pytest.mark.parametrize("L,T,n", [(5, 7, 4), (3, 5, 6), (2, 3, 8), (1, 1, 1)])
def test_operator_fp64_matches_oracle(L, T, n):
    w = wl.random_coil(11, L, T, n)
    with _coil(w) as c:
        Mg = c.operator()
    Mo = oracle_of(w).M
    assert np.array_equal(Mg, Mg.T)                       # bitwise symmetric assembly
    assert np.max(np.abs(Mg - Mo) / np.abs(Mo)) < 1e-11   # entrywise, all entries positive


@pytest.mark.parametrize("prec,bound", [("fp32", 1.2e-7), ("bf16", 8e-3)])
def test_operator_storage_rounding(prec, bound):
    w = wl.random_coil(12, 4, 6, 4)
    with _coil(w, precision=prec) as c:
        Mg = c.operator()
    Mo = oracle_of(w).M
    assert np.array_equal(Mg, Mg.T)
    assert np.max(np.abs(Mg - Mo) / np.abs(Mo)) < bound


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-7), ("bf16", 5e-3)])
def test_apply_operator(prec, tol):
    w = wl.random_coil(13, 5, 7, 4)                       # 560 rows: 17.5 row tiles
    rng = np.random.default_rng(3)
    p = rng.standard_normal(w.n_elem)
    with _coil(w, precision=prec) as c:
        y = c.apply_operator(p)
    Mo = oracle_of(w).M
    assert rel(y, Mo @ p) < tol


# ------------------------------------------------------------- time steps

def _march(w, steps, tol=TOL64, every=1, precision="fp64", rtol=1e-11, cols=8):
    orc = oracle_of(w)
    worst = np.zeros(4)
    with _coil(w, precision=precision, rtol=rtol) as c:
        for k in range(steps):
            c.step(1, w.drive)
            orc.step(w.drive)
            if (k + 1) % every == 0 or k == steps - 1:
                e = compare_state(c.read(w.drive), orc, w.drive, w.material["T_bath"], tol, tol, tol)
                worst = np.maximum(worst, e)
        dg = c.diag()
    do = np.array(orc.diag)
    assert dg.shape[0] == steps
    for j in range(cols):
        scale = np.max(np.abs(do[:, j]))
        if np.isfinite(scale) and scale > 0:
            assert np.max(np.abs(dg[:, j] - do[:, j])) <= tol * scale, (j, dg[:, j][:5], do[:, j][:5])
    return worst


@pytest.mark.parametrize("L,T,n,seed", [(5, 7, 4, 21), (3, 5, 6, 22), (2, 3, 8, 23)])
def test_steps_fp64_nonlinear_regime(L, T, n, seed):
    """Ramp past the critical current with heating: flux flow, Jc(T) feedback."""
    mtl = dict(wl.MATERIAL, Jc0=2e8)
    w = wl.random_coil(seed, L, T, n, ramp_rate=5e4, material=mtl)
    worst = _march(w, 160, every=10)
    assert worst[0] < TOL64


def test_small_coil_full_run():
    """4 x 8 turns, 4 x 4 elements (512), 10 A/s, dt 1e-5 s, 2000 steps."""
    w = wl.small_coil()
    _march(w, 2000, every=250)


def test_applied_field_loop_free_loops():
    """Free loops (no transport) under a triangular applied field."""
    mtl = dict(wl.MATERIAL, Jc0=2e8)
    w = wl.random_coil(31, 3, 4, 4, ramp_rate=0.0, I_max=0.0, material=mtl, dt=1e-4,
                       Ba_rate=40.0, Ba_max=0.02, Ba_waveform=2)
    w.geometry["transport"] = 0
    _march(w, 60, every=10)


def test_list_geometry_two_and_four_loops():
    p = dict(wl.MATERIAL, thermal=0, jc_model=1, Jc0=2e8)
    geom = {"kind": "list", "r": np.array([0.020, 0.0205, 0.020, 0.0205]),
            "z": np.array([0.0, 0.0, 0.0008, 0.0008]), "h": np.full(4, 4e-4), "block": 2,
            "block_transport": np.array([1, 1])}
    mat = np.array([1, 0, 1, 0])
    drive = {"dt": 1e-5, "ramp_rate": 3e5, "I_max": 1e9, "Ba_rate": 0.0, "Ba_max": 0.0, "Ba_waveform": 0}
    orc = oracle.build(geom, p, np.ones(4), np.zeros(4), mat, np.array([True, True]))
    with Coil(geom, p, np.ones(4), np.zeros(4), mat) as c:
        for _ in range(60):
            c.step(1, drive)
            orc.step(drive)
        I = c.currents()
        dg = c.diag()
    assert rel(I, orc.I) < 1e-9
    assert rel(dg[:, 2], np.array(orc.diag)[:, 2]) < 1e-9         # V_term


def test_thermal_relaxation_single_element():
    """n = 1 element with four bath faces: exponential decay, lambda ~ 37.9 1/s."""
    geom = {"kind": "solenoid", "n_layers": 1, "n_turns": 1, "n_sub": 1, "r_in": 0.02,
            "pitch": 0.9e-3, "wire_d": 0.8e-3, "transport": 0}
    p = dict(wl.MATERIAL, jc_model=1)
    drive = {"dt": 1e-5, "ramp_rate": 0.0, "I_max": 0.0}
    with Coil(geom, p, np.ones(1), np.zeros(1), np.zeros(1, np.int32)) as c:
        st = c.save_state()
        # raise T to 6 K through the state buffer (T^4 sits after I, flux, Idot
        # and the two steps' Idot before it)
        hdr = 8 + 8 * 4 + 8
        u = np.frombuffer(st[hdr + 40:hdr + 48].tobytes(), dtype=np.float64)
        assert abs(u[0] - 4.2 ** 4) < 1e-9
        st[hdr + 40:hdr + 48] = np.frombuffer(np.array([6.0 ** 4]).tobytes(), dtype=np.uint8)
        c.load_state(st)
        c.step(2000, drive)
        T = c.read(drive)["T"][0]
    lam = 4 * 500.0 / (8900 * 0.1 * 0.8e-3 * 4.2 ** 3)
    exact = 4.2 + 1.8 * math.exp(-lam * 0.02)
    assert abs(T - exact) / 1.8 < 2 * lam * 1e-5


# ------------------------------------------------------- mixed precision

# FP32 storage keeps every result within 1e-5 of the FP64 oracle.  BF16 storage
# (2^-9 per entry) is an experimental mode: the rounding perturbs the
# differences of neighbouring entries that drive the current distribution
# inside a wire, so J is off by several percent; these bounds only guard it
# against regressions (measured: J <= 0.11, B <= 0.07, m <= 3.3e-4).
@pytest.mark.parametrize("prec,tJ,tB,tT,tm", [("fp32", 1e-5, 1e-5, 1e-5, 1e-7),
                                              ("bf16", 0.15, 0.1, 0.05, 5e-4)])
def test_mixed_precision_bounds(prec, tJ, tB, tT, tm):
    mtl = dict(wl.MATERIAL, Jc0=2e8)
    w = wl.random_coil(41, 5, 7, 4, ramp_rate=5e4, material=mtl)
    orc = oracle_of(w)
    with _coil(w, precision=prec, rtol=1e-9) as c:
        for k in range(8):
            c.step(20, w.drive)
            for _ in range(20):
                orc.step(w.drive)
            e = compare_state(c.read(w.drive), orc, w.drive, w.material["T_bath"], tJ, tB, tT)
            assert e[3] < tm, ("moment", e[3])


# ------------------------------------------------------ state and errors

def test_state_roundtrip_continues_identically():
    w = wl.random_coil(51, 3, 4, 4, ramp_rate=1e4)
    with _coil(w) as a, _coil(w) as b:
        a.step(30, w.drive)
        b.load_state(a.save_state())
        a.step(20, w.drive)
        b.step(20, w.drive)
        assert np.array_equal(a.currents(), b.currents())
        assert np.array_equal(a.read(w.drive)["T"], b.read(w.drive)["T"])


def test_iteration_cap_reports_not_converged():
    from paper_2403_07666_b300.coil import CoilError, ERR_NOT_CONVERGED
    w = wl.random_coil(52, 4, 5, 4, ramp_rate=1e4)
    with _coil(w, maxit=1, rtol=1e-14) as c:
        with pytest.raises(CoilError) as ei:
            c.step(3, w.drive)
        assert ei.value.status == ERR_NOT_CONVERGED
        assert c.info().steps == 0                 # state left at the last completed step


def test_nonfinite_input_rejected():
    from paper_2403_07666_b300.coil import CoilError, ERR_NONFINITE
    w = wl.random_coil(53, 2, 2, 4)
    w.jc_factor[5] = float("nan")
    with pytest.raises(CoilError) as ei:
        _coil(w)
    assert ei.value.status == ERR_NONFINITE


def test_huge_request_reports_oom():
    from paper_2403_07666_b300.coil import CoilError, ERR_OOM
    # 300 x 300 turns of 4 x 4 elements: 1.44 M elements, a 16.6 TB FP64 operator
    w = wl.solenoid("huge", 300, 300, 4, 1, steps=1)
    with pytest.raises(CoilError) as ei:
        _coil(w)
    assert ei.value.status == ERR_OOM
