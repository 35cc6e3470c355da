"""Block-Toeplitz storage of the far operator (regular solenoids): the same
FP32 entries as the dense form applied as a Toeplitz-structured CUDA-core
product ("toeplitz"), and the FP16 hi/lo split of the entries applied on the
tensor cores ("toeplitz_tc")."""
import numpy as np
import pytest

from paper_2403_07666_b300 import build as B
from paper_2403_07666_b300 import workloads as wl
from tests.gpu_common import rel, oracle_of, compare_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _coil(w, **kw):
    from paper_2403_07666_b300.coil import Coil
    return Coil.from_workload(w, **kw)


# C = 80, 108, 128, 16 channels per turn row: ragged channel tiles and k chunks;
# 7, 5, 3, 40 turns: one or more row tiles with shifted rows falling outside.
SHAPES = [(5, 7, 4), (3, 5, 6), (2, 3, 8), (1, 40, 4)]
FORMATS = ["toeplitz", "toeplitz_tc"]


@pytest.mark.parametrize("L,T,n", SHAPES)
def test_toeplitz_entries_equal_dense_fp32(L, T, n):
    w = wl.random_coil(91, L, T, n)
    with _coil(w, precision="fp32") as d, _coil(w, precision="fp32", format="toeplitz") as t:
        assert np.array_equal(t.operator(), d.operator())
        assert t.info().operator_bytes < d.info().operator_bytes or w.geometry["n_turns"] < 3


@pytest.mark.parametrize("L,T,n", SHAPES)
def test_tc_entries_match_oracle(L, T, n):
    """hi + lo of the FP16 split carries ~22 bits: entries within FP32 rounding."""
    w = wl.random_coil(91, L, T, n)
    M = oracle_of(w).M
    with _coil(w, precision="fp32", format="toeplitz_tc") as t:
        Mt = t.operator()
        C = L * n * n
        assert t.info().operator_bytes == 4 * T * C * ((C + 63) // 64 * 64)      # offsets >= 0 only
    err = np.abs(Mt - M)
    assert np.max(err / np.abs(M).max()) < 2.0 ** -22
    assert rel(Mt, M) < 2e-7


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("L,T,n", SHAPES)
def test_toeplitz_apply_matches_oracle(L, T, n, fmt):
    w = wl.random_coil(92, L, T, n)
    rng = np.random.default_rng(4)
    p = rng.standard_normal(w.n_elem)
    with _coil(w, precision="fp32", format=fmt) as t:
        y = t.apply_operator(p)
        y2 = t.apply_operator(p)
    assert rel(y, oracle_of(w).M @ p) < 2e-6
    assert np.array_equal(y, y2)                          # fixed-order sums: deterministic


# tensor-core edge shapes: C = 147 (two channel tiles, the second ragged, C not a
# multiple of 8), one turn (only offset 0), 112 turns (the largest staged copy of p),
# a single-element wire, inputs spanning 30 decades and an input of zeros
@pytest.mark.parametrize("L,T,n", [(3, 4, 7), (4, 1, 4), (1, 112, 2), (9, 6, 1)])
def test_tc_edge_shapes(L, T, n):
    w = wl.random_coil(98, L, T, n)
    rng = np.random.default_rng(6)
    M = oracle_of(w).M
    with _coil(w, precision="fp32", format="toeplitz_tc") as t:
        for p in (rng.standard_normal(w.n_elem),
                  rng.standard_normal(w.n_elem) * 10.0 ** rng.uniform(-15, 15, w.n_elem),
                  np.zeros(w.n_elem)):
            y = t.apply_operator(p)
            ref = M @ p
            if not p.any():
                assert not y.any()
                continue
            # per element: error within FP32-class rounding of the largest term
            bound = 4e-6 * (np.abs(M) @ np.abs(p)) + 1e-300
            assert np.all(np.abs(y - ref) <= bound)


def test_tc_rejects_unsupported():
    from paper_2403_07666_b300.coil import CoilError, ERR_INVALID
    for w, prec in ((wl.random_coil(97, 1, 113, 2), "fp32"), (wl.random_coil(97, 2, 3, 4), "fp64"),
                    (wl.random_coil(97, 2, 3, 4), "bf16")):
        with pytest.raises(CoilError) as ei:
            _coil(w, precision=prec, format="toeplitz_tc")
        assert ei.value.status == ERR_INVALID


@pytest.mark.parametrize("fmt", FORMATS)
def test_toeplitz_steps_match_oracle_and_dense(fmt):
    mtl = dict(wl.MATERIAL, Jc0=2e8)
    w = wl.random_coil(93, 5, 7, 4, ramp_rate=5e4, material=mtl)
    orc = oracle_of(w)
    with _coil(w, precision="fp32", format=fmt, rtol=1e-9) as t, \
            _coil(w, precision="fp32", rtol=1e-9) as d:
        for k in range(6):
            t.step(20, w.drive)
            d.step(20, w.drive)
            for _ in range(20):
                orc.step(w.drive)
            compare_state(t.read(w.drive), orc, w.drive, w.material["T_bath"], 1e-5, 1e-5, 1e-5)
        assert rel(t.currents(), d.currents()) < 1e-5        # both within 1e-5 of the oracle


@pytest.mark.parametrize("fmt", FORMATS)
def test_toeplitz_batch_equals_single(fmt):
    from paper_2403_07666_b300.coil import batch_step
    mtl = dict(wl.MATERIAL, Jc0=2e8)
    ws = [wl.random_coil(94, 3, 4, 4, ramp_rate=4e4, material=mtl),
          wl.random_coil(95, 5, 9, 6, ramp_rate=1e4, material=mtl),
          wl.random_coil(96, 2, 40, 4, ramp_rate=2e4, material=mtl)]
    batch = [_coil(w, precision="fp32", format=fmt, rtol=1e-10) for w in ws]
    alone = [_coil(w, precision="fp32", format=fmt, rtol=1e-10) for w in ws]
    if fmt == "toeplitz_tc":
        # batched applies take the two-fill schedule with its step floor (they run
        # side by side); alone with the same schedule a coil gets the same bits
        for c in alone:
            c.set_tc_schedule(0)
    try:
        batch_step(batch, 30, [w.drive for w in ws])
        for c, w in zip(alone, ws):
            c.step(30, w.drive)
        for b, a in zip(batch, alone):
            assert np.array_equal(b.currents(), a.currents())
    finally:
        for c in batch + alone:
            c.close()


def test_toeplitz_rejects_lists_and_other_precisions():
    from paper_2403_07666_b300.coil import CoilError, ERR_INVALID
    w = wl.random_coil(97, 2, 3, 4)
    with pytest.raises(CoilError) as ei:
        _coil(w, precision="fp64", format="toeplitz")
    assert ei.value.status == ERR_INVALID
