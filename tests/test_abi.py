"""CPU checks of the C-ABI library: it builds, loads, exports every symbol
that include/coil.h declares, and rejects invalid input before touching a GPU."""
import ctypes as C
import subprocess

import numpy as np
import pytest

from paper_2403_07666_b300 import build as B
from paper_2403_07666_b300 import coil as K
from paper_2403_07666_b300.workloads import MATERIAL


@pytest.fixture(scope="module")
def lib():
    B.build()
    return K.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = K.header_symbols()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert getattr(lib, n) is not None


def _material(N):
    m = K.Material()
    for k in ("E0", "n", "Jc0", "Tc", "Bc2_0", "B_reg", "C_eps", "p_eps", "rho_n", "rho_m", "c0",
              "kappa_cu", "kappa_ep", "h0", "T_ref", "T_bath"):
        setattr(m, k, float(MATERIAL[k]))
    m.jc_model, m.thermal = 0, 1
    arrs = [np.ones(N), np.zeros(N), np.ones(N, np.int32)]
    m.jc_factor, m.strain = K._ptr(arrs[0]), K._ptr(arrs[1])
    m.mat = K._ptr(arrs[2], C.c_int)
    return m, arrs


@pytest.mark.parametrize("bad", ["n_sub", "pitch", "kind", "precision", "rtol", "nan", "young", "groups_many",
                                 "groups_empty", "groups_range"])
def test_invalid_input_rejected_on_host(lib, bad):
    g = K.Geometry()
    g.kind = K.GEOM_SOLENOID
    g.n_layers, g.n_turns, g.n_sub = 2, 2, 2
    g.r_in, g.pitch, g.wire_d, g.transport = 0.02, 0.9e-3, 0.8e-3, 1
    m, keep = _material(16)
    o = K.Options(K.PREC_FP64, 1e-10, 100, 0, None, 64)
    expect = K.ERR_INVALID
    if bad == "n_sub":
        g.n_sub = 9                      # 81 elements per wire > 64
    elif bad == "pitch":
        g.pitch = 0.5e-3                 # wires overlap
    elif bad == "kind":
        g.kind = 7
    elif bad == "precision":
        o.precision = 5
    elif bad == "rtol":
        o.rtol = 0.0
    elif bad == "nan":
        m.T_bath = float("nan")
        expect = K.ERR_NONFINITE
    elif bad == "young":
        m.Y_eff = -1.0                   # Lorentz strain needs Y_eff >= 0
    elif bad.startswith("groups"):
        # subelements of the 4-element turns: more than 6 groups, an empty group,
        # an id outside [0, n_groups)
        grp, n_groups = {"groups_many": (np.arange(4, dtype=np.int32), 7),
                         "groups_empty": (np.array([0, 0, 2, 2], dtype=np.int32), 3),
                         "groups_range": (np.array([0, 1, 5, 1], dtype=np.int32), 3)}[bad]
        keep.append(grp)
        g.group = K._ptr(grp, C.c_int)
        g.n_groups = n_groups
    h = C.c_void_p()
    st = lib.coil_create(C.byref(g), C.byref(m), C.byref(o), C.byref(h))
    assert st == expect and not h.value


def test_null_handle_calls_are_safe(lib):
    assert lib.coil_step(None, 1, None) == K.ERR_INVALID
    assert lib.coil_last_error(None) == b"null coil handle"
    lib.coil_destroy(None)
