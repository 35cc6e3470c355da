"""Shared helpers of the GPU parity tests (library vs oracle on the same inputs)."""
import numpy as np

import oracle


def rel(a, b):
    """max |a - b| / max |b| (absolute when b is identically zero)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.max(np.abs(b)) if b.size else 0.0
    err = np.max(np.abs(a - b)) if b.size else 0.0
    return err / scale if scale > 0 else err


def oracle_of(w, constrained=None):
    return oracle.build(w.geometry, w.material, w.jc_factor, w.strain, w.mat, constrained)


def compare_state(gpu_out, orc, drive, T_bath, tol_J, tol_B, tol_T):
    ref = orc.read(drive)
    eJ = rel(gpu_out["J"], ref["J"])
    eB = max(rel(gpu_out["Br"], ref["Br"]), rel(gpu_out["Bz"], ref["Bz"]))
    # temperature: relative to the heating, with a floor of 1e-6 T_bath so that a
    # rise far below the FP64 resolution of T itself is not compared bit by bit
    dT_ref = np.max(np.abs(ref["T"] - T_bath))
    eT = np.max(np.abs(gpu_out["T"] - ref["T"])) / max(dT_ref, 1e-6 * T_bath)
    em = abs(gpu_out["moment"] - ref["moment"]) / max(abs(ref["moment"]), 1e-300)
    assert eJ <= tol_J, ("J", eJ)
    assert eB <= tol_B, ("B", eB)
    assert eT <= tol_T, ("T", eT)
    return eJ, eB, eT, em
