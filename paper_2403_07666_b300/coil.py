"""Thin ctypes binding of the C ABI in include/coil.h (argument marshalling only).

Every step of the coupled update runs in the CUDA kernels of libcoil.so; this
module only converts Python/numpy arguments into the C structs and back.
There is no CPU fallback: if the shared library is missing the import fails.
"""

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcoil.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "coil.h")

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_NONFINITE = 0, -1, -2, -3, -4, -5
GEOM_SOLENOID, GEOM_LIST = 0, 1
PREC_FP64, PREC_FP32, PREC_BF16 = 0, 1, 2
PRECISIONS = {"fp64": PREC_FP64, "fp32": PREC_FP32, "bf16": PREC_BF16}
FORMAT_DENSE, FORMAT_TOEPLITZ, FORMAT_TOEPLITZ_TC = 0, 1, 2
FORMATS = {"dense": FORMAT_DENSE, "toeplitz": FORMAT_TOEPLITZ, "toeplitz_tc": FORMAT_TOEPLITZ_TC}
DIAG_WIDTH = 10
DIAG_FIELDS = ("t", "I_t", "V_term", "moment", "P_joule", "T_max", "max_jratio",
               "max_rho_frac", "pcg_iters", "resid")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class Geometry(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_layers", C.c_int), ("n_turns", C.c_int), ("n_sub", C.c_int),
                ("r_in", C.c_double), ("pitch", C.c_double), ("wire_d", C.c_double),
                ("transport", C.c_int), ("n_elem", C.c_int), ("block", C.c_int),
                ("r", _dp), ("z", _dp), ("h", _dp), ("block_transport", _ip),
                ("n_groups", C.c_int), ("group", _ip)]


class Material(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("E0", "n", "Jc0", "Tc", "Bc2_0", "B_reg", "C_eps", "p_eps",
                                          "rho_n", "rho_m", "c0", "kappa_cu", "kappa_ep", "h0",
                                          "T_ref", "T_bath")] + \
              [("jc_model", C.c_int), ("thermal", C.c_int), ("jc_factor", _dp), ("strain", _dp),
               ("mat", _ip), ("Y_eff", C.c_double)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("rtol", C.c_double), ("maxit", C.c_int), ("device", C.c_int),
                ("stream", C.c_void_p), ("diag_capacity", C.c_long), ("profile", C.c_int),
                ("format", C.c_int)]


class Drive(C.Structure):
    _fields_ = [("dt", C.c_double), ("ramp_rate", C.c_double), ("I_max", C.c_double),
                ("Ba_rate", C.c_double), ("Ba_max", C.c_double), ("Ba_waveform", C.c_int)]


class Info(C.Structure):
    _fields_ = [("n_elem", C.c_long), ("n_blocks", C.c_long), ("block", C.c_long), ("grid_r", C.c_long),
                ("grid_z", C.c_long), ("precision", C.c_int), ("operator_bytes", C.c_size_t),
                ("device_bytes", C.c_size_t), ("steps", C.c_long), ("t", C.c_double),
                ("setup_ms", C.c_double), ("kernel_launches", C.c_longlong),
                ("operator_launches", C.c_longlong), ("operator_ms", C.c_double),
                ("pcg_iterations", C.c_longlong), ("descriptor_bytes", C.c_size_t), ("step_graph", C.c_int)]


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libcoil.so not built ({path}); run python -m paper_2403_07666_b300.build")
    lib = C.CDLL(path)
    P = C.c_void_p
    sig = {
        "coil_create": ([C.POINTER(Geometry), C.POINTER(Material), C.POINTER(Options), C.POINTER(P)], C.c_int),
        "coil_step": ([P, C.c_long, C.POINTER(Drive)], C.c_int),
        "coil_batch_step": ([C.POINTER(P), C.c_int, C.c_long, C.POINTER(Drive)], C.c_int),
        "coil_read": ([P, C.POINTER(Drive), _dp, _dp, _dp, _dp, _dp], C.c_int),
        "coil_read_device": ([P, C.POINTER(Drive), P, P, P, P], C.c_int),
        "coil_read_diag": ([P, C.c_long, C.c_long, _dp], C.c_int),
        "coil_read_onsets": ([P, C.POINTER(C.c_long), C.POINTER(C.c_long)], C.c_int),
        "coil_read_wire_stats": ([P, C.POINTER(C.c_double)], C.c_int),
        "coil_reset_wire_stats": ([P], C.c_int),
        "coil_get_currents": ([P, _dp], C.c_int),
        "coil_set_currents": ([P, _dp], C.c_int),
        "coil_apply_operator": ([P, _dp, _dp], C.c_int),
        "coil_apply_operator_static": ([P, P, P, P], C.c_int),
        "coil_read_operator": ([P, _dp], C.c_int),
        "coil_save_state": ([P, P, C.POINTER(C.c_size_t)], C.c_int),
        "coil_load_state": ([P, P, C.c_size_t], C.c_int),
        "coil_set_params": ([P, _dp, C.c_double, C.c_double], C.c_int),
        "coil_adjoint": ([P, C.c_long, C.POINTER(Drive), C.c_int, _dp, _dp, _dp, _dp], C.c_int),
        "coil_adjoint_losses": ([P, C.c_long, C.POINTER(Drive), C.c_int, _dp, _dp, _dp, _dp, _dp], C.c_int),
        "coil_tc_schedule": ([P, _ip, _ip, _ip, _dp], C.c_int),
        "coil_tc_candidates": ([P, _ip, _dp], C.c_int),
        "coil_set_tc_schedule": ([P, C.c_int, C.c_int, C.c_int], C.c_int),
        "coil_info": ([P, C.POINTER(Info)], C.c_int),
        "coil_reset_counters": ([P], C.c_int),
        "coil_set_wait_limit": ([P, C.c_longlong], C.c_int),
        "coil_last_error": ([P], C.c_char_p),
        "coil_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


class CoilError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"coil status {status}: {msg}")
        self.status = status


def _ptr(a, ctype=C.c_double):
    return a.ctypes.data_as(C.POINTER(ctype))


def make_drive(d):
    return Drive(float(d["dt"]), float(d.get("ramp_rate", 0.0)), float(d.get("I_max", 0.0)),
                 float(d.get("Ba_rate", 0.0)), float(d.get("Ba_max", 0.0)), int(d.get("Ba_waveform", 0)))


class Coil:
    """One coil on the GPU behind the C ABI."""

    def __init__(self, geometry, material, jc_factor, strain, mat, precision="fp64", rtol=1e-10,
                 maxit=500, device=0, stream=None, diag_capacity=65536, block_transport=None,
                 profile=False, format="dense"):
        self._lib = lib()
        self._keep = []
        g = Geometry()
        if geometry["kind"] == "solenoid":
            g.kind = GEOM_SOLENOID
            g.n_layers, g.n_turns, g.n_sub = (int(geometry[k]) for k in ("n_layers", "n_turns", "n_sub"))
            g.r_in, g.pitch, g.wire_d = (float(geometry[k]) for k in ("r_in", "pitch", "wire_d"))
            g.transport = int(geometry.get("transport", 1))
        else:
            g.kind = GEOM_LIST
            r = np.ascontiguousarray(geometry["r"], dtype=np.float64)
            z = np.ascontiguousarray(geometry["z"], dtype=np.float64)
            h = np.ascontiguousarray(geometry["h"], dtype=np.float64)
            g.n_elem = r.size
            g.block = int(geometry["block"])
            bt = np.ascontiguousarray(block_transport if block_transport is not None
                                      else geometry.get("block_transport", np.ones(r.size // g.block)),
                                      dtype=np.int32)
            self._keep += [r, z, h, bt]
            g.r, g.z, g.h = _ptr(r), _ptr(z), _ptr(h)
            g.block_transport = _ptr(bt, C.c_int)
        if geometry.get("groups") is not None:
            gr = np.ascontiguousarray(geometry["groups"], dtype=np.int32)
            self._keep.append(gr)
            g.n_groups = int(gr.max()) + 1 if gr.size else 0
            g.group = _ptr(gr, C.c_int)
        m = Material()
        for k in ("E0", "n", "Jc0", "Tc", "Bc2_0", "B_reg", "C_eps", "p_eps", "rho_n", "rho_m", "c0",
                  "kappa_cu", "kappa_ep", "h0", "T_ref", "T_bath"):
            setattr(m, k, float(material[k]))
        m.jc_model = int(material["jc_model"])
        m.Y_eff = float(material.get("Y_eff", 0.0))
        m.thermal = int(material["thermal"])
        jf = np.ascontiguousarray(jc_factor, dtype=np.float64)
        st = np.ascontiguousarray(strain, dtype=np.float64)
        mt = np.ascontiguousarray(mat, dtype=np.int32)
        self._keep += [jf, st, mt]
        m.jc_factor, m.strain, m.mat = _ptr(jf), _ptr(st), _ptr(mt, C.c_int)
        o = Options(PRECISIONS[precision] if isinstance(precision, str) else int(precision), float(rtol),
                    int(maxit), int(device), stream, int(diag_capacity), int(bool(profile)),
                    FORMATS[format] if isinstance(format, str) else int(format))
        h = C.c_void_p()
        status = self._lib.coil_create(C.byref(g), C.byref(m), C.byref(o), C.byref(h))
        if status != OK:
            raise CoilError(status, "coil_create failed (see stderr)")
        self._h = h
        info = self.info()
        self.N = int(info.n_elem)
        self.W = int(info.n_blocks)

    @classmethod
    def from_workload(cls, w, **kw):
        return cls(w.geometry, w.material, w.jc_factor, w.strain, w.mat, **kw)

    # -- plumbing ----------------------------------------------------------------
    def _check(self, status):
        if status != OK:
            msg = self._lib.coil_last_error(self._h).decode()
            raise CoilError(status, msg)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.coil_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- API ---------------------------------------------------------------------
    def step(self, n_steps, drive):
        self._check(self._lib.coil_step(self._h, int(n_steps), C.byref(make_drive(drive))))

    def read(self, drive=None):
        N = self.N
        out = {k: np.empty(N) for k in ("J", "Br", "Bz", "T")}
        mom = C.c_double()
        dr = C.byref(make_drive(drive)) if drive is not None else None
        self._check(self._lib.coil_read(self._h, dr, _ptr(out["J"]), _ptr(out["Br"]), _ptr(out["Bz"]),
                                        _ptr(out["T"]), C.byref(mom)))
        out["moment"] = mom.value
        return out

    def read_into(self, drive, J, Br, Bz, T):
        """coil_read into caller-owned (e.g. pinned) float64 host arrays."""
        mom = C.c_double()
        dr = C.byref(make_drive(drive)) if drive is not None else None
        self._check(self._lib.coil_read(self._h, dr, _ptr(J), _ptr(Br), _ptr(Bz), _ptr(T), C.byref(mom)))
        return mom.value

    def read_device(self, drive, J, Br, Bz, T):
        """coil_read_device into caller-owned device buffers (raw pointers)."""
        dr = C.byref(make_drive(drive)) if drive is not None else None
        self._check(self._lib.coil_read_device(self._h, dr, J, Br, Bz, T))

    def diag(self, first=0, count=None):
        steps = self.info().steps
        if count is None:
            count = steps - first
        out = np.empty((count, DIAG_WIDTH))
        if count:
            self._check(self._lib.coil_read_diag(self._h, int(first), int(count), _ptr(out)))
        return out

    def onsets(self):
        a = np.empty(self.W, dtype=np.int64)
        b = np.empty(self.W, dtype=np.int64)
        self._check(self._lib.coil_read_onsets(self._h, _ptr(a, C.c_long), _ptr(b, C.c_long)))
        return a, b

    def wire_stats(self):
        """Rows Q_total, T_max, P_max, Q_at_jump, Q_at_rise, Q_at_quench,
        first_rise (as float) of each wire: an array of shape (7, W)."""
        out = np.empty((7, self.W))
        self._check(self._lib.coil_read_wire_stats(self._h, _ptr(out)))
        return out

    def reset_wire_stats(self):
        self._check(self._lib.coil_reset_wire_stats(self._h))

    def currents(self):
        I = np.empty(self.N)
        self._check(self._lib.coil_get_currents(self._h, _ptr(I)))
        return I

    def set_currents(self, I):
        I = np.ascontiguousarray(I, dtype=np.float64)
        self._check(self._lib.coil_set_currents(self._h, _ptr(I)))

    def apply_operator(self, p):
        p = np.ascontiguousarray(p, dtype=np.float64)
        y = np.empty(self.N)
        self._check(self._lib.coil_apply_operator(self._h, _ptr(p), _ptr(y)))
        return y

    def apply_operator_static(self, d_p, d_y, stream=None):
        """coil_apply_operator_static on raw device pointers (no allocation;
        asynchronous on `stream`, a cudaStream_t handle or None)."""
        self._check(self._lib.coil_apply_operator_static(self._h, C.c_void_p(d_p), C.c_void_p(d_y),
                                                         C.c_void_p(stream) if stream else None))

    def operator(self):
        M = np.empty((self.N, self.N))
        self._check(self._lib.coil_read_operator(self._h, _ptr(M)))
        return M

    def save_state(self):
        n = C.c_size_t()
        self._check(self._lib.coil_save_state(self._h, None, C.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        self._check(self._lib.coil_save_state(self._h, buf.ctypes.data_as(C.c_void_p), C.byref(n)))
        return buf

    def load_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(self._lib.coil_load_state(self._h, buf.ctypes.data_as(C.c_void_p), buf.size))

    def set_params(self, jc_factor=None, n=30.0, C_eps=900.0):
        jf = None if jc_factor is None else np.ascontiguousarray(jc_factor, dtype=np.float64)
        self._check(self._lib.coil_set_params(self._h, None if jf is None else _ptr(jf), float(n),
                                              float(C_eps)))

    def adjoint(self, n_steps, drive, dL_dm, ckpt_every=50):
        """Gradients (dL/d jc_factor [N], dL/dn, dL/dC_eps) of a loss whose
        derivative with respect to the moment after each step is dL_dm."""
        dm = np.ascontiguousarray(dL_dm, dtype=np.float64)
        gf = np.empty(self.N)
        gn = C.c_double()
        gc = C.c_double()
        self._check(self._lib.coil_adjoint(self._h, int(n_steps), C.byref(make_drive(drive)),
                                           int(ckpt_every), _ptr(dm), _ptr(gf), C.byref(gn), C.byref(gc)))
        return gf, gn.value, gc.value

    def adjoint_losses(self, n_steps, drive, dL_dm=None, dL_dP=None, ckpt_every=50):
        """coil_adjoint_losses: gradients of a loss on the moment series
        (dL_dm) and the Joule-power series (dL_dP, per step's start state)."""
        dm = None if dL_dm is None else np.ascontiguousarray(dL_dm, dtype=np.float64)
        dp = None if dL_dP is None else np.ascontiguousarray(dL_dP, dtype=np.float64)
        gf = np.empty(self.N)
        gn = C.c_double()
        gc = C.c_double()
        self._check(self._lib.coil_adjoint_losses(self._h, int(n_steps), C.byref(make_drive(drive)),
                                                  int(ckpt_every), None if dm is None else _ptr(dm),
                                                  None if dp is None else _ptr(dp), _ptr(gf), C.byref(gn),
                                                  C.byref(gc)))
        return gf, gn.value, gc.value

    def tc_schedule(self):
        """The tensor-core apply's schedule: dict(mode, n_cta, stages, us) and the
        autotuner's candidates as rows (mode, n_cta, stages, us)."""
        m, n, st = C.c_int(), C.c_int(), C.c_int()
        us = C.c_double()
        self._check(self._lib.coil_tc_schedule(self._h, C.byref(m), C.byref(n), C.byref(st), C.byref(us)))
        cnt = C.c_int(0)
        self._check(self._lib.coil_tc_candidates(self._h, C.byref(cnt), None))
        rows = np.empty((cnt.value, 4))
        if cnt.value:
            self._check(self._lib.coil_tc_candidates(self._h, C.byref(cnt), _ptr(rows)))
        return {"mode": m.value, "n_cta": n.value, "stages": st.value, "us": us.value,
                "candidates": rows.tolist()}

    def set_tc_schedule(self, mode, n_cta=0, stages=0):
        self._check(self._lib.coil_set_tc_schedule(self._h, int(mode), int(n_cta), int(stages)))

    def set_wait_limit(self, cycles):
        """coil_set_wait_limit: test hook of the tensor-core apply's bounded
        waits (0 = the default limit)."""
        self._check(self._lib.coil_set_wait_limit(self._h, int(cycles)))

    def reset_counters(self):
        self._check(self._lib.coil_reset_counters(self._h))

    def info(self):
        inf = Info()
        self._check(self._lib.coil_info(self._h, C.byref(inf)))
        return inf


def batch_step(coils, n_steps, drives):
    """coil_batch_step over several Coil objects (one drive dict per coil)."""
    n = len(coils)
    handles = (C.c_void_p * n)(*[c._h.value for c in coils])
    drv = (Drive * n)(*[make_drive(d) for d in drives])
    status = lib().coil_batch_step(handles, n, int(n_steps), drv)
    if status != OK:
        msgs = "; ".join(lib().coil_last_error(c._h).decode() for c in coils[:1])
        raise CoilError(status, msgs)


def header_symbols(path=HEADER):
    """Function names declared in include/coil.h."""
    import re
    txt = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:coil_status|void|const char \*)\s*(coil_\w+)\s*\(", txt, re.M)))
