"""Benchmark of the coupled electromagnetic-thermal coil step on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload real|mid|small] [--precision bf16|fp32|fp64]

One step = one full pass of the hot path over every element of the coil:
pointwise E-J/Jc/Joule, per-wire factorisation, the projected PCG solve of
the transport-constrained circuit equations (dense operator applies), flux
and current update, ADI heat step, diagnostics.  Metric: element-steps/s.

Default workload: the 96,000-element real-size coil (60 x 100 turns, 4 x 4
elements per wire), transport ramp 2 A/s, dt = 1e-5 s, synthetic seeded
inputs.  Main leg: the far operator in the tensor-core block-Toeplitz form
(offsets >= 0 of the C x C turn-offset blocks, each FP32-class entry stored
as an FP16 hi + lo pair: 0.37 GB, larger than the 126 MB L2, so no flush is
needed between steps), applied with tcgen05 MMAs fed by TMA; its roofline is
HBM (the table streamed once per apply).  Beside it: the FP32 block-Toeplitz
form on CUDA cores (bound by the FP32 pipe), the dense FP32 storage (36.9 GB,
HBM-bound), the plain FP64 dense form (the mixed/FP64 ratio: storage format
and precision change together), the adjoint/forward cost on the 4,608-element
field-loop coil and the 64-coil batch.  BF16 storage (--precision bf16)
rounds the operator by 2^-9 per entry, which at this size is more than its
smallest eigenvalue: the stored operator is no longer positive definite and
the conjugate-gradient solve breaks down, so FP32-class storage is the mixed
form here.

Multi-GPU: the coil does not shard across GPUs in this build ("replicas
only"): under torchrun each rank steps its own replica; value = all ranks'
element-steps / max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2403_07666_b300 import workloads as wl  # noqa: E402
from paper_2403_07666_b300.replicas import job_throughput, shard_coils  # noqa: E402

METRIC = "element-steps/s (EM+thermal)"
UNIT = "element-steps/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# DRAM traffic per launch of the dominant kernel from one ncu capture
# (profiles/k_gemv_f32_profile19968.md: dram__bytes_read.sum +
# dram__bytes_write.sum on the 19,968-element coil).  The kernel streams the
# operator once, so traffic scales with the operator bytes; it is scaled to
# the bench launch by that ratio.  Kernels without a capture report null.
PROFILED_TRAFFIC = {
    "fp32": {"dram_bytes": 1.595007e9 + 3.258624e6, "operator_bytes": 1594884096},
    # profiles/k_toeplitz_f32_real96k.md: the bench workload itself (table 0.73 GB)
    "toeplitz": {"dram_bytes": 1.556434e9 + 14.971904e6, "operator_bytes": 733593600},
    # profiles/k_toeplitz_tc_real96k.md: the bench workload itself (split table 0.37 GB)
    "toeplitz_tc": {"dram_bytes": 459.704832e6 + 3.323904e6, "operator_bytes": 368640000},
}


def pick_workload(name):
    return {"real": wl.real_coil, "mid": wl.mid_coil, "small": wl.small_coil,
            "prof": wl.profile_coil}[name]()


# ------------------------------------------------------------------ clocks

class _Nvml:
    """Read-only NVML queries through ctypes (the driver's libnvidia-ml): SM
    clock, its maximum and the clock-event reason bits of the CUDA device."""

    def __init__(self, gpu):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.lib, self.ct = lib, ctypes
        self.h = ctypes.c_void_p()
        bus = None
        try:
            import torch
            pr = torch.cuda.get_device_properties(gpu)
            bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        except Exception:
            pass
        if bus is None or lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(self.h)) != 0:
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(gpu), ctypes.byref(self.h)) != 0:
                raise RuntimeError("no NVML handle")
        v = ctypes.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(v)) != 0:      # NVML_CLOCK_SM = 1
            raise RuntimeError("max clock query failed")
        self.maxsm = float(v.value)
        self.sample()

    def sample(self):
        ct, lib = self.ct, self.lib
        v, bits = ct.c_uint(), ct.c_ulonglong()
        if lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(v)) != 0:
            raise RuntimeError("clock query failed")
        if lib.nvmlDeviceGetCurrentClocksThrottleReasons(self.h, ct.byref(bits)) != 0:
            raise RuntimeError("reason query failed")
        return (float(v.value), self.maxsm, int(bits.value))


class ClockSampler:
    """SM clock and clock-event reasons during the timed region.

    In-process NVML polling every 5 ms (plus one sample on entry and one on
    exit), so that even a timed region of a few tens of milliseconds is
    covered; nvidia-smi -lms 200 is the fallback when libnvidia-ml is not
    loadable."""
    REASONS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40), ("sw_thermal_slowdown", 0x20),
               ("sw_power_cap", 0x4))
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.samples = []            # (sm MHz, max sm MHz, reason bits)
        self.nv = None
        self.stop = threading.Event()
        try:
            self.nv = _Nvml(gpu)
        except Exception:
            self.nv = None

    def _sample(self):
        self.samples.append(self.nv.sample())

    def _poll(self):
        while not self.stop.wait(0.005):
            try:
                self._sample()
            except Exception:
                return

    def __enter__(self):
        if self.nv is not None:
            try:
                self._sample()
                self.t = threading.Thread(target=self._poll, daemon=True)
                self.t.start()
                return self
            except Exception:
                self.nv = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.nv is not None:
            self.stop.set()
            self.t.join(timeout=1)
            try:
                self._sample()
            except Exception:
                pass
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        for f, m, bits in self.samples:
            sm.append(f)
            mx.append(m)
            for nm, b in self.REASONS:
                if bits & b:
                    reasons.add(nm)
        names = [nm for nm, _ in self.REASONS]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "source": "nvml 5 ms" if self.samples else "nvidia-smi 200 ms"}


# ------------------------------------------------------------- oracle (CPU)

def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        return max(n) if n else os.cpu_count()
    except Exception:
        return os.cpu_count()


class OracleSample:
    """Bounded sample of the oracle's step on the full workload.

    The oracle solves every step directly (Cholesky of M + dt G, Schur
    complement for the loop voltages): O(N^3) per step, hours at N = 96,000.
    The sample times the oracle's own routines on the leading k-element block
    of the coil's operator (Cholesky, and the Schur solves with k / block
    right-hand sides) and scales them to N by N^3 and N^2 W, and times the
    O(N) parts (field stencil, Jc, E-J law, ADI heat step) on all N elements.
    """

    def __init__(self, w, k=2048):
        import oracle
        from oracle.thermal import ThermalGrid
        g = w.geometry
        self.w = w
        self.geo = oracle.solenoid_elements(g["n_layers"], g["n_turns"], g["n_sub"], g["r_in"],
                                            g["pitch"], g["wire_d"])
        geo = self.geo
        self.N = geo["N"]
        self.k = min(k, self.N)
        sl = slice(0, self.k)
        self.Mk = oracle.assemble_M(geo["r"][sl], geo["z"][sl], geo["h"][sl])
        self.th = ThermalGrid(geo, w.material)
        self.oracle = oracle

    def step_seconds(self):
        import scipy.linalg as sla
        o, geo, w = self.oracle, self.geo, self.w
        N, k, B, W = self.N, self.k, geo["block"], geo["W"]
        rng = np.random.default_rng(0)
        t0 = time.perf_counter()
        phi = np.pi * geo["r"] ** 2 * 0.01 + 1e-9 * rng.standard_normal(N)
        Br, Bz = o.field_from_flux(geo, phi)
        T = np.full(N, w.material["T_bath"])
        Jc = o.critical_current(np.hypot(Br, Bz), T, w.strain, w.jc_factor, w.mat, w.material)
        tm = o.ej_terms(1e-3 * rng.standard_normal(N), Jc, w.mat, geo["r"], geo["area"], w.material)
        u = self.th.to_grid(T ** 4)
        self.th.adi_step(u, self.th.to_grid(tm["q"]), w.drive["dt"])
        t_lin = time.perf_counter() - t0
        A = self.Mk + np.diag(w.drive["dt"] * tm["G"][:k])
        t0 = time.perf_counter()
        cho = sla.cho_factor(A, lower=True)
        t_chol = time.perf_counter() - t0
        nrhs = max(1, k // B)
        P = np.zeros((k, nrhs))
        for j in range(nrhs):
            P[j * B:(j + 1) * B, j] = 1.0
        t0 = time.perf_counter()
        Y = sla.cho_solve(cho, P)
        S = P.T @ Y
        np.linalg.solve(S, np.ones(nrhs))
        t_schur = time.perf_counter() - t0
        scale3 = (N / k) ** 3
        scale_schur = (N / k) ** 2 * (W / nrhs)
        return t_lin + t_chol * scale3 + t_schur * scale_schur

    def describe(self):
        return (f"oracle direct step: Cholesky and Schur solves timed on the leading {self.k}-element "
                f"block of the operator, scaled by (N/k)^3 and (N/k)^2 W/(k/B); field stencil, Jc, "
                f"E-J law and ADI timed on all {self.N} elements")


def cpu_baseline(w, budget_s=20.0):
    smp = OracleSample(w)
    times = []
    t_start = time.perf_counter()
    while not times or (time.perf_counter() - t_start < budget_s and len(times) < 5):
        times.append(smp.step_seconds())
    t = min(times)
    return {"value": smp.N / t, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
            "sample": smp.describe() + f"; best of {len(times)} samples, {t:.1f} s per step"}


# --------------------------------------------------------------- GPU arm

def timed_steps(coil, drive, K, stream, torch):
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    coil.step(K, drive)
    end.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(end) / 1e3


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2403_07666_b300.coil import Coil
    dist = None
    if world > 1:
        import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    w = pick_workload(args.workload)
    drive = w.drive
    stream = torch.cuda.Stream()
    hbm, peak_kind = peaks()
    t0 = time.perf_counter()
    toep = args.format != "dense"
    coil = Coil.from_workload(w, precision=args.precision, rtol=args.rtol, device=local_rank,
                              stream=stream.cuda_stream, format=args.format)
    setup_s = time.perf_counter() - t0
    if args.tc_mode >= 0 and args.format == "toeplitz_tc":
        coil.set_tc_schedule(args.tc_mode)
    info = coil.info()
    N = coil.N
    schedule = coil.tc_schedule() if args.format == "toeplitz_tc" else None
    coil.step(args.warmup, drive)
    coil.reset_counters()
    if dist:
        dist.barrier()
    with ClockSampler(local_rank) as clk:
        secs = timed_steps(coil, drive, args.steps, stream, torch)
    inf = coil.info()
    # replicas: the units of all ranks over the slowest rank's time
    value, secs = job_throughput(secs, N * args.steps, dist, "cuda")
    op_bytes = int(info.operator_bytes)
    applies = int(inf.operator_launches) / args.steps
    launches = int(inf.kernel_launches)
    step_graph = bool(inf.step_graph)
    # the operator apply's own duration: the same warm-up and timed steps on a
    # second coil whose every apply is bracketed by CUDA events on its stream
    # (event records cannot sit inside the step graph's loop, so this coil
    # launches its kernels one by one)
    cp = Coil.from_workload(w, precision=args.precision, rtol=args.rtol, device=local_rank,
                            stream=stream.cuda_stream, profile=True, format=args.format)
    if args.tc_mode >= 0 and args.format == "toeplitz_tc":
        cp.set_tc_schedule(args.tc_mode)
    cp.step(args.warmup, drive)
    cp.reset_counters()
    timed_steps(cp, drive, args.steps, stream, torch)
    ip = cp.info()
    cp.close()
    gemv_ms = ip.operator_ms / max(int(ip.operator_launches), 1)
    roofline = roofline_of(args.format, args.precision, N, op_bytes, gemv_ms, hbm, peak_kind)
    roofline["timed"] = "every apply of the same steps, CUDA events on the coil's stream, kernels launched one by one"

    # end to end through the public API: host buffers, copies inside the region
    import torch as _t
    bufs = [_t.empty(N, dtype=_t.float64, pin_memory=True).numpy() for _ in range(4)]
    Ke = max(1, min(args.steps, 20))
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(Ke):
        coil.step(1, drive)
        coil.read_into(drive, *bufs)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - te
    e2e_value, _ = job_throughput(e2e_s, N * Ke, dist, "cuda")
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": int(inf.descriptor_bytes) + 48,
           "d2h_bytes_per_step": 4 * N * 8 + 8}

    coil.close()
    # the same coil from a state well into a scaled ramp (flux flow under way):
    # the mixed form timed over a window there, then the plain FP64 form and
    # the mixed form stepped side by side from that state
    start_fine = None
    if args.rtol_fine > 0 and args.rtol_fine != args.rtol and args.precision != "fp64":
        start_fine = window_at(args, local_rank, stream, torch, w, drive, args.rtol_fine)
    traj_real = mid_window = None
    if args.traj_steps > 0 and args.precision != "fp64":
        mid_window, traj_real = real_trajectory_leg(args, local_rank, stream, torch, w)
    traj_mid = None
    if args.traj_mid_steps > 0 and args.precision != "fp64":
        traj_mid = trajectory_leg(args, local_rank, stream, torch, wl.mid_coil(), MID_RAMP, 0,
                                  args.traj_mid_steps)

    batched = batch_leg(args, local_rank, stream, torch, rank, world, dist) if args.batch_steps > 0 else None
    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("fp16 hi+lo split operator and input (fp32-class), tensor-core products with fp32 "
                  "accumulation, fp64 solve/accumulation" if args.format == "toeplitz_tc" else
                  {"bf16": "bf16-stored operator, fp32 products, fp64 solve/accumulation",
                   "fp32": "fp32-stored operator, fp32 products, fp64 solve/accumulation",
                   "fp64": "f64"}[args.precision]),
        "data": "synthetic (seeded coil geometry, lognormal Jc factor, uniform strain)",
        "config": {"workload": w.name, "n_elem": N, "n_layers": w.geometry["n_layers"],
                   "n_turns": w.geometry["n_turns"], "n_sub": w.geometry["n_sub"],
                   "precision": args.precision, "dt": drive["dt"], "ramp_A_per_s": drive["ramp_rate"],
                   "rtol": args.rtol, "rtol_fp64": args.rtol_fp64,
                   "parallelism": f"replicas x{world}", "step_graph": step_graph,
                   "operator_format": args.format,
                   "l2": (f"operator table {op_bytes / 1e9:.2f} GB > 126 MB L2 (no flush needed)" if toep else
                          f"operator {op_bytes / 1e9:.1f} GB > 126 MB L2 (no flush needed)")},
        "applies_per_step": applies,
        "rtol_note": ("the mixed form's operator apply is FP32-class (about 1e-7 relative), so its projected PCG "
                      "stops at rtol 1e-6: solving to 1e-9 takes about 11 instead of 4 iterations per step for the "
                      "same solution (its distance from the FP64 form is set by the operator, not the tolerance); "
                      "windows.*.at_rtol_fine time the same steps at 1e-9, and the fp64 legs compare the mixed "
                      "form at this tolerance with the FP64 form at rtol_fp64" if args.precision != "fp64" else
                      "FP64 form"),
        "setup_s": setup_s,
        "roofline": roofline,
        "autotune": schedule,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if mid_window is not None:
        start = {"start_step": args.warmup, "ramp_A_per_s": drive["ramp_rate"], "rtol": args.rtol,
                 "value": value, "ms_per_step": 1e3 * secs / args.steps, "applies_per_step": applies}
        if start_fine is not None:
            start["at_rtol_fine"] = start_fine
        line["windows"] = {"start": start, "mid_ramp": mid_window}
    if traj_real is not None:
        line["fp64"] = traj_real
        line["mixed_over_fp64"] = traj_real["mixed_value"] / traj_real["value"]
        line["mixed_over_fp64_note"] = ("tensor-core block-Toeplitz operator (FP16 hi/lo, FP32-class) with the FP32 "
                                        "pointwise chain against the dense FP64 operator with the FP64 chain, on the "
                                        "same steps from the same state: storage format and precision change together")
    if traj_mid is not None:
        line["fp64_mid"] = traj_mid
    if args.other_format and args.precision == "fp32":
        line["other_formats"] = {f: format_leg(args, local_rank, stream, torch, f)
                                 for f in ("toeplitz_tc", "toeplitz", "dense") if f != args.format}
    if args.lorentz:
        line["lorentz_strain"] = lorentz_leg(args, local_rank, stream, torch)
        line["lorentz_strain"]["over_static"] = line["lorentz_strain"]["value"] / value
    if args.subelements:
        line["subelements"] = subelement_leg(args, local_rank, stream, torch)
        line["subelements"]["over_one_group"] = line["subelements"]["value"] / value
    if args.adjoint_steps > 0:
        line["adjoint"] = adjoint_leg(args, local_rank, stream, torch)
    if batched is not None:
        line["batched"] = batched
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    return line


# FP32 CUDA-core peak of B300 from its unit counts: 148 SMs x 128 FP32 lanes x
# 2 flops per FMA x 2.032 GHz maximum SM clock.
FP32_ALU_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12


def roofline_of(fmt, precision, N, op_bytes, op_ms, hbm, peak_kind):
    """Roofline of the operator apply (all its launches) of one storage format.

    dense: HBM-bound GEMV, algorithmic bytes = the stored operator.
    toeplitz (CUDA cores, FP32): bound by the FP32 pipe, 2 N^2 flops.
    toeplitz_tc (tensor cores): HBM-bound, algorithmic bytes = the split table
    (read once) + the operator's input and result (4 + 8 bytes per element);
    the duration is the product kernel's (k_toeplitz_tc) alone, the input
    split being a kernel of its own; its tensor work, 3 x 2 N^2 FP16 flops
    (hi.hi, hi.lo, lo.hi), is reported beside it."""
    if fmt == "toeplitz":
        flops = 2.0 * N * N
        achieved = flops / (op_ms / 1e3) / 1e12
        prof = PROFILED_TRAFFIC.get("toeplitz")
        traffic = prof["dram_bytes"] * op_bytes / prof["operator_bytes"] if prof else None
        return {"bound": "alu", "achieved": achieved, "peak": FP32_ALU_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_ALU_TFLOPS, "traffic": traffic,
                "kernel": "k_toeplitz_f32 (+transpose, reduce)",
                "peak_kind": "derived: 148 SM x 128 FP32 lanes x 2 flop x 2.032 GHz",
                "avg_launch_ms": op_ms, "flops_per_launch": flops, "table_bytes": op_bytes}
    if fmt == "toeplitz_tc":
        nbytes = op_bytes + 12.0 * N
        achieved = nbytes / (op_ms / 1e3) / 1e9
        prof = PROFILED_TRAFFIC.get("toeplitz_tc")
        traffic = prof["dram_bytes"] * op_bytes / prof["operator_bytes"] if prof else None
        return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "kernel": "k_toeplitz_tc", "peak_kind": peak_kind,
                "avg_launch_ms": op_ms, "bytes_per_launch": nbytes, "table_bytes": op_bytes,
                "tensor_tflops_fp16": 6.0 * N * N / (op_ms / 1e3) / 1e12}
    achieved = op_bytes / (op_ms / 1e3) / 1e9
    prof = PROFILED_TRAFFIC.get(precision)
    traffic = prof["dram_bytes"] * op_bytes / prof["operator_bytes"] if prof else None
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "kernel": f"k_gemv_{precision}", "peak_kind": peak_kind,
            "avg_launch_ms": op_ms, "bytes_per_launch": op_bytes}


def format_leg(args, local_rank, stream, torch, fmt):
    """The same coil and steps with the far operator in another FP32 storage format."""
    from paper_2403_07666_b300.coil import Coil
    w = pick_workload(args.workload)
    hbm, peak_kind = peaks()
    secs, inf, N = None, None, 0
    for profile in (False, True):           # the step's time, then every apply's (as the main line)
        c = Coil.from_workload(w, precision="fp32", rtol=args.rtol, device=local_rank,
                               stream=stream.cuda_stream, profile=profile, format=fmt)
        c.step(args.warmup, w.drive)
        c.reset_counters()
        t = timed_steps(c, w.drive, args.steps, stream, torch)
        if not profile:
            secs, N = t, c.N
        else:
            inf = c.info()
        c.close()
    op_ms = inf.operator_ms / max(int(inf.operator_launches), 1)
    op_bytes = int(inf.operator_bytes)
    return {"value": N * args.steps / secs, "unit": UNIT, "ms_per_step": 1e3 * secs / args.steps,
            "applies_per_step": int(inf.operator_launches) / args.steps, "operator_bytes": op_bytes,
            "roofline": roofline_of(fmt, "fp32", N, op_bytes, op_ms, hbm, peak_kind)}


# Effective Young's modulus of an epoxy-impregnated Nb3Sn winding [Pa] for the
# Lorentz hoop-strain leg.
Y_WINDING = 5e10


def lorentz_leg(args, local_rank, stream, torch):
    """The same coil and steps with the Lorentz hoop strain feeding Jc."""
    from paper_2403_07666_b300.coil import Coil
    w = pick_workload(args.workload)
    w.material["Y_eff"] = Y_WINDING
    c = Coil.from_workload(w, precision=args.precision, rtol=args.rtol, device=local_rank,
                           stream=stream.cuda_stream, format=args.format)
    c.step(args.warmup, w.drive)
    secs = timed_steps(c, w.drive, args.steps, stream, torch)
    N = c.N
    c.close()
    return {"Y_eff_Pa": Y_WINDING, "value": N * args.steps / secs, "unit": UNIT,
            "ms_per_step": 1e3 * secs / args.steps}


def subelement_leg(args, local_rank, stream, torch):
    """The same coil and steps with every turn split into subelements (the Cu
    ring and the four filament quadrants): the transport part solved per turn,
    one net-current constraint per subelement in the coupled solve."""
    from paper_2403_07666_b300.coil import Coil
    w = pick_workload(args.workload)
    grp = wl.subelement_groups(w.geometry["n_sub"])
    w.geometry["groups"] = grp
    c = Coil.from_workload(w, precision=args.precision, rtol=args.rtol, device=local_rank,
                           stream=stream.cuda_stream, format=args.format)
    c.step(args.warmup, w.drive)
    c.reset_counters()
    secs = timed_steps(c, w.drive, args.steps, stream, torch)
    inf = c.info()
    N = c.N
    c.close()
    return {"groups_per_turn": int(grp.max()) + 1, "value": N * args.steps / secs, "unit": UNIT,
            "ms_per_step": 1e3 * secs / args.steps,
            "applies_per_step": int(inf.operator_launches) / args.steps}


def adjoint_leg(args, local_rank, stream, torch):
    """Adjoint / forward cost on the 4,608-element field-loop coil (one full
    triangle loop of the applied field in 1000 steps of 1e-4 s, checkpoints
    every 50 steps), in the headline operator form and in the plain FP64
    form.  The loss is a magnetization-loop term on the moment series plus a
    soft maximum of the Joule-power series (the quench-onset term)."""
    from paper_2403_07666_b300.coil import Coil
    w = wl.adjoint_coil()
    K = args.adjoint_steps
    out = {"workload": w.name, "n_elem": w.n_elem, "steps": K, "checkpoint_every": 50,
           "loss": "sum (m_k - m_target)^2 + soft maximum of the Joule power P_k",
           "note": "adjoint_s includes the checkpointed forward pass and the segment recomputation"}
    forms = [(args.format, {"precision": args.precision, "format": args.format})]
    if args.format != "dense" or args.precision != "fp64":
        forms.append(("fp64", {"precision": "fp64"}))
    for name, kw in forms:
        rt = args.rtol_fp64 if name == "fp64" else args.rtol
        c = Coil.from_workload(w, rtol=rt, device=local_rank, stream=stream.cuda_stream, **kw)
        s0 = c.save_state()
        c.step(3, w.drive)
        c.load_state(s0)
        c.reset_counters()
        fwd = timed_steps(c, w.drive, K, stream, torch)
        it_fwd = int(c.info().pcg_iterations)
        d = c.diag(0, K)
        m, P = d[:, 3], d[:, 4]
        target = 0.95 * m
        scale = 0.05 * max(float(np.max(P)), 1e-300)
        z = P / scale
        wts = np.exp(z - np.max(z))
        dLdP = wts / np.sum(wts)
        c.load_state(s0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c.reset_counters()
        c.adjoint_losses(K, w.drive, 2.0 * (m - target), dLdP, ckpt_every=50)
        torch.cuda.synchronize()
        adj = time.perf_counter() - t0
        it_adj = int(c.info().pcg_iterations)
        c.close()
        out[name] = {"rtol": rt, "forward_s": fwd, "adjoint_s": adj, "adjoint_over_forward": adj / fwd,
                     "pcg_iterations_forward": it_fwd, "pcg_iterations_adjoint_call": it_adj}
    out["adjoint_over_forward"] = out[args.format]["adjoint_over_forward"]
    return out


# Scaled transport ramps of the trajectory legs (the configurations' ramps
# reach only a few amperes in their step windows; x1000 brings the coils into
# flux flow and past their first flux jump within a few thousand steps: the
# 96,000-element coil's first jump at 2000 A/s comes near step 1990, the
# 51,200-element coil's at 5000 A/s near step 970).
REAL_RAMP = 2000.0
MID_RAMP = 5000.0


def c13_errors(got, ref, T_bath, m_scale):
    """Per-step errors of the mixed form against the FP64 form: J, B and the
    heating T - T_bath relative to the step's maximum (the heating with a
    floor of 1e-6 T_bath), the moment relative to the largest |m| so far."""
    def rel(a, b):
        sc = np.max(np.abs(b))
        return float(np.max(np.abs(a - b)) / sc) if sc > 0 else float(np.max(np.abs(a - b)))
    eJ = rel(got["J"], ref["J"])
    eB = max(rel(got["Br"], ref["Br"]), rel(got["Bz"], ref["Bz"]))
    eT = float(np.max(np.abs(got["T"] - ref["T"])) / max(np.max(np.abs(ref["T"] - T_bath)), 1e-6 * T_bath))
    em = abs(got["moment"] - ref["moment"]) / max(m_scale, 1e-300)
    return eJ, eB, eT, em


C13_BOUNDS = {"J": 1e-3, "B": 1e-4, "T": 1e-3, "m": 1e-4}


def trajectory_leg(args, local_rank, stream, torch, w, ramp, pre_steps, steps, state=None):
    """The mixed form (tensor-core operator) and the plain FP64 form (dense
    FP64 operator) stepped side by side on a scaled ramp, from t = 0 or from
    a saved state; every step's J, B, T and moment compared (C-13 bounds)."""
    from paper_2403_07666_b300.coil import Coil
    d = dict(w.drive, ramp_rate=ramp)
    T_bath = w.material["T_bath"]
    cm = Coil.from_workload(w, precision="fp32", format="toeplitz_tc", rtol=args.rtol, device=local_rank,
                            stream=stream.cuda_stream)
    c64 = Coil.from_workload(w, precision="fp64", rtol=args.rtol_fp64, device=local_rank, stream=stream.cuda_stream)
    if state is not None:
        cm.load_state(state)
        c64.load_state(state)
    elif pre_steps > 0:
        cm.step(pre_steps, d)
        st = cm.save_state()
        c64.load_state(st)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    t64 = tm = 0.0
    worst = {"J": 0.0, "B": 0.0, "T": 0.0, "m": 0.0}
    m_scale = 0.0
    max_jr = 0.0
    c64.reset_counters()
    cm.reset_counters()
    for _ in range(steps):
        ev[0].record(stream)
        c64.step(1, d)
        ev[1].record(stream)
        cm.step(1, d)
        ev[2].record(stream)
        ref, got = c64.read(d), cm.read(d)
        torch.cuda.synchronize()
        t64 += ev[0].elapsed_time(ev[1]) / 1e3
        tm += ev[1].elapsed_time(ev[2]) / 1e3
        m_scale = max(m_scale, abs(ref["moment"]))
        for k, e in zip(("J", "B", "T", "m"), c13_errors(got, ref, T_bath, m_scale)):
            worst[k] = max(worst[k], e)
    dg = c64.diag()
    max_jr = float(np.max(dg[-steps:, 6]))
    fj, _ = c64.onsets()
    fjm, _ = cm.onsets()
    i64, im = c64.info(), cm.info()
    N = cm.N
    out = {"workload": w.name, "n_elem": N, "ramp_A_per_s": ramp,
           "start_step": int(i64.steps) - steps, "compared_steps": steps,
           "value": N * steps / t64, "ms_per_step": 1e3 * t64 / steps,
           "applies_per_step": int(i64.operator_launches) / steps,
           "mixed_value": N * steps / tm, "mixed_ms_per_step": 1e3 * tm / steps,
           "mixed_applies_per_step": int(im.operator_launches) / steps,
           "max_rel_err": worst, "bounds": C13_BOUNDS,
           "within_bounds": all(worst[k] <= C13_BOUNDS[k] for k in C13_BOUNDS),
           "max_J_over_Jc": max_jr,
           "wires_jumped": {"fp64": int((fj >= 0).sum()), "mixed": int((fjm >= 0).sum())},
           "first_jump_step": {"fp64": int(fj[fj >= 0].min()) if (fj >= 0).any() else -1,
                               "mixed": int(fjm[fjm >= 0].min()) if (fjm >= 0).any() else -1},
           "timed": "CUDA events around every step of each form (state read back between steps, not timed)"}
    cm.close()
    c64.close()
    return out


def window_at(args, local_rank, stream, torch, w, d, rtol, state=None):
    """The same timed window of the mixed form at another PCG tolerance."""
    from paper_2403_07666_b300.coil import Coil
    c = Coil.from_workload(w, precision=args.precision, rtol=rtol, device=local_rank,
                           stream=stream.cuda_stream, format=args.format)
    if state is not None:
        c.load_state(state)
    c.step(args.warmup, d)
    c.reset_counters()
    secs = timed_steps(c, d, args.steps, stream, torch)
    inf = c.info()
    N = c.N
    c.close()
    return {"rtol": rtol, "value": N * args.steps / secs, "ms_per_step": 1e3 * secs / args.steps,
            "applies_per_step": int(inf.operator_launches) / args.steps}


def real_trajectory_leg(args, local_rank, stream, torch, w):
    """The bench coil from a state well into the scaled ramp: a timed window
    of the mixed form there, then the FP64 comparison from the same state."""
    from paper_2403_07666_b300.coil import Coil
    d = dict(w.drive, ramp_rate=REAL_RAMP)
    c = Coil.from_workload(w, precision=args.precision, rtol=args.rtol, device=local_rank,
                           stream=stream.cuda_stream, format=args.format)
    c.step(args.traj_pre, d)
    state = c.save_state()
    c.step(args.warmup, d)
    c.reset_counters()
    secs = timed_steps(c, d, args.steps, stream, torch)
    inf = c.info()
    N = c.N
    window = {"start_step": args.traj_pre + args.warmup, "ramp_A_per_s": REAL_RAMP, "steps": args.steps,
              "rtol": args.rtol, "value": N * args.steps / secs, "ms_per_step": 1e3 * secs / args.steps,
              "applies_per_step": int(inf.operator_launches) / args.steps,
              "max_J_over_Jc": float(np.max(c.diag()[-args.steps:, 6]))}
    c.close()
    if args.rtol_fine > 0 and args.rtol_fine != args.rtol:
        window["at_rtol_fine"] = window_at(args, local_rank, stream, torch, w, d, args.rtol_fine, state)
    traj = trajectory_leg(args, local_rank, stream, torch, w, REAL_RAMP, 0, args.traj_steps, state=state)
    return window, traj


def batch_leg(args, local_rank, stream, torch, rank=0, world=1, dist=None):
    """64 coils of uneven size (2k-41k elements) stepped together; with several
    ranks each steps its share of the coils (dealt by element count)."""
    from paper_2403_07666_b300.coil import Coil, batch_step
    ws_all = wl.batch_coils()
    ws = [ws_all[i] for i in shard_coils([w.n_elem for w in ws_all], world, rank)]
    fmt = args.batch_format if args.precision == "fp32" else "dense"
    coils = [Coil.from_workload(w, precision=args.precision, rtol=args.rtol, device=local_rank,
                                stream=stream.cuda_stream, format=fmt) for w in ws]
    drives = [w.drive for w in ws]
    batch_step(coils, args.warmup, drives)
    for c in coils:
        c.reset_counters()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    batch_step(coils, args.batch_steps, drives)
    end.record(stream)
    torch.cuda.synchronize()
    secs = start.elapsed_time(end) / 1e3
    local_elem = sum(c.N for c in coils)
    launches = int(coils[0].info().kernel_launches)
    op_bytes = sum(int(c.info().operator_bytes) for c in coils)
    for c in coils:
        c.close()
    value, secs = job_throughput(secs, local_elem * args.batch_steps, dist, "cuda")
    total_elem = sum(w.n_elem for w in ws_all)
    return {"workload": f"batch of {len(ws_all)} coils", "n_elem_total": total_elem,
            "n_elem_min": min(w.n_elem for w in ws_all), "n_elem_max": max(w.n_elem for w in ws_all),
            "ranks": world, "steps": args.batch_steps, "value": value, "unit": UNIT,
            "ms_per_step": 1e3 * secs / args.batch_steps, "operator_format": fmt, "operator_bytes": op_bytes,
            "gpu_launches": launches}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    w = pick_workload(args.workload)
    smp = OracleSample(w)
    for _ in range(args.warmup):
        smp.step_seconds()
    total = 0.0
    for _ in range(args.steps):
        total += smp.step_seconds()
    value = smp.N * args.steps / total
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded coil geometry, lognormal Jc factor, uniform strain)",
            "config": {"workload": w.name, "n_elem": smp.N},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                             "sample": smp.describe()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def apply_once(args):
    """One operator apply on the workload (for profiler captures of the apply
    kernel): the coil built as in the main leg, the tensor-core schedule
    optionally pinned (--tc-mode), one apply of a seeded input; prints the
    schedule and the apply's wall time."""
    import torch
    from paper_2403_07666_b300.coil import Coil
    w = pick_workload(args.workload)
    c = Coil.from_workload(w, precision=args.precision, rtol=args.rtol, device=0, format=args.format)
    if args.tc_mode >= 0:
        c.set_tc_schedule(args.tc_mode)
    p = np.random.default_rng(0).standard_normal(c.N)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c.apply_operator(p)
    torch.cuda.synchronize()
    out = {"workload": w.name, "apply_s": time.perf_counter() - t0}
    if args.format == "toeplitz_tc":
        out["schedule"] = c.tc_schedule()
    c.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 50 for the GPU arm, 10 oracle samples for the reference arm)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="real", choices=["real", "mid", "small", "prof"])
    ap.add_argument("--precision", default="fp32", choices=["bf16", "fp32", "fp64"])
    ap.add_argument("--rtol", type=float, default=None,
                    help="PCG tolerance of the timed form (default: 1e-6 for the mixed form, whose "
                         "FP32-class operator does not support a finer solve, 1e-9 for FP64)")
    ap.add_argument("--rtol-fp64", type=float, default=1e-9, help="PCG tolerance of the plain FP64 form")
    ap.add_argument("--rtol-fine", type=float, default=1e-9,
                    help="the mixed form's headline window also timed at this tolerance (0: skip)")
    ap.add_argument("--traj-pre", type=int, default=1900,
                    help="steps of the mixed form on the scaled ramp before the mid-ramp window and the FP64 comparison")
    ap.add_argument("--traj-steps", type=int, default=200,
                    help="steps of the plain FP64 form beside the mixed form from the mid-ramp state (0: skip)")
    ap.add_argument("--traj-mid-steps", type=int, default=1100,
                    help="steps of the FP64 / mixed comparison on the 51,200-element coil from t = 0 (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--format", default="toeplitz_tc", choices=["toeplitz_tc", "toeplitz", "dense"],
                    help="storage of the far operator in the main leg")
    ap.add_argument("--other-format", type=int, default=1, help="also time the other operator formats")
    ap.add_argument("--adjoint-steps", type=int, default=1000)
    ap.add_argument("--lorentz", type=int, default=1, help="also time the step with the Lorentz hoop strain")
    ap.add_argument("--subelements", type=int, default=1, help="also time the step with subelement decoupling")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--batch-format", default="toeplitz_tc", choices=["toeplitz_tc", "toeplitz", "dense"])
    ap.add_argument("--apply-once", action="store_true",
                    help="build the coil, run one operator apply and exit (profiler captures of the apply)")
    ap.add_argument("--tc-mode", type=int, default=-1,
                    help="pin the tensor-core schedule of the main leg and of --apply-once (0 two-fill, "
                         "1 one-fill; default: the autotuner's choice), e.g. for profiler captures, under "
                         "which the autotuner's timings differ")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.steps is None:
        args.steps = 10 if args.impl == "reference" else 50
    if args.rtol is None:
        args.rtol = 1e-9 if args.precision == "fp64" else 1e-6
    if args.apply_once:
        print(json.dumps(apply_once(args)), flush=True)
        return
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        line = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
