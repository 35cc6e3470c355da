"""Seeded synthetic coil workloads (inputs only: no arithmetic of the method).

The paper's measured coils and wire data are not available (Data
Availability: on request), so synthetic coils of the paper's shapes stand in
for them (Experiments section: Nb3Sn solenoid, 4.2 K bath, ramped transport
current; quench section: 20 x 20 turns, 2 A/s).  Every random array comes
from numpy's PCG64 generator seeded per workload and is handed unchanged to
the library and to the oracle.

Recipe per solenoid workload:
  * n_layers x n_turns square wires, n_sub x n_sub elements each, inner
    radius 20 mm, wire side 0.8 mm on a 0.9 mm pitch;
  * filament mask: an element is superconducting when its centre lies in the
    centred square of half-side d / (2 sqrt(2.05)) (Cu : Nb3Sn = 1.05 by
    area), else Cu;
  * per-element Jc factor exp(0.05 z), z ~ N(0, 1) (median-1 lognormal);
  * per-element strain uniform in [-0.003, 0];
  * drive: transport ramp, dt = 1e-5 s.
"""

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 7666000

# material constants of the synthetic Nb3Sn coil (SI units)
MATERIAL = {
    "E0": 1e-4, "n": 30.0, "Jc0": 5e10, "Tc": 18.0, "Bc2_0": 28.0, "B_reg": 0.1,
    "C_eps": 900.0, "p_eps": 1.7, "rho_n": 1.7e-10, "rho_m": 8900.0, "c0": 0.1,
    "kappa_cu": 2.44e-8 * 4.2 / 1.7e-10,          # Wiedemann-Franz at 4.2 K
    "kappa_ep": 2.44e-8 * 4.2 / 1.7e-10 * 10 ** -3.5,
    "h0": 500.0, "T_ref": 4.2, "T_bath": 4.2, "jc_model": 0, "thermal": 1,
}


@dataclass
class Workload:
    name: str
    geometry: dict                      # solenoid parameters or explicit list
    material: dict
    jc_factor: np.ndarray
    strain: np.ndarray
    mat: np.ndarray                     # 1 = filament, 0 = Cu, element order
    drive: dict
    steps: int
    constrained: np.ndarray = None      # per block; None = every block
    extra: dict = field(default_factory=dict)

    @property
    def n_elem(self):
        return int(self.jc_factor.size)


def filament_mask(n_layers, n_turns, n_sub):
    """1 where the element centre is inside the filament zone, element order."""
    n = n_sub
    N = n_layers * n_turns * n * n
    e = np.arange(N)
    a = e % n
    b = (e // n) % n
    half = 0.5 / np.sqrt(2.05)             # in units of the wire side
    xa = (a + 0.5) / n - 0.5
    xb = (b + 0.5) / n - 0.5
    return ((np.abs(xa) < half) & (np.abs(xb) < half)).astype(np.int32)


def subelement_groups(n_sub, tile=None):
    """Subelement id of every element position of a wire (position b n + a):
    the Cu elements (outside the filament zone) form one group; the filament
    zone splits into its four quadrants about the wire centre, or with `tile`
    into tile x tile squares of filament elements counted from the zone's
    corner; ids renumbered from 0 in order of (Cu, subelement index)."""
    n = n_sub
    fil = filament_mask(1, 1, n)
    ks = [k for k in range(n * n) if fil[k]]
    a0 = min(k % n for k in ks) if ks else 0
    b0 = min(k // n for k in ks) if ks else 0
    raw = []
    for b in range(n):
        for a in range(n):
            k = b * n + a
            if not fil[k]:
                raw.append(0)
            elif tile is None:
                raw.append(1 + int(2 * a >= n) + 2 * int(2 * b >= n))
            else:
                raw.append(1 + (a - a0) // tile + n * ((b - b0) // tile))
    ids = {v: i for i, v in enumerate(sorted(set(raw)))}
    return np.array([ids[v] for v in raw], dtype=np.int32)


def solenoid(name, n_layers, n_turns, n_sub, seed, ramp_rate=10.0, I_max=400.0, dt=1e-5,
             steps=2000, r_in=0.020, pitch=0.9e-3, wire_d=0.8e-3, material=None,
             Ba_rate=0.0, Ba_max=0.0, Ba_waveform=0):
    rng = np.random.Generator(np.random.PCG64(seed))
    N = n_layers * n_turns * n_sub * n_sub
    zf = rng.standard_normal(N)
    jc_factor = np.exp(0.05 * zf)
    strain = rng.uniform(-0.003, 0.0, N)
    mat = filament_mask(n_layers, n_turns, n_sub)
    geom = {"kind": "solenoid", "n_layers": n_layers, "n_turns": n_turns, "n_sub": n_sub,
            "r_in": r_in, "pitch": pitch, "wire_d": wire_d, "transport": 1}
    drive = {"dt": dt, "ramp_rate": ramp_rate, "I_max": I_max, "Ba_rate": Ba_rate,
             "Ba_max": Ba_max, "Ba_waveform": Ba_waveform}
    mtl = dict(MATERIAL if material is None else material)
    return Workload(name, geom, mtl, jc_factor, strain, mat, drive, steps)


def small_coil():
    """4 layers x 8 turns, 4 x 4 elements: 512 elements, FP64, 2000 steps."""
    return solenoid("small-32turn-512el", 4, 8, 4, SEED_BASE + 1, ramp_rate=10.0,
                    I_max=400.0, steps=2000)


def mid_coil():
    """20 layers x 40 turns, 8 x 8 elements: 51,200 elements."""
    return solenoid("mid-800turn-51200el", 20, 40, 8, SEED_BASE + 2, ramp_rate=5.0,
                    I_max=600.0, steps=20000)


def profile_coil():
    """24 layers x 52 turns, 4 x 4 elements: 19,968 elements (operator > L2)."""
    return solenoid("profile-1248turn-19968el", 24, 52, 4, SEED_BASE + 6, ramp_rate=2.0,
                    I_max=800.0, steps=100)


def adjoint_coil():
    """12 layers x 24 turns, 4 x 4 elements: 4,608 elements, field loop."""
    w = solenoid("adjoint-288turn-4608el", 12, 24, 4, SEED_BASE + 4, ramp_rate=0.0,
                 I_max=0.0, dt=1e-4, steps=1000, Ba_rate=4.0, Ba_max=0.1, Ba_waveform=2)
    return w


def real_coil():
    """60 layers x 100 turns, 4 x 4 elements: 96,000 elements."""
    return solenoid("real-6000turn-96000el", 60, 100, 4, SEED_BASE + 5, ramp_rate=2.0,
                    I_max=800.0, steps=100000)


def batch_coils(count=64, seed=SEED_BASE + 3, n_min=2000, n_max=41472):
    """Uneven coils: layers U{4..24}, turns U{8..48}, n in {4, 6}, redrawn
    until n_min <= N <= n_max; ramp log-uniform in [0.5, 50] A/s, bath
    uniform in [1.9, 4.5] K."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < count:
        L = int(rng.integers(4, 25))
        T = int(rng.integers(8, 49))
        n = int(rng.choice([4, 6]))
        N = L * T * n * n
        if not (n_min <= N <= n_max):
            continue
        ramp = float(np.exp(rng.uniform(np.log(0.5), np.log(50.0))))
        tb = float(rng.uniform(1.9, 4.5))
        mtl = dict(MATERIAL)
        mtl["T_bath"] = tb
        out.append(solenoid(f"batch-{len(out)}-{L}x{T}x{n}", L, T, n,
                            seed + 1000 + len(out), ramp_rate=ramp, I_max=800.0,
                            material=mtl, steps=100))
    return out


def random_coil(seed, n_layers, n_turns, n_sub, **kw):
    """Small seeded coil for parity tests."""
    return solenoid(f"coil-{n_layers}x{n_turns}x{n_sub}-s{seed}", n_layers, n_turns, n_sub,
                    seed, **kw)
