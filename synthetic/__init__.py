"""Seeded synthetic inputs for the LLG + cavity workloads.

This module holds no arithmetic of the method: only counter-based random
numbers, initial magnetisation patterns, masks, coupling-profile shapes and
the workload table (grid, cell size, material, bias, cavity and integrator
settings).  Both the FP64 oracle and the CUDA library receive identical arrays
from here (rounded to float32 first where the library takes float32).

The paper's own workloads need COMSOL / 3D-MLSI field maps that are not
available; the workloads below are synthetic films, wires and disks with the
paper's material constants (YIG and Permalloy, Appendix D) and the script style
of its example (Appendix D listing).

Random numbers: splitmix64 (Steele, Lea & Flood 2014) in counter mode,
u_k = mix(seed + (k + 1) * 0x9E3779B97F4A7C15) / 2^64 (top 53 bits).
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

MASTER_SEED = 20241001
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_HERE = os.path.dirname(os.path.abspath(__file__))
LITERALS_PATH = os.path.join(_HERE, "workload_literals.json")


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Raw 64-bit outputs number `counters` of the splitmix64 stream started at `seed`."""
    with np.errstate(over="ignore"):
        c = np.asarray(counters, dtype=np.uint64)
        return _mix(np.uint64(seed % (1 << 64)) + (c + np.uint64(1)) * _GOLDEN)


def uniform(seed: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the 53 top bits of the stream."""
    return (splitmix64(seed, counters) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def derive_seed(*keys: int) -> int:
    """Seed for (config, instance, ...) from the master seed by chained mixing."""
    s = MASTER_SEED
    for k in keys:
        s = int(splitmix64(s, np.array([k]))[0])
    return s


# ---------------------------------------------------------------------------
# initial states, masks, profiles
# ---------------------------------------------------------------------------

def tilted_m(n: int, seed: int, theta_max: float = 0.05, axis: str = "x") -> np.ndarray:
    """n unit vectors tilted from `axis` by theta ~ U[0, theta_max], phi ~ U[0, 2pi); float32 (n, 3)."""
    k = np.arange(n, dtype=np.uint64)
    th = theta_max * uniform(seed, 2 * k)
    ph = 2.0 * math.pi * uniform(seed, 2 * k + 1)
    a = np.cos(th)
    b = np.sin(th) * np.cos(ph)
    c = np.sin(th) * np.sin(ph)
    if axis == "x":
        m = np.stack([a, b, c], 1)
    elif axis == "y":
        m = np.stack([c, a, b], 1)
    else:
        m = np.stack([b, c, a], 1)
    return m.astype(np.float32)


def random_m(n: int, seed: int) -> np.ndarray:
    """n directions uniform on the sphere (float32 (n,3)); used for field-parity inputs."""
    k = np.arange(n, dtype=np.uint64)
    z = 2.0 * uniform(seed, 2 * k) - 1.0
    ph = 2.0 * math.pi * uniform(seed, 2 * k + 1)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(ph), r * np.sin(ph), z], 1).astype(np.float32)


def cell_centres(nx, ny, nz, dx, dy, dz):
    """Cell-centre coordinates measured from the grid centre, arrays of shape (nz, ny, nx)."""
    x = (np.arange(nx) + 0.5 - nx / 2) * dx
    y = (np.arange(ny) + 0.5 - ny / 2) * dy
    z = (np.arange(nz) + 0.5 - nz / 2) * dz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def disk_ms(nx, ny, nz, dx, dy, diameter, Ms) -> np.ndarray:
    """Ms map (float32, N) of a disk: Ms inside (cell centre within the circle), 0 outside."""
    X, Y, _ = cell_centres(nx, ny, nz, dx, dy, 1.0)
    inside = X * X + Y * Y <= (diameter / 2) ** 2
    return np.where(inside, Ms, 0.0).astype(np.float32).ravel()


def uniform_ms_map(n: int, seed: int, lo: float, hi: float) -> np.ndarray:
    return (lo + (hi - lo) * uniform(seed, np.arange(n, dtype=np.uint64))).astype(np.float32)


def vortex_m(nx, ny, nz, dx, dy, seed, core_radius=10e-9) -> Tuple[np.ndarray, int, int]:
    """Vortex ansatz with seeded chirality c and polarity p (each +-1); float32 (N, 3)."""
    u = uniform(seed, np.arange(2, dtype=np.uint64))
    chir = 1 if u[0] < 0.5 else -1
    pol = 1 if u[1] < 0.5 else -1
    X, Y, _ = cell_centres(nx, ny, nz, dx, dy, 1.0)
    r = np.sqrt(X * X + Y * Y)
    mz = pol * np.exp(-(r / core_radius) ** 2)
    ip = np.sqrt(np.maximum(0.0, 1.0 - mz * mz))
    phi = np.arctan2(Y, X)
    m = np.stack([-chir * ip * np.sin(phi), chir * ip * np.cos(phi), mz], -1).reshape(-1, 3)
    return m.astype(np.float32), chir, pol


def lorentzian_profile(nx, ny, nz, dx, width, direction=(0.0, 1.0, 0.0)) -> np.ndarray:
    """Dimensionless coupling profile p_i = dir / (1 + (x_i / width)^2), x from the grid centre."""
    X, _, _ = cell_centres(nx, ny, nz, dx, 1.0, 1.0)
    s = 1.0 / (1.0 + (X / width) ** 2)
    d = np.asarray(direction, dtype=np.float64)
    return (s.reshape(-1, 1) * d[None, :]).astype(np.float32)


# ---------------------------------------------------------------------------
# workload table
# ---------------------------------------------------------------------------

PY = dict(Ms=8e5, Aex=1.3e-11)           # Permalloy-like
YIG = dict(Ms=1.4e5, Aex=3.65e-12)       # YIG-like


@dataclass
class Instance:
    """One simulation: grid, material, bias, cavity."""
    nx: int
    ny: int
    nz: int
    d: float
    Ms: float
    Aex: float
    alpha: float
    Ku: float = 0.0
    axis: Tuple[float, float, float] = (1.0, 0.0, 0.0)
    bias: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    omega_c: float = 0.0
    kappa: float = 0.0
    g: float = 0.0
    seed: int = 0
    tilt: float = 0.05
    profile: str = "uniform_y"           # or "lorentzian"
    profile_width: float = 0.0

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    def m0(self) -> np.ndarray:
        return tilted_m(self.n, self.seed, self.tilt, "x")

    def coupling_profile(self) -> Optional[np.ndarray]:
        if self.profile == "lorentzian":
            return lorentzian_profile(self.nx, self.ny, self.nz, self.d, self.profile_width)
        return None


@dataclass
class Workload:
    name: str
    instances: List[Instance]
    integrator: str        # "rk4" or "dp45"
    dt: float              # fixed step (rk4) or first trial step (dp45)
    horizon: float         # simulated time per instance (s)
    tol: float = 1e-6
    note: str = ""


def literals() -> dict:
    """Numbers derived once by synthetic/make_literals.py (Kittel frequencies)."""
    with open(LITERALS_PATH) as f:
        return json.load(f)


def _twopi(f):
    return 2.0 * math.pi * f


def film_32() -> Workload:
    """Permalloy film 32x32x1 cells of 4 nm, RK4 dt = 0.1 ps for 5000 steps."""
    lit = literals()
    inst = Instance(32, 32, 1, 4e-9, alpha=0.01, bias=(0.05, 0.0, 0.0),
                    omega_c=lit["film_32_omega_kittel"], kappa=_twopi(10e6), g=_twopi(50e6),
                    seed=derive_seed(1, 0), **PY)
    return Workload("film 32x32x1 @4nm", [inst], "rk4", 1e-13, 5000 * 1e-13)


def yig_wire_sweep(n_sweep: int = 21) -> Workload:
    """YIG wire 256x64x16 cells of 5 nm, omega_c swept over the uniform mode in 21 values."""
    lit = lit_ = literals()
    wk = lit_["yig_wire_omega_kittel"]
    g = _twopi(50e6)
    insts = []
    for k in range(n_sweep):
        insts.append(Instance(256, 64, 16, 5e-9, alpha=1e-4, Ku=1e3, axis=(1.0, 0.0, 0.0),
                              bias=(0.1, 0.0, 0.0), omega_c=wk + (k - n_sweep // 2) * g / 2,
                              kappa=_twopi(10e6), g=g, seed=derive_seed(2, k), **YIG))
    return Workload("YIG wire 256x64x16 @5nm, 21-value omega_c sweep", insts, "dp45", 1e-13, 10e-9)


BATCH_GRIDS = [(32, 32, 1), (64, 64, 2), (128, 128, 2), (256, 256, 4)]


def batched_map(n_inst: int = 64) -> Workload:
    """64 Permalloy instances of mixed grids on an 8x8 (bias, omega_c) anticrossing map."""
    seed = derive_seed(3)
    pick = uniform(seed, np.arange(n_inst, dtype=np.uint64))
    perm = np.argsort(uniform(derive_seed(3, 1), np.arange(n_inst, dtype=np.uint64)), kind="stable")
    side = int(round(math.sqrt(n_inst)))
    biases = np.linspace(0.02, 0.2, side)
    fcs = np.linspace(2e9, 12e9, side)
    insts = []
    for i in range(n_inst):
        nx, ny, nz = BATCH_GRIDS[int(pick[i] * len(BATCH_GRIDS))]
        cell = int(perm[i])
        insts.append(Instance(nx, ny, nz, 4e-9, alpha=0.01, bias=(float(biases[cell // side]), 0.0, 0.0),
                              omega_c=_twopi(fcs[cell % side]), kappa=_twopi(10e6), g=_twopi(100e6),
                              seed=derive_seed(3, 2, i), **PY))
    return Workload("batched 64 mixed grids, anticrossing map", insts, "rk4", 5e-14, 2e-9)


def large_cpw() -> Workload:
    """1024x1024x8 cells of 4 nm Permalloy, Lorentzian coupling profile g(x), DP45 for 5 ns."""
    lit = literals()
    inst = Instance(1024, 1024, 8, 4e-9, alpha=0.01, bias=(0.03, 0.0, 0.0),
                    omega_c=lit["large_cpw_omega_kittel"], kappa=_twopi(10e6), g=_twopi(20e6),
                    seed=derive_seed(5, 0), profile="lorentzian", profile_width=500e-9, **PY)
    return Workload("CPW-like 1024x1024x8 @4nm, Lorentzian coupling", [inst], "dp45", 1e-13, 5e-9)


def disk_vortex():
    """Gradient workload: Permalloy disk of 200 nm diameter, 128x128x4 cells of
    2 nm, seeded vortex, alpha 0.02, Ms map U[7.5e5, 8.5e5] inside the disk,
    g/2pi = 200 MHz, omega_c/2pi = 1.3 GHz (near the gyrotropic mode of this
    disk, an estimate), kappa/2pi = 10 MHz, RK4 dt = 5e-14 s.  Returns
    (instance, Ms map, initial m)."""
    nx, ny, nz, d = 128, 128, 4, 2e-9
    inst = Instance(nx, ny, nz, d, Ms=8e5, Aex=1.3e-11, alpha=0.02, bias=(0.0, 0.0, 0.0),
                    omega_c=_twopi(1.3e9), kappa=_twopi(10e6), g=_twopi(200e6), seed=derive_seed(4, 0))
    ms = disk_ms(nx, ny, nz, d, d, 200e-9, 1.0) * uniform_ms_map(nx * ny * nz, derive_seed(4, 1), 7.5e5, 8.5e5)
    m0, _, _ = vortex_m(nx, ny, nz, d, d, derive_seed(4, 2))
    m0[ms <= 0] = 0.0
    return inst, ms.astype(np.float32), m0


def scaled(inst: Instance, nx: int, ny: int, nz: int) -> Instance:
    """Same material and cavity on another grid (parity tests at reduced size)."""
    return replace(inst, nx=nx, ny=ny, nz=nz)
