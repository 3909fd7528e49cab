"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA-side tests / bench.

This module holds no arithmetic of the method: only grid descriptors (sizes, spacings,
wave speed, boundary kinds), seeded Gaussian pulse lists and seeded probe nodes.  The enum
values mirror the C-ABI header ``include/lbw.h`` (the interface, not an implementation).

Workloads (the paper's examples are synthetic analytic geometries, Sec. IV; no dataset):
  disk      2-D polar annulus 128 x 128, FP64, 4000 steps, 1 off-centre pulse, 4 probes
  cylinder  3-D cylinder 128(r) x 128(theta) x 256(z), FP32, 20k steps, 8 random-phase
            pulses, 16 probes, Dirichlet caps
  trumpet   exponential-flare horn 256 x 256 x 512, 16-bit storage vs FP32, 50k steps,
            32 probes
  torus     192(r) x 1024(theta, major) x 256(phi, minor), R / a = 3, FP32 and BF16
            storage, 50k steps, 64 probes
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

KIND_CARTESIAN, KIND_POLAR, KIND_CYLINDRICAL, KIND_TRUMPET, KIND_TOROIDAL = range(5)
BC_PERIODIC, BC_BOUNCE, BC_ANTIBOUNCE, BC_FREE = range(4)
PREC_F64, PREC_F32, PREC_F16S, PREC_BF16S = range(4)
PROFILE_BESSEL, PROFILE_EXP = 0, 1
GEOM_AUTO, GEOM_TABLE, GEOM_ANALYTIC = range(3)
EQ_CURVILINEAR, EQ_MOMENT_MATCHING, EQ_HERMITE = range(3)

# Azimuthal lattice speed c / (r h_theta) allowed at the innermost node.  The step operator
# of every workload kind stays neutrally stable there at c = 0.4 (oracle eigenvalue pins);
# the inner radius r_in follows from it.
KAPPA_THETA = 1.0
WAVE_SPEED = 0.4


@dataclass(frozen=True)
class GridSpec:
    kind: int
    n: tuple
    h: tuple
    x0: tuple
    c: float
    cs2: float = 0.25
    damping: float = 1.0
    geom: tuple = (0.0, 0.0, 0.0, 0.0)
    profile: int = 0
    bc: tuple = (BC_PERIODIC,) * 6
    prec: int = PREC_F64
    geom_mode: int = 0  # lbw_geom_mode of include/lbw.h (the oracle always evaluates the metric)
    equilibrium: int = 0  # lbw_equilibrium: 0 the paper's method, 1 / 2 the Cartesian schemes

    @property
    def nodes(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])

    def with_(self, **kw) -> "GridSpec":
        return replace(self, **kw)


def r_inner(c: float, n_theta: int, kappa: float = KAPPA_THETA) -> float:
    """Smallest whole inner radius whose first node (r_in + 1/2) has an azimuthal lattice
    speed c / (r h_theta) <= kappa."""
    return float(max(1, math.ceil(c / (kappa * (2.0 * math.pi / n_theta)) - 0.5)))


def disk(n_r=128, n_theta=128, c=WAVE_SPEED, prec=PREC_F64) -> GridSpec:
    r_in = r_inner(c, n_theta)
    return GridSpec(kind=KIND_POLAR, n=(n_r, n_theta, 1), h=(1.0, 2 * math.pi / n_theta, 1.0),
                    x0=(r_in, 0.0, 0.0), c=c,
                    bc=(BC_BOUNCE, BC_ANTIBOUNCE, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC,
                        BC_PERIODIC), prec=prec)


def cylinder(n_r=128, n_theta=128, n_z=256, c=WAVE_SPEED, prec=PREC_F32) -> GridSpec:
    r_in = r_inner(c, n_theta)
    return GridSpec(kind=KIND_CYLINDRICAL, n=(n_r, n_theta, n_z),
                    h=(1.0, 2 * math.pi / n_theta, 1.0), x0=(r_in, 0.0, 0.0), c=c,
                    bc=(BC_BOUNCE, BC_ANTIBOUNCE, BC_PERIODIC, BC_PERIODIC, BC_ANTIBOUNCE,
                        BC_ANTIBOUNCE), prec=prec)


def trumpet_params(seed: int, n_r: int, n_z: int):
    """Seeded exponential flare a(z) = a0 + b e^{alpha z}: a0/n_r in [0.6, 0.9],
    b/n_r in [0.05, 0.2], alpha set so that a(L)/a(0) is in [1.5, 4]."""
    rng = np.random.default_rng(seed)
    a0 = rng.uniform(0.6, 0.9) * n_r
    b = rng.uniform(0.05, 0.2) * n_r
    ratio = rng.uniform(1.5, 4.0)
    # a(L) = ratio * (a0 + b)  ->  e^{alpha L} = (ratio (a0 + b) - a0) / b
    alpha = math.log((ratio * (a0 + b) - a0) / b) / n_z
    return a0, b, alpha


def trumpet(n_r=256, n_theta=256, n_z=512, c=WAVE_SPEED, seed=3, prec=PREC_F32) -> GridSpec:
    r_in = r_inner(c, n_theta)
    a0, b, alpha = trumpet_params(seed, n_r, n_z)
    return GridSpec(kind=KIND_TRUMPET, n=(n_r, n_theta, n_z),
                    h=(1.0, 2 * math.pi / n_theta, 1.0), x0=(r_in, 0.0, 0.0), c=c,
                    geom=(a0, b, alpha, 0.0), profile=PROFILE_EXP,
                    bc=(BC_BOUNCE, BC_BOUNCE, BC_PERIODIC, BC_PERIODIC, BC_BOUNCE, BC_BOUNCE),
                    prec=prec)


def bessel_horn(lam: float, n=(3, 4, 64), z_gap: float = 12.0, c: float = WAVE_SPEED,
                prec=PREC_F64) -> GridSpec:
    """The paper's Bessel horn s = (Zmax - z)^-lam over 0 < z < n3, Zmax = n3 + z_gap, rigid
    walls and rigid ends (lam = 0 is the straight pipe).  The radial spacing h_r = 1 / s_min
    keeps the physical cell at least one unit wide where the horn is narrowest; r_in keeps the
    azimuthal lattice speed c / (r s h_theta) <= KAPPA_THETA there and the ghost node half a
    cell inside the inner wall at r > 0."""
    n1, n2, n3 = n
    zmax = n3 + z_gap
    s_min = zmax ** -lam
    h_r = 1.0 / s_min
    r_in = float(max(math.ceil(h_r), math.ceil(c / (KAPPA_THETA * s_min * 2 * math.pi / n2) - 0.5 * h_r)))
    return GridSpec(kind=KIND_TRUMPET, n=tuple(n), h=(h_r, 2 * math.pi / n2, 1.0),
                    x0=(r_in, 0.0, 0.0), c=c, geom=(zmax, lam, 0.0, 0.0), profile=PROFILE_BESSEL,
                    bc=(BC_BOUNCE, BC_BOUNCE, BC_PERIODIC, BC_PERIODIC, BC_BOUNCE, BC_BOUNCE),
                    prec=prec)


def torus(n_r=192, n_theta=1024, n_phi=256, c=WAVE_SPEED, prec=PREC_F32) -> GridSpec:
    r_in = r_inner(c, n_phi)
    a = r_in + n_r
    R = 3.0 * a
    return GridSpec(kind=KIND_TOROIDAL, n=(n_r, n_theta, n_phi),
                    h=(1.0, 2 * math.pi / n_theta, 2 * math.pi / n_phi), x0=(r_in, 0.0, 0.0),
                    c=c, geom=(R, 0.0, 0.0, 0.0),
                    bc=(BC_BOUNCE, BC_BOUNCE, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC,
                        BC_PERIODIC), prec=prec)


def node_coords(spec: GridSpec, q1, q2, q3):
    """Physical coordinates (u1, u2, u3) of lattice node q: x0 + (q + 1/2) h."""
    return tuple(spec.x0[a] + (q + 0.5) * spec.h[a] for a, q in enumerate((q1, q2, q3)))


def embedding(spec: GridSpec, u1, u2, u3):
    """Cartesian position of physical coordinates, used only to place pulses."""
    k = spec.kind
    if k == KIND_CARTESIAN:
        return np.array([u1, u2, u3])
    if k in (KIND_POLAR, KIND_CYLINDRICAL):
        return np.array([u1 * math.cos(u2), u1 * math.sin(u2), u3])
    if k == KIND_TRUMPET:
        if spec.profile == PROFILE_BESSEL:
            s = (spec.geom[0] - u3) ** (-spec.geom[1])
        else:
            a0, b, al = spec.geom[:3]
            s = (a0 + b * math.exp(al * u3)) / (a0 + b)
        return np.array([u1 * s * math.cos(u2), u1 * s * math.sin(u2), u3])
    R = spec.geom[0]
    return np.array([(R + u1 * math.cos(u3)) * math.cos(u2),
                     (R + u1 * math.cos(u3)) * math.sin(u2), u1 * math.sin(u3)])


def _interior_node(rng, spec: GridSpec, margin: int):
    q = []
    for a in range(3):
        n = spec.n[a]
        lo, hi = (margin, n - margin) if n > 2 * margin else (0, n)
        q.append(int(rng.integers(lo, hi)))
    return q


def pulses(spec: GridSpec, seed: int, count: int = 1, sigma: float = 3.0,
           random_phase: bool = False, margin: int = 8) -> np.ndarray:
    """count x (X, Y, Z, sigma, amp): Gaussian centres at seeded interior nodes.  With
    random_phase, amplitude cos(phi_k) with phi_k ~ U[0, 2 pi)."""
    rng = np.random.default_rng(seed)
    out = np.zeros((count, 5))
    for k in range(count):
        q = _interior_node(rng, spec, margin)
        X = embedding(spec, *node_coords(spec, *q))
        amp = math.cos(rng.uniform(0.0, 2.0 * math.pi)) if random_phase else 1.0
        out[k] = (X[0], X[1], X[2], sigma, amp)
    return out


def probes(spec: GridSpec, seed: int, count: int, margin: int = 2) -> np.ndarray:
    """count x (q1, q2, q3) seeded interior probe nodes (int32)."""
    rng = np.random.default_rng(seed + 1000)
    return np.array([_interior_node(rng, spec, margin) for _ in range(count)], dtype=np.int32)


@dataclass
class Workload:
    name: str
    spec: GridSpec
    steps: int
    pulses: np.ndarray
    probes: np.ndarray
    notes: str = ""
    extra: dict = field(default_factory=dict)


def workload(name: str, shape=None) -> Workload:
    """A benchmark workload; `shape` = (n1, n2, n3) resizes its lattice (same kind, wave speed,
    faces and seeds; the inner radius and the torus's R follow the new sizes as they do for the
    default), which serves smaller profiling captures of the same kernels."""
    if name == "disk":
        n = shape or (128, 128, 1)
        s = disk(n[0], n[1])
        return Workload("disk", s, 4000, pulses(s, 1, 1), probes(s, 1, 4),
                        f"2-D polar annulus r {n[0]} x theta {n[1]}")
    if name == "cylinder":
        n = shape or (128, 128, 256)
        s = cylinder(*n)
        return Workload("cylinder", s, 20000, pulses(s, 2, 8, random_phase=True),
                        probes(s, 2, 16), f"cylinder r {n[0]} x theta {n[1]} x z {n[2]}")
    if name == "trumpet":
        n = shape or (256, 256, 512)
        s = trumpet(*n)
        return Workload("trumpet", s, 50000, pulses(s, 3, 1), probes(s, 3, 32),
                        f"exponential-flare trumpet r {n[0]} x theta {n[1]} x z {n[2]}")
    if name == "torus":
        n = shape or (192, 1024, 256)
        s = torus(*n)
        return Workload("torus", s, 50000, pulses(s, 4, 1), probes(s, 4, 64),
                        f"torus r {n[0]} x theta (major) {n[1]} x phi (minor) {n[2]}, R/a = 3")
    raise KeyError(name)


def ensemble_member(n_r: int, n_theta: int, n_z: int, a0: float, b: float, alpha: float,
                    c: float = WAVE_SPEED, prec: int = PREC_F32) -> GridSpec:
    """One exponential-flare trumpet of the ensemble: rigid walls and rigid ends (halfway
    bounce-back, D = 1) for clean normal modes."""
    r_in = r_inner(c, n_theta)
    return GridSpec(kind=KIND_TRUMPET, n=(n_r, n_theta, n_z),
                    h=(1.0, 2 * math.pi / n_theta, 1.0), x0=(r_in, 0.0, 0.0), c=c,
                    geom=(a0, b, alpha, 0.0), profile=PROFILE_EXP,
                    bc=(BC_BOUNCE, BC_BOUNCE, BC_PERIODIC, BC_PERIODIC, BC_BOUNCE, BC_BOUNCE),
                    prec=prec)


def ensemble(n: int, seed: int = 5, r_range=(32, 96), theta_range=(32, 96), z_range=(128, 512),
             prec: int = PREC_F32):
    """n seeded trumpets of uneven sizes (uniform integer sizes in the given ranges) and
    seeded flares.  Returns (specs, params) with params[m] = (n_r, n_theta, n_z, a0, b, alpha)."""
    rng = np.random.default_rng(seed)
    specs, params = [], []
    for _ in range(n):
        n_r = int(rng.integers(r_range[0], r_range[1] + 1))
        n_t = int(rng.integers(theta_range[0], theta_range[1] + 1))
        n_z = int(rng.integers(z_range[0], z_range[1] + 1))
        a0, b, alpha = trumpet_params(int(rng.integers(1 << 30)), n_r, n_z)
        specs.append(ensemble_member(n_r, n_t, n_z, a0, b, alpha, prec=prec))
        params.append((n_r, n_t, n_z, a0, b, alpha))
    return specs, params


def ensemble_excitation(spec: GridSpec, sigma: float = 3.0, n_ring: int = 12):
    """Pulses and probes at fixed relative positions of a member, so its spectrum depends on
    its geometry only.  A ring of n_ring Gaussian pulses next to the rigid outer wall at the
    q3 = 0 end (nodes (n1 - 2, j n2 / n_ring, 1)) excites axisymmetric modes (azimuthal orders
    that are multiples of n_ring aside); 8 probes on a ring at the opposite corner
    (n1 - 1, j n2 / 8, n3 - 1) record them.  With rigid walls and ends every axisymmetric mode
    has an antinode at both corners, so the summed probes see each mode without the
    cancellations that scattered probes suffer."""
    n1, n2, n3 = spec.n
    pulse = []
    for j in range(n_ring):
        X = embedding(spec, *node_coords(spec, n1 - 2, j * n2 / n_ring, 1))
        pulse.append([X[0], X[1], X[2], sigma, 1.0])
    pr = np.array([[n1 - 1, (j * n2) // 8, n3 - 1] for j in range(8)], dtype=np.int32)
    return np.array(pulse), pr
