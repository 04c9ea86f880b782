"""Seeded synthetic workloads: model systems shaped like the paper's 1D He and
linear H3+ (Sec. 3.1, 3.2), and random symmetric test matrices.

This module holds no arithmetic of the method itself: it only draws the
parameters (nuclear charges and positions, box, grid sizes, mesh parameters)
and random matrices. Both the CUDA library's tests/benchmarks and the CPU
oracle take their inputs from here; neither the library nor the oracle imports
the other.

Seeds: a per-system stream is splitmix64(master ^ config_id ^ system_id),
master = 9114348, drawn on the host.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MASTER_SEED = 9114348
_MASK = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One output of the SplitMix64 generator (Steele, Lea, Flood 2014)."""
    x = (x + 0x9E3779B97F4A7C15) & _MASK
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def system_rng(config_id: int, system_id: int = 0) -> np.random.Generator:
    """numpy Generator seeded from splitmix64(master ^ config_id ^ system_id)."""
    seed = splitmix64(MASTER_SEED ^ (int(config_id) << 32) ^ int(system_id))
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class System:
    """One model system: box, FE grid, nuclei, soft-Coulomb parameters,
    electron count, inverse temperature and power-mesh parameters."""
    name: str
    xmin: float
    xmax: float
    n_elem: int
    order: int            # polynomial order n_g; order + 1 GLL points per element
    Z: list = field(default_factory=list)
    R: list = field(default_factory=list)
    soft_en: float = 1.0
    soft_ee: float = 1.0
    n_elec: int = 2
    beta: float = 100.0
    u: int = 4
    p: int = 16
    grid_kind: int = 0
    mixing: float = 0.5
    tol: float = 1e-8

    @property
    def pts_per_elem(self) -> int:
        """GLL points per element, order + 1 (the library's build_fedvr argument)."""
        return self.order + 1

    @property
    def n_b(self) -> int:
        """Matrix dimension n_e * order - 1 (both box ends clamped)."""
        return self.n_elem * self.order - 1

    @property
    def n_tau(self) -> int:
        return 2 * self.u * self.p + 1


def he_small() -> System:
    """1D He, Z=2, box [-10,10], 4 elements x 5 GLL points (order 4, n_b=15),
    beta=100, 129-point mesh (u=4, p=16)."""
    return System("He n_b=15 M=129", -10.0, 10.0, 4, 4, [2.0], [0.0], u=4, p=16)


def he_medium() -> System:
    """1D He, box [-50,50], 25 elements x 9 GLL points (order 8, n_b=199),
    beta=100, 513-point mesh (u=16, p=16)."""
    return System("He n_b=199 M=513", -50.0, 50.0, 25, 8, [2.0], [0.0], u=16, p=16)


def he_paper() -> System:
    """The paper's second-Born He run (Sec. 3.1): graded (case II) grid of 29
    elements of order 7 over 200 a.u. (n_b=202), beta=100, 1025-point mesh
    (u=32, p=16)."""
    return System("He case II n_b=202 M=1025", -100.0, 100.0, 29, 7, [2.0], [0.0], u=32, p=16,
                  grid_kind=1)


def h3p_large(system_id: int = 0) -> System:
    """Linear H3+: unit charges at (-R, 0, R), R = 1.8, each nucleus shifted by
    an independent U(-0.1, 0.1) jitter; box [-60,60], 30 elements x 11 GLL
    points (order 10, n_b=299), beta=100, 1025-point mesh (u=32, p=16)."""
    rng = system_rng(3, system_id)
    jit = rng.uniform(-0.1, 0.1, size=3)
    R = [-1.8 + jit[0], 0.0 + jit[1], 1.8 + jit[2]]
    return System("H3+ n_b=299 M=1025", -60.0, 60.0, 30, 10, [1.0, 1.0, 1.0], R, u=32, p=16)


def h3p_curve(Rs=None) -> list[System]:
    """The paper's H3+ binding-curve grid (Sec. 3.2): 13 graded (case II)
    elements of order 11 over a 50 a.u. interval (n_b = 142), beta = 100,
    1025-point mesh (u = 32, p = 16); symmetric unit nuclei at (-R, 0, R) for
    each R (default 1.6, 1.8, ..., 3.6, i.e. outer distance d = 2R from 3.2 to
    7.2)."""
    if Rs is None:
        Rs = [1.6 + 0.2 * k for k in range(11)]
    return [System(f"H3+ R={R:.3f}", -25.0, 25.0, 13, 11, [1.0, 1.0, 1.0], [-R, 0.0, R], u=32,
                   p=16, grid_kind=1) for R in Rs]


def batch_systems(count: int = 64, config_id: int = 4) -> list[System]:
    """Uneven batch: half He (Z ~ U[1.5,2.5], box [-50,50]), half H3+
    (R ~ U[1.2,3.0], box [-60,60]); order ~ U{4..10},
    n_e ~ U[ceil(60/order), floor(240/order)], u ~ U{8..16}, p = 16."""
    out = []
    for s in range(count):
        rng = system_rng(config_id, s)
        order = int(rng.integers(4, 11))
        lo, hi = -(-60 // order), 240 // order
        ne = int(rng.integers(lo, hi + 1))
        u = int(rng.integers(8, 17))
        if s % 2 == 0:
            Z = float(rng.uniform(1.5, 2.5))
            out.append(System(f"He#{s}", -50.0, 50.0, ne, order, [Z], [0.0], u=u, p=16))
        else:
            R = float(rng.uniform(1.2, 3.0))
            out.append(System(f"H3+#{s}", -60.0, 60.0, ne, order, [1.0, 1.0, 1.0],
                              [-R, 0.0, R], u=u, p=16))
    return out


def warmstart_system(system_id: int, config_id: int = 5) -> System:
    """Warm-start family: 20 elements x 7 GLL points (order 6, n_b=119),
    257-point mesh (u=8, p=16); even ids He (Z ~ U[1.5,2.5], box [-50,50]),
    odd ids H3+ (R ~ U[1.2,3.0], box [-60,60])."""
    rng = system_rng(config_id, system_id)
    if system_id % 2 == 0:
        Z = float(rng.uniform(1.5, 2.5))
        return System(f"He#{system_id}", -50.0, 50.0, 20, 6, [Z], [0.0], u=8, p=16)
    R = float(rng.uniform(1.2, 3.0))
    return System(f"H3+#{system_id}", -60.0, 60.0, 20, 6, [1.0, 1.0, 1.0], [-R, 0.0, R],
                  u=8, p=16)


@dataclass
class KbeRun:
    """A real-time propagation: the system (its HF ground state is the
    uncorrelated initial state), the time step, the number of steps and a
    dipole field E(t) = amp sin(omega t) sin^2(pi t / t_end) applied as the
    potential x_a E(t) at the nodes."""
    system: System
    dt: float
    n_steps: int
    amp: float
    omega: float

    def field(self) -> np.ndarray:
        """E(t_k) for k = 0 .. n_steps."""
        t = np.arange(self.n_steps + 1) * self.dt
        t_end = self.n_steps * self.dt
        return self.amp * np.sin(self.omega * t) * np.sin(np.pi * t / t_end) ** 2


def kbe_he(n_steps: int = 100) -> KbeRun:
    """1D He, Z=2, box [-15,15], 10 elements of order 4 (n_b = 39), driven from
    its HF ground state by a 0.1 a.u. field at omega = 0.9 Ha; dt = 0.04 keeps
    Heun's step stable (max|e| of h about 10 Ha)."""
    s = System("He n_b=39 (real time)", -15.0, 15.0, 10, 4, [2.0], [0.0])
    return KbeRun(s, 0.04, n_steps, 0.1, 0.9)


def random_symmetric(rng: np.random.Generator, n: int, scale: float = 1.0) -> np.ndarray:
    """Random symmetric n x n matrix with U(-scale, scale) entries."""
    a = rng.uniform(-scale, scale, size=(n, n))
    return 0.5 * (a + a.T)


def random_symmetric_stack(rng: np.random.Generator, m: int, n: int, scale: float = 1.0) -> np.ndarray:
    """m independent random symmetric n x n matrices."""
    a = rng.uniform(-scale, scale, size=(m, n, n))
    return 0.5 * (a + a.transpose(0, 2, 1))
