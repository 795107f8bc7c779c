"""Plain data containers that describe one Pennes bio-heat problem.

These hold the inputs named in the problem statement of the paper (Section 2.1,
Eq. 1-5): the mesh, the tissue material laws, blood perfusion, metabolic and
regional heat sources, and the three kinds of boundary condition.  No part of
the method's arithmetic lives here; both the CPU oracle and the CUDA library
receive exactly these arrays.

Units are SI with temperatures in degrees Celsius.  ``w_b`` is the blood
perfusion rate in kg/(m^3 s), the unit the paper uses in Eq. 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

HEX8 = 8
TET4 = 4


@dataclass(frozen=True)
class Material:
    """Linear temperature laws p(T) = p0 + dp * (T - T_ref) for rho, c and k.

    Constant properties (Eq. 1) are the special case drho = dc = dk = 0;
    temperature-dependent properties (Eq. 2, Section 3.1.6) use the slopes.
    """
    T_ref: float
    rho0: float
    drho: float
    c0: float
    dc: float
    k0: float
    dk: float

    # Optional piecewise-linear tables (T_j, rho_j, c_j, k_j), T_j increasing,
    # linear inside each interval and along the end intervals beyond the table.
    # When set, T_ref/rho0/c0/k0 are the first point and the linear slopes unused.
    table: Optional[tuple] = None

    @staticmethod
    def constant(rho: float, c: float, k: float, T_ref: float = 37.0) -> "Material":
        return Material(T_ref, rho, 0.0, c, 0.0, k, 0.0)

    @staticmethod
    def tabulated(T, rho, c, k) -> "Material":
        """Piecewise-linear laws through the points (T_j, rho_j), (T_j, c_j), (T_j, k_j)."""
        T, rho, c, k = (tuple(float(v) for v in a) for a in (T, rho, c, k))
        if not (2 <= len(T) <= 8 and len(rho) == len(c) == len(k) == len(T)):
            raise ValueError("2 to 8 points, one value of each property per point")
        if any(b <= a for a, b in zip(T, T[1:])):
            raise ValueError("table temperatures must increase")
        return Material(T[0], rho[0], 0.0, c[0], 0.0, k[0], 0.0, table=(T, rho, c, k))

    @staticmethod
    def from_two_points(T1: float, T2: float, rho: tuple, c: tuple, k: tuple) -> "Material":
        """Linear interpolation between property values given at T1 and T2
        (the form of Section 3.1.6: values at 37 and 65 degC)."""
        span = T2 - T1
        return Material(T1, rho[0], (rho[1] - rho[0]) / span,
                        c[0], (c[1] - c[0]) / span,
                        k[0], (k[1] - k[0]) / span)


@dataclass(frozen=True)
class Perfusion:
    """Pennes perfusion and metabolic terms of Eq. 1: w_b [kg/(m^3 s)],
    c_b [J/(kg K)], arterial T_a [degC], metabolic Q_m [W/m^3]."""
    w_b: float = 0.0
    c_b: float = 0.0
    T_a: float = 37.0
    Q_m: float = 0.0


@dataclass(frozen=True)
class GaussianSource:
    """Regional source Q_r(x) = peak * exp(-|x - x0|^2 / (2 sigma^2)) in W/m^3."""
    x0: tuple
    sigma: float
    peak: float


@dataclass
class Problem:
    elem_type: int                       # 8 (hex8, one-point) or 4 (tet4)
    xyz: np.ndarray                      # (N, 3) float64, metres
    conn: np.ndarray                     # (E, elem_type) int32, 0-based node ids
    material: Material
    perfusion: Perfusion = field(default_factory=Perfusion)
    sources: List[GaussianSource] = field(default_factory=list)
    q_r: Optional[np.ndarray] = None     # (N,) extra source density at nodes, W/m^3
    dirichlet_nodes: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    dirichlet_T: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    conv_faces: np.ndarray = field(default_factory=lambda: np.zeros((0, 4), np.int32))
    conv_h: float = 0.0                  # film coefficient, W/(m^2 K)
    conv_T_inf: float = 0.0              # ambient temperature, degC
    flux_nodes: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    flux_q: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))  # W per node
    T0: float | np.ndarray = 37.0
    T_lo: float = 0.0                    # declared admissible temperature range
    T_hi: float = 100.0
    # time-varying regional sources (Algorithm 1 updates the loads every step):
    # the regional source density is multiplied by schedule_factor[k] while the
    # step's start time t lies in [schedule_end[k-1], schedule_end[k]); after the
    # last end the last factor holds.  Empty: sources always on.
    schedule_end: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    schedule_factor: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    # heterogeneous tissue: element e takes region_materials[regions[e]] and the
    # w_b, c_b, Q_m of region_perfusion[regions[e]] (T_a stays perfusion.T_a);
    # None: material and perfusion everywhere
    regions: Optional[np.ndarray] = None
    region_materials: tuple = ()
    region_perfusion: tuple = ()
    # hex8 integration: "one-point" (Eq. 14, the paper's), "full" (2 x 2 x 2 Gauss) or
    # "hourglass" (one point plus hourglass stabilisation of strength hourglass_eps)
    hex_rule: str = "one-point"
    hourglass_eps: float = 0.0
    # perfusion and metabolic heat per node: "element" (V_e / nv shares, as C)
    # or "uniform" (V / N for every node, the paper's verification runs)
    lumping: str = "element"
    uniform_volume_per_node: Optional[float] = None   # V / N of the whole mesh (for sub-meshes); None: this mesh's

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.conn.shape[0])

    def T0_array(self) -> np.ndarray:
        """The initial field as given, broadcast to one value per node."""
        T0 = np.asarray(self.T0, dtype=np.float64)
        if T0.ndim == 0:
            return np.full(self.n_nodes, float(T0))
        return T0.copy()
