"""Seeded synthetic workloads: the five configurations the library is measured on.

Each builder returns a :class:`synth.problem.Problem` plus the run length.  The
readings of unstated details are fixed here once, as data:

* perfusion is given as a volumetric rate omega_b [1/s]; the paper's Eq. 1 uses
  w_b in kg/(m^3 s), so w_b = omega_b * rho_b with rho_b = 1060 kg/m^3;
* a Gaussian source's stated value is its peak density at the centre (W/m^3);
* "Dirichlet on the surface" of a voxel ellipsoid means every node of a voxel
  face that is not shared by two inside voxels.

Only random draws, unit conversions and node/face selections happen here.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np

from .meshes import (box_face_nodes, ellipsoid_node_count, hex_box, hex_box_top_faces,
                     tet_ellipsoid)
from .problem import GaussianSource, Material, Perfusion, Problem

RHO_BLOOD = 1060.0            # kg/m^3, converts omega_b [1/s] to w_b [kg/(m^3 s)]
OMEGA_B = 0.0064              # 1/s
C_BLOOD = 3600.0              # J/(kg K)
T_ARTERIAL = 37.0

# constant tissue of the 10 mm cube
TISSUE_CONST = Material.constant(rho=1060.0, c=3600.0, k=0.512)
# k(T) = 0.512 (1 + 0.00161 (T - 37)),  c(T) = 3600 (1 - 0.0015 (T - 37)),  rho constant
TISSUE_TD = Material(T_ref=37.0, rho0=1060.0, drho=0.0,
                     c0=3600.0, dc=-3600.0 * 0.0015,
                     k0=0.512, dk=0.512 * 0.00161)
PERFUSION = Perfusion(w_b=OMEGA_B * RHO_BLOOD, c_b=C_BLOOD, T_a=T_ARTERIAL, Q_m=0.0)

ELLIPSOID_AXES = (0.060, 0.045, 0.035)
ELLIPSOID_SEED = 1909050982


@dataclass
class Workload:
    name: str
    problem: Problem
    n_steps: int
    dt_fraction: float = 0.5   # dt = dt_fraction * critical step


def cube_hex_fp64(n: int = 10, h: float = 1e-3, n_steps: int = 2000) -> Workload:
    """10 x 10 x 10 mm cube of 10^3 hex8 elements (1331 nodes), constant
    properties, perfusion, Dirichlet 37 degC on all six faces, a Gaussian source
    (sigma 1.5 mm, 5e6 W/m^3) at the centre, dt = 0.5 critical, 2000 steps."""
    m = hex_box(n, n, n, h)
    dn = box_face_nodes(m)
    L = n * h
    prob = Problem(8, m.xyz, m.conn, TISSUE_CONST, PERFUSION,
                   sources=[GaussianSource((L / 2, L / 2, L / 2), 1.5e-3, 5e6)],
                   dirichlet_nodes=dn, dirichlet_T=np.full(len(dn), 37.0),
                   T0=37.0, T_lo=30.0, T_hi=100.0)
    return Workload(f"hex cube {n}^3 elements, h={h*1e3:g} mm, constant properties", prob, n_steps)


def _sample_sources(rng, axes, count, sigma_range=(2e-3, 5e-3), peak_range=(1e6, 1e7)):
    """Sources with sigma ~ U[sigma_range], peak ~ U[peak_range] and a centre
    uniform inside the ellipsoid shrunk by 2 sigma (rejection sampling); on
    small ellipsoids each semi-axis keeps at least a quarter of its length."""
    out = []
    a = np.asarray(axes)
    while len(out) < count:
        sigma = rng.uniform(*sigma_range)
        peak = rng.uniform(*peak_range)
        inner = np.maximum(a - 2 * sigma, 0.25 * a)
        while True:
            x = rng.uniform(-inner, inner)
            if np.sum((x / inner) ** 2) <= 1.0:
                break
        out.append(GaussianSource(tuple(float(v) for v in x), float(sigma), float(peak)))
    return out


def ellipsoid_tet_td(h: float = 1e-3, axes=ELLIPSOID_AXES, seed: int = ELLIPSOID_SEED,
                     n_sources: int = 3, n_steps: int = 20000, T_hi: float = 400.0) -> Workload:
    """Jittered Kuhn-tet ellipsoid (semi-axes 60/45/35 mm, voxel h, jitter 0.2 h),
    temperature-dependent k and c, three seeded Gaussian sources, perfusion,
    Dirichlet 37 degC on the surface, 2e4 steps."""
    m = tet_ellipsoid(axes, h, 0.2 * h, seed)
    rng = np.random.default_rng(seed + 1)
    src = _sample_sources(rng, axes, n_sources)
    dn = m.surface_nodes
    prob = Problem(4, m.xyz, m.conn, TISSUE_TD, PERFUSION, sources=src,
                   dirichlet_nodes=dn, dirichlet_T=np.full(len(dn), 37.0),
                   T0=37.0, T_lo=25.0, T_hi=T_hi)
    return Workload(f"tet4 ellipsoid {axes[0]*1e3:g}/{axes[1]*1e3:g}/{axes[2]*1e3:g} mm, h={h*1e3:g} mm, "
                    f"T-dependent k,c", prob, n_steps)


def cube_hex_td_convective(n: int = 128, h: float = 1e-3, n_steps: int = 10000) -> Workload:
    """n^3 hex8 cube (128^3: 2,146,689 nodes, 2,097,152 elements), the
    temperature-dependent laws of the ellipsoid, perfusion, a centred Gaussian
    source (sigma 1.5 mm, 5e6 W/m^3), a film condition h = 10 W/(m^2 K) at
    25 degC on the z = max face and Dirichlet 37 degC on the other five faces."""
    m = hex_box(n, n, n, h)
    dn = box_face_nodes(m, ("x0", "x1", "y0", "y1", "z0"))
    L = n * h
    prob = Problem(8, m.xyz, m.conn, TISSUE_TD, PERFUSION,
                   sources=[GaussianSource((L / 2, L / 2, L / 2), 1.5e-3, 5e6)],
                   dirichlet_nodes=dn, dirichlet_T=np.full(len(dn), 37.0),
                   conv_faces=hex_box_top_faces(n, n, n), conv_h=10.0, conv_T_inf=25.0,
                   T0=37.0, T_lo=20.0, T_hi=100.0)
    return Workload(f"hex cube {n}^3 elements, h={h*1e3:g} mm, T-dependent k,c, convective top face",
                    prob, n_steps)


# the six mesh densities (nodes, tetrahedra) of the paper's timing study
# (Section 3.2, Fig. 8 and Table 6)
PAPER_TIMING_SIZES = ((1445, 6738), (1840, 8724), (2644, 12852), (3339, 16371), (5304, 26550), (7872, 40021))


def paper_size_ellipsoid(target_nodes: int, temperature_dependent: bool = True, h: float = 1e-3,
                         seed: int = ELLIPSOID_SEED) -> Workload:
    """The ellipsoid recipe (jittered Kuhn tets, three seeded sources,
    perfusion) with its 60/45/35 mm shape scaled until the node count is the
    first one at or above target_nodes; temperature-dependent k, c or the
    constant tissue values.  Like the paper's liver, only the bottom is held
    at 37 degC: the surface nodes below half the short semi-axis under the
    centre; the rest of the surface is insulated.  The paper's timing study
    runs 2000 steps of 0.005 s."""
    shape = np.asarray(ELLIPSOID_AXES)
    lo, hi = 0.01, 1.5
    for _ in range(30):   # bisection on the node count
        s = 0.5 * (lo + hi)
        if ellipsoid_node_count(shape * s, h) < target_nodes:
            lo = s
        else:
            hi = s
    axes = tuple(float(v) for v in shape * hi)
    m = tet_ellipsoid(axes, h, 0.2 * h, seed)
    rng = np.random.default_rng(seed + 1)
    src = _sample_sources(rng, axes, 3)
    z = m.xyz[m.surface_nodes, 2]
    zc = 0.5 * (m.xyz[:, 2].min() + m.xyz[:, 2].max())
    dn = m.surface_nodes[z < zc - 0.5 * axes[2]]
    mat = TISSUE_TD if temperature_dependent else TISSUE_CONST
    prob = Problem(4, m.xyz, m.conn, mat, PERFUSION, sources=src,
                   dirichlet_nodes=dn, dirichlet_T=np.full(len(dn), 37.0),
                   T0=37.0, T_lo=25.0, T_hi=400.0)
    return Workload(f"tet4 ellipsoid scaled to {len(m.xyz)} nodes, {'TD' if temperature_dependent else 'TI'}",
                    prob, 2000)


@dataclass
class PlanningMesh:
    seed: int
    target_nodes: int
    problems: List[Problem]    # one Problem per scenario; the mesh is shared


def planning_batch(n_meshes: int = 64, n_scenarios: int = 4, n_range=(5_000, 200_000),
                   h: float = 1e-3, base_seed: int = 0) -> List[PlanningMesh]:
    """Uneven ellipsoid tet meshes (node counts log-uniform in n_range), each
    with n_scenarios single-source scenarios (sigma U[2,5] mm, peak U[1e6,1e7]
    W/m^3, centre uniform inside), T-dependent properties."""
    out = []
    for m_i in range(n_meshes):
        seed = base_seed + m_i
        rng = np.random.default_rng(seed)
        target = int(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1]))))
        shape = np.asarray(ELLIPSOID_AXES) * (1.0 + rng.uniform(-0.2, 0.2, 3))
        lo, hi = 0.01, 1.5
        for _ in range(22):   # bisection on the node count
            s = 0.5 * (lo + hi)
            if ellipsoid_node_count(shape * s, h) < target:
                lo = s
            else:
                hi = s
        axes = tuple(float(v) for v in shape * hi)
        m = tet_ellipsoid(axes, h, 0.2 * h, seed)
        dn = m.surface_nodes
        probs = []
        for s_i in range(n_scenarios):
            src = _sample_sources(rng, axes, 1)
            probs.append(Problem(4, m.xyz, m.conn, TISSUE_TD, PERFUSION, sources=src,
                                 dirichlet_nodes=dn, dirichlet_T=np.full(len(dn), 37.0),
                                 T0=37.0, T_lo=25.0, T_hi=400.0))
        out.append(PlanningMesh(seed, target, probs))
    return out


def surrogate_sources(n: int, seed: int, cube_mm: float = 10.0, inner_mm: float = 6.0,
                      sigma_range=(1e-3, 3e-3), peak_range=(1e6, 1e7)) -> List[GaussianSource]:
    """Training / evaluation scenarios of the surrogate on the 10 mm cube: one
    source per scenario, centre uniform in the central 6 mm cube, sigma
    U[1, 3] mm, peak U[1e6, 1e7] W/m^3."""
    rng = np.random.default_rng(seed)
    lo = (cube_mm - inner_mm) / 2e3
    out = []
    for _ in range(n):
        x0 = tuple(float(v) for v in rng.uniform(lo, lo + inner_mm / 1e3, 3))
        out.append(GaussianSource(x0, float(rng.uniform(*sigma_range)), float(rng.uniform(*peak_range))))
    return out


def source_density(xyz: np.ndarray, sources: List[GaussianSource]) -> np.ndarray:
    """Nodal source densities (W/m^3), one row per scenario -- the input field
    the scenario prescribes."""
    q = np.zeros((len(sources), len(xyz)))
    for i, s in enumerate(sources):
        q[i] = s.peak * np.exp(-np.sum((xyz - np.asarray(s.x0)) ** 2, axis=1) / (2.0 * s.sigma ** 2))
    return q
