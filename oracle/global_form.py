"""Global assembled form of the FED-FEM step, Eq. 7-8 with lumped C (Section 2.3.4).

Oracle code (test infrastructure only).  Per time step (Algorithm 1, the
time-stepping block, taken in its global matrix form):

1. k at every node from the nodal temperature, k_e = mean of the element's
   nodal k (Eq. 13);
2. K = sum_e k_e A_e assembled into one global sparse matrix (Eq. 11);
3. C_i = V_i rho(T_i) c(T_i) (lumped, Section 2.3.4);
4. R = -K T + beta (T_a - T) + Q + hA (T_inf - T), beta_i = w_b c_b V_i
   (the pre-computed K_b and Q_b of Section 2.3.5 in difference form);
5. T <- T + dt R / C on free nodes (Eq. 8, Eq. 19); Dirichlet nodes keep
   their initial value (Eq. 3).

Material laws are linear in T (Section 3.1.6) or, optionally, piecewise
linear through tabulated points, extended linearly beyond the table.

Perfusion and metabolic heat may instead take the same share V / N at every
node (the form of the paper's verification runs, Sections 3.1.3-3.1.4); C
stays lumped by element shares.

Heterogeneous tissue (finite elements let the properties vary from element to
element, as the introduction notes): each element belongs to a region with its
own laws and perfusion.  Step 1 averages the element's own k law over its
nodes; the lumped C_i, beta_i and metabolic heat of node i become sums over
its elements of (V_e / nv) times the element's rho(T_i) c(T_i), w_b c_b and
Q_m.

Time-varying loads (the boundary/load update at the end of each step of
Algorithm 1; the two-stage heating and relaxation of Section 3.1.5): the
regional source part of Q is scaled by the schedule factor of the step's start
time, Q(t) = Q_const + f(t) Q_src.  Thermal dose (the treatment-planning use
named in Section 5; the paper gives no formula): cumulative equivalent minutes
at 43 degC (Sapareto and Dewey, 1984), CEM43 += (dt / 60) R^(43 - T), R = 1/2
for T >= 43 degC and 1/4 below, with T the node's temperature at the start of
the step.  Alternatively the Arrhenius damage integral (Henriques and
Moritz, 1947), Omega += dt A exp(-Ea / (R T_K)), at the same temperature.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .elements import element_matrices


def lumped_volumes(conn: np.ndarray, V_e: np.ndarray, n_nodes: int) -> np.ndarray:
    """V_i = sum over elements containing i of V_e / (nodes per element)."""
    nv = conn.shape[1]
    V = np.zeros(n_nodes)
    np.add.at(V, conn.ravel(), np.repeat(V_e / nv, nv))
    return V


def uniform_share(V_total: float, n_nodes: int) -> float:
    """The volume V / N that the paper's verification runs give every node
    (Sections 3.1.3-3.1.4: the film h and the nodal heat flow q per node)."""
    return V_total / n_nodes


def lumped_face_areas(xyz: np.ndarray, faces: np.ndarray, n_nodes: int) -> np.ndarray:
    """A_i = sum over boundary faces containing i of (face area) / (face nodes).

    Triangles: |(x1-x0) x (x2-x0)| / 2.  Quadrilaterals: |d1 x d2| / 2 with the
    two diagonals d1 = x2-x0, d2 = x3-x1 (exact for planar quadrilaterals)."""
    A = np.zeros(n_nodes)
    if len(faces) == 0:
        return A
    x = xyz[faces]
    if faces.shape[1] == 3:
        area = 0.5 * np.linalg.norm(np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), axis=1)
    elif faces.shape[1] == 4:
        area = 0.5 * np.linalg.norm(np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 1]), axis=1)
    else:
        raise ValueError("faces must have 3 or 4 nodes")
    np.add.at(A, faces.ravel(), np.repeat(area / faces.shape[1], faces.shape[1]))
    return A


def gaussian_density(xyz: np.ndarray, sources) -> np.ndarray:
    """Q_r(x_i) = sum_s peak_s exp(-|x_i - x0_s|^2 / (2 sigma_s^2)), W/m^3."""
    q = np.zeros(len(xyz))
    for s in sources:
        r2 = np.sum((xyz - np.asarray(s.x0)) ** 2, axis=1)
        q += s.peak * np.exp(-r2 / (2.0 * s.sigma ** 2))
    return q


class Oracle:
    """Plain FP64 global-matrix stepper for one :class:`synth.problem.Problem`."""

    def __init__(self, problem):
        p = problem
        self.p = p
        N = p.n_nodes
        self.N = N
        self.conn = np.asarray(p.conn, dtype=np.int64)
        self.A_e, self.det_e, self.V_e = element_matrices(p.elem_type, p.xyz, self.conn,
                                                          getattr(p, "hex_rule", "one-point"),
                                                          getattr(p, "hourglass_eps", 0.0))
        self.V = lumped_volumes(self.conn, self.V_e, N)
        self.hA = p.conv_h * lumped_face_areas(p.xyz, np.asarray(p.conv_faces, dtype=np.int64), N)
        lumping = getattr(p, "lumping", "element")
        if lumping == "uniform" and p.regions is not None:
            raise ValueError("uniform lumping takes one material")
        if p.regions is None and lumping == "uniform":
            # the paper's verification runs (Sections 3.1.3-3.1.4): every node
            # gets the same share V / N of the perfusion and the metabolic heat
            self.regions = None
            share = getattr(p, "uniform_volume_per_node", None)   # given for a sub-mesh of a larger mesh
            if share is None:
                share = uniform_share(self.V_e.sum(), N)
            self.beta = np.full(N, p.perfusion.w_b * p.perfusion.c_b * share)
            metabolic = np.full(N, p.perfusion.Q_m * share)
        elif p.regions is None:
            self.regions = None
            self.beta = p.perfusion.w_b * p.perfusion.c_b * self.V
            metabolic = self.V * p.perfusion.Q_m
        else:
            # W[r]: lumped volume of node i from the elements of region r
            self.regions = np.asarray(p.regions, dtype=np.int64)
            R = len(p.region_materials)
            self.W = [lumped_volumes(self.conn[self.regions == r], self.V_e[self.regions == r], N) for r in range(R)]
            pr = p.region_perfusion
            self.beta = sum(self.W[r] * pr[r].w_b * pr[r].c_b for r in range(R))
            metabolic = sum(self.W[r] * pr[r].Q_m for r in range(R))
        qr = gaussian_density(p.xyz, p.sources)
        if p.q_r is not None:
            qr = qr + np.asarray(p.q_r, dtype=np.float64)
        self.Q = metabolic + self.V * qr
        if len(p.flux_nodes):
            np.add.at(self.Q, np.asarray(p.flux_nodes, dtype=np.int64), np.asarray(p.flux_q, dtype=np.float64))
        # split for time-varying sources: Q(t) = Q_const + f(t) Q_src
        self.sched_end = np.asarray(p.schedule_end, dtype=np.float64)
        self.sched_f = np.asarray(p.schedule_factor, dtype=np.float64)
        self.Q_src = self.V * qr
        self.Q_const = metabolic.copy()
        if len(p.flux_nodes):
            np.add.at(self.Q_const, np.asarray(p.flux_nodes, dtype=np.int64), np.asarray(p.flux_q, dtype=np.float64))
        self.free = np.ones(N, dtype=bool)
        self.free[np.asarray(p.dirichlet_nodes, dtype=np.int64)] = False
        # sparsity pattern of K: one entry per (row, col) pair met in any element
        nv = self.conn.shape[1]
        rows = np.repeat(self.conn, nv, axis=1).ravel()
        cols = np.tile(self.conn, (1, nv)).ravel()
        key = rows * N + cols
        uniq, self._slot = np.unique(key, return_inverse=True)
        self._rows = uniq // N
        self._cols = uniq % N
        self.indptr = np.searchsorted(self._rows, np.arange(N + 1))

    # --- material laws (linear in T, Section 3.1.6) -------------------------
    def k_of(self, T, m=None):
        m = self.p.material if m is None else m
        if m.table is not None:
            return piecewise_linear(m.table[0], m.table[3], T)
        return m.k0 + m.dk * (T - m.T_ref)

    def rho_of(self, T, m=None):
        m = self.p.material if m is None else m
        if m.table is not None:
            return piecewise_linear(m.table[0], m.table[1], T)
        return m.rho0 + m.drho * (T - m.T_ref)

    def c_of(self, T, m=None):
        m = self.p.material if m is None else m
        if m.table is not None:
            return piecewise_linear(m.table[0], m.table[2], T)
        return m.c0 + m.dc * (T - m.T_ref)

    # --- Eq. 11 and Eq. 13: global conduction matrix at the current field ---
    def element_conductivity(self, T):
        if self.regions is None:
            return self.k_of(T)[self.conn].mean(axis=1)
        k_e = np.empty(len(self.conn))
        for r, m in enumerate(self.p.region_materials):
            sel = self.regions == r
            k_e[sel] = self.k_of(T[self.conn[sel]], m).mean(axis=1)
        return k_e

    def assemble_K(self, k_e) -> sp.csr_matrix:
        vals = (k_e[:, None, None] * self.A_e).ravel()
        data = np.bincount(self._slot, weights=vals, minlength=len(self._rows))
        return sp.csr_matrix((data, self._cols, self.indptr), shape=(self.N, self.N))

    def conduction_load(self, K: sp.csr_matrix, T) -> np.ndarray:
        """(K T)_i evaluated row by row as sum_j K_ij (T_j - T_i)."""
        contrib = K.data * (T[self._cols] - T[self._rows])
        return np.bincount(self._rows, weights=contrib, minlength=self.N)

    def initial_field(self) -> np.ndarray:
        T = self.p.T0_array()
        if len(self.p.dirichlet_nodes):
            T[np.asarray(self.p.dirichlet_nodes, dtype=np.int64)] = self.p.dirichlet_T
        return T

    def schedule_factor(self, t: float) -> float:
        """f(t): the factor of the segment that contains t (the last one after its end)."""
        if len(self.sched_f) == 0:
            return 1.0
        k = int(np.searchsorted(self.sched_end, t, side="right"))
        return float(self.sched_f[min(k, len(self.sched_f) - 1)])

    def nodal_load(self, t: float) -> np.ndarray:
        if len(self.sched_f) == 0:
            return self.Q
        return self.Q_const + self.schedule_factor(t) * self.Q_src

    def rate(self, T, t: float = 0.0) -> np.ndarray:
        """R = -K(T) T + beta (T_a - T) + Q(t) + hA (T_inf - T)  (W per node)."""
        K = self.assemble_K(self.element_conductivity(T))
        F = self.conduction_load(K, T)
        pf = self.p.perfusion
        return -F + self.beta * (pf.T_a - T) + self.nodal_load(t) + self.hA * (self.p.conv_T_inf - T)

    def capacitance(self, T) -> np.ndarray:
        if self.regions is None:
            return self.V * self.rho_of(T) * self.c_of(T)
        return sum(self.W[r] * self.rho_of(T, m) * self.c_of(T, m) for r, m in enumerate(self.p.region_materials))

    def step(self, T, dt: float, t: float = 0.0) -> np.ndarray:
        """One explicit Euler step (Eq. 6, Eq. 8) with lumped C, from time t."""
        Tn = T + dt * self.rate(T, t) / self.capacitance(T)
        Tn[~self.free] = T[~self.free]
        return Tn

    def run(self, dt: float, n_steps: int, T=None, dose=False):
        """n_steps steps from t = 0; with dose=True also returns CEM43
        (minutes), with dose=("arrhenius", A, Ea) the damage integral Omega."""
        T = self.initial_field() if T is None else np.array(T, dtype=np.float64)
        D = np.zeros(self.N)
        for k in range(n_steps):
            if isinstance(dose, tuple):
                D = D + arrhenius_increment(T, dt, dose[1], dose[2])
            elif dose:
                D = D + cem43_increment(T, dt)
            T = self.step(T, dt, k * dt)
        return (T, D) if dose else T


def piecewise_linear(Tj, pj, T):
    """p(T) through the points (Tj, pj): on the interval [Tj[i], Tj[i+1]] that
    holds T, and along the first / last interval outside the table,
    p = pj[i] + slope_i (T - Tj[i]) with slope_i = (pj[i+1] - pj[i]) / (Tj[i+1] - Tj[i])."""
    Tj = np.asarray(Tj, dtype=np.float64)
    pj = np.asarray(pj, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    i = np.clip(np.searchsorted(Tj, T, side="right") - 1, 0, len(Tj) - 2)
    slope = (pj[1:] - pj[:-1]) / (Tj[1:] - Tj[:-1])
    return pj[i] + slope[i] * (T - Tj[i])


GAS_CONSTANT = 8.314462618   # J/(mol K), CODATA 2018
KELVIN = 273.15


def arrhenius_increment(T, dt: float, A: float, Ea: float) -> np.ndarray:
    """Arrhenius thermal damage (Henriques and Moritz, 1947): the damage
    integral Omega = int A exp(-Ea / (R T_K)) dt, one step at the step's start
    temperature: dt A exp(-Ea / (R (T + 273.15)))."""
    T = np.asarray(T, dtype=np.float64)
    return dt * A * np.exp(-Ea / (GAS_CONSTANT * (T + KELVIN)))


def cem43_increment(T, dt: float) -> np.ndarray:
    """(dt / 60) R^(43 - T) minutes, R = 1/2 at or above 43 degC, 1/4 below."""
    T = np.asarray(T, dtype=np.float64)
    R = np.where(T >= 43.0, 0.5, 0.25)
    return (dt / 60.0) * R ** (43.0 - T)
