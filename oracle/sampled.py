"""Oracle values at a few sampled nodes of a mesh too large to step whole.

Oracle code (test infrastructure only).  After s explicit steps the value at
node i depends only on nodes within s element-neighbour rings of i (each step
of Eq. 8 couples a node to the nodes of the elements that contain it).  So the
oracle steps the sub-mesh made of every element that touches a node within
s - 1 rings of the samples.  Nodes of that sub-mesh further out have incomplete
element sets and go wrong, but the error front moves inward one ring per step
and does not reach the samples in s steps.
"""
from __future__ import annotations

import copy

import numpy as np
import scipy.sparse as sp

from .global_form import Oracle


def _node_adjacency(conn: np.ndarray, n_nodes: int) -> sp.csr_matrix:
    E, nv = conn.shape
    rows = np.repeat(np.arange(E), nv)
    inc = sp.csr_matrix((np.ones(E * nv, dtype=np.int8), (rows, conn.ravel())), shape=(E, n_nodes))
    return inc


def sampled_run(problem, dt: float, n_steps: int, samples: np.ndarray) -> np.ndarray:
    """T after n_steps at the sample nodes (initial field = problem.T0)."""
    conn = np.asarray(problem.conn, dtype=np.int64)
    N = problem.n_nodes
    inc = _node_adjacency(conn, N)            # element x node incidence
    inc_t = inc.T.tocsr()
    ring = np.zeros(N, dtype=bool)
    ring[samples] = True
    for _ in range(max(n_steps - 1, 0)):
        elems = np.unique(inc_t[np.nonzero(ring)[0]].indices)
        ring[np.unique(conn[elems].ravel())] = True
    elems = np.unique(inc_t[np.nonzero(ring)[0]].indices)
    nodes = np.unique(conn[elems].ravel())
    local = -np.ones(N, dtype=np.int64)
    local[nodes] = np.arange(len(nodes))

    sub = copy.copy(problem)
    sub.xyz = problem.xyz[nodes]
    sub.conn = local[conn[elems]].astype(np.int32)
    T0 = problem.T0_array()[nodes]
    sub.T0 = T0
    if problem.q_r is not None:
        sub.q_r = np.asarray(problem.q_r)[nodes]
    dn = np.asarray(problem.dirichlet_nodes, dtype=np.int64)
    keep = local[dn] >= 0
    sub.dirichlet_nodes = local[dn[keep]].astype(np.int32)
    sub.dirichlet_T = np.asarray(problem.dirichlet_T)[keep]
    fn = np.asarray(problem.flux_nodes, dtype=np.int64)
    keep = local[fn] >= 0 if len(fn) else np.zeros(0, bool)
    sub.flux_nodes = local[fn[keep]].astype(np.int32) if len(fn) else problem.flux_nodes
    sub.flux_q = np.asarray(problem.flux_q)[keep] if len(fn) else problem.flux_q
    cf = np.asarray(problem.conv_faces, dtype=np.int64)
    if len(cf):
        keep = np.all(local[cf] >= 0, axis=1)
        sub.conv_faces = local[cf[keep]].astype(np.int32)
    if getattr(problem, "regions", None) is not None:
        sub.regions = np.asarray(problem.regions)[elems]
    if getattr(problem, "lumping", "element") == "uniform":
        # the share V / N belongs to the whole mesh, not to the sub-mesh
        sub.uniform_volume_per_node = Oracle(problem).V_e.sum() / N
    orc = Oracle(sub)
    T = orc.run(dt, n_steps)
    return T[local[np.asarray(samples, dtype=np.int64)]]
