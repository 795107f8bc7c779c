"""The surrogate's graph: directed edges between nodes that share an element
(the sparsity pattern of the conduction matrix).  Topology only."""
from __future__ import annotations

import numpy as np


def mesh_edges(conn: np.ndarray, n_nodes: int):
    """(src, dst) of every ordered pair of distinct nodes sharing an element,
    sorted by destination then source."""
    conn = np.asarray(conn, dtype=np.int64)
    nv = conn.shape[1]
    a = np.repeat(conn, nv, axis=1).ravel()
    b = np.tile(conn, (1, nv)).ravel()
    keep = a != b
    key = np.unique(b[keep] * n_nodes + a[keep])      # dst-major
    return (key % n_nodes).astype(np.int32), (key // n_nodes).astype(np.int32)
