"""Single-mesh partition over several GPUs: the host plan of the halo exchange.

The parallel loops of the method (Section 2.4) are independent over elements
and over nodes; only the sum of element loads into a node (Eq. 11) and the
temperatures an element reads couple them.  A rank therefore owns a contiguous
range of the free nodes in the internal (space-filling) order and holds every
element that touches one of them, so each owned node finds all of its element
loads on its own rank and sums them in the fixed order of the one-GPU path
(no partial sums cross ranks, no floating-point reduction).  Elements on a
range boundary are computed by every rank that touches them, as the tiles of
the tiled kernels are.  The only exchange per time step is the new
temperature of each owned node that another rank reads (its halo), sent to
that rank before the next step.

This module is host logic only (index sets, no arithmetic of the method).
``plan_partition`` returns, per rank, the global ids of its owned nodes, its
elements (increasing global id), its halo nodes, and for every peer the
owned nodes it sends and the halo nodes it receives, each list in increasing
global id, so that both sides of an exchange agree on the order.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List

import numpy as np


@dataclass
class RankPlan:
    rank: int
    owned: np.ndarray                      # free nodes this rank updates (global ids, increasing)
    elements: np.ndarray                   # elements touching an owned node (global ids, increasing)
    nodes: np.ndarray                      # every node of those elements (global ids, increasing)
    halo: np.ndarray                       # free nodes of those elements owned elsewhere
    send: Dict[int, np.ndarray] = field(default_factory=dict)   # peer -> owned nodes it reads
    recv: Dict[int, np.ndarray] = field(default_factory=dict)   # peer -> halo nodes it owns


def plan_partition(conn: np.ndarray, n_nodes: int, free: np.ndarray, n_ranks: int,
                   node_order: np.ndarray | None = None) -> List[RankPlan]:
    """Split the free nodes into n_ranks contiguous ranges of `node_order`
    (a permutation of the nodes, e.g. the library's internal order; default:
    input order) and derive each rank's elements, halo and exchange lists."""
    conn = np.asarray(conn, dtype=np.int64)
    free = np.asarray(free, dtype=bool)
    order = np.arange(n_nodes) if node_order is None else np.asarray(node_order, dtype=np.int64)
    free_in_order = order[free[order]]
    bounds = np.linspace(0, len(free_in_order), n_ranks + 1).round().astype(np.int64)
    owner = np.full(n_nodes, -1, dtype=np.int64)             # -1: Dirichlet (held everywhere)
    for r in range(n_ranks):
        owner[free_in_order[bounds[r]:bounds[r + 1]]] = r
    plans = []
    for r in range(n_ranks):
        owned = np.sort(free_in_order[bounds[r]:bounds[r + 1]])
        mine = np.zeros(n_nodes, dtype=bool)
        mine[owned] = True
        elements = np.nonzero(mine[conn].any(axis=1))[0]
        nodes = np.unique(conn[elements])
        halo = nodes[(owner[nodes] >= 0) & (owner[nodes] != r)]
        plans.append(RankPlan(r, owned, elements, nodes, halo))
    for p in plans:
        for q in range(n_ranks):
            if q == p.rank:
                continue
            recv = p.halo[owner[p.halo] == q]
            if len(recv):
                p.recv[q] = recv
                plans[q].send[p.rank] = recv          # q sends exactly what p receives, same order
    return plans


def check_plan(plans: List[RankPlan], conn: np.ndarray, n_nodes: int, free: np.ndarray) -> None:
    """Raise AssertionError unless the plan is consistent: every free node is
    owned exactly once; a rank holds every element of each owned node; its
    halo is every free non-owned node of its elements; sends and receives
    pair up."""
    conn = np.asarray(conn, dtype=np.int64)
    count = np.zeros(n_nodes, dtype=np.int64)
    for p in plans:
        count[p.owned] += 1
    assert np.all(count[free] == 1) and np.all(count[~free] == 0)
    for p in plans:
        mine = np.zeros(n_nodes, dtype=bool)
        mine[p.owned] = True
        need = np.nonzero(mine[conn].any(axis=1))[0]
        assert np.array_equal(need, p.elements)
        touched = np.unique(conn[p.elements])
        assert np.array_equal(touched, p.nodes)
        want_halo = touched[free[touched] & ~mine[touched]]
        assert np.array_equal(np.sort(np.concatenate(list(p.recv.values()) or [np.zeros(0, np.int64)])), want_halo)
        for q, ids in p.send.items():
            assert np.array_equal(plans[q].recv[p.rank], ids)
            assert mine[ids].all()
