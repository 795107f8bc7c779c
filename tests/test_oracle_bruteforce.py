"""Brute-force pins of the oracle's assembled conduction matrix (Eq. 10-11
with k_e of Eq. 13) and of its reporting statistics.

* K(T) = sum_e k_e A_e, built here by explicit loops over elements and their
  corner pairs on jittered meshes of one to eight elements, with the element
  matrices formed by a route of their own: tet4 shape-function gradients by
  solving the 4 x 4 interpolation system of each tetrahedron (Eq. 15), hex8
  shape-function derivatives at the element centre by central differences of
  the trilinear functions written out (Eq. 14; exact for functions linear in
  each natural coordinate).  It must equal the oracle's sparse K entry by
  entry, and the oracle's row-difference product must equal K T.
* The table statistics (min, max, median, RMS, quartiles, the rows of
  Tables 1-5) against values worked out by hand on small samples.
"""
import numpy as np
import pytest

from oracle import Oracle, table_stats
from synth.meshes import hex_box, kuhn_tet_box
from synth.problem import Material, Problem
from synth.scenarios import TISSUE_TD

H = 1e-3


def _tet_matrix(x):
    """V grad N_a . grad N_b with N_a the linear function equal to 1 at corner a."""
    Vm = np.hstack([np.ones((4, 1)), x])                  # rows [1, x, y, z]
    coef = np.linalg.solve(Vm, np.eye(4))                 # column a: coefficients of N_a
    G = coef[1:, :]                                       # (3, 4) gradients
    vol = abs(np.linalg.det(x[1:] - x[0])) / 6.0
    A = np.zeros((4, 4))
    for a in range(4):
        for b in range(4):
            A[a, b] = vol * np.dot(G[:, a], G[:, b])
    return A


_SIGNS = [(-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1), (-1, -1, 1), (1, -1, 1), (1, 1, 1), (-1, 1, 1)]


def _trilinear(n, xi):
    s = _SIGNS[n]
    return (1 + s[0] * xi[0]) * (1 + s[1] * xi[1]) * (1 + s[2] * xi[2]) / 8.0


def _hex_matrix(x):
    """One-point hexahedron: J and dN/dx at the centre from central differences."""
    d = 0.5
    dN = np.zeros((3, 8))                                 # dN_n / dxi_j at the centre
    for n in range(8):
        for j in range(3):
            e = np.zeros(3)
            e[j] = d
            dN[j, n] = (_trilinear(n, e) - _trilinear(n, -e)) / (2 * d)
    J = np.zeros((3, 3))                                  # J_ij = d x_i / d xi_j
    for n in range(8):
        for i in range(3):
            for j in range(3):
                J[i, j] += x[n, i] * dN[j, n]
    G = np.linalg.solve(J.T, dN)                          # dN/dx = J^-T dN/dxi
    detJ = np.linalg.det(J)
    A = np.zeros((8, 8))
    for a in range(8):
        for b in range(8):
            A[a, b] = 8.0 * detJ * np.dot(G[:, a], G[:, b])
    return A


def _jittered(mesh, seed, amount=0.2):
    rng = np.random.default_rng(seed)
    return mesh.xyz + rng.uniform(-amount * H, amount * H, mesh.xyz.shape)


MESHES = {
    "one tet": (4, lambda: kuhn_tet_box(1, 1, 1, H), [0]),
    "six Kuhn tets": (4, lambda: kuhn_tet_box(1, 1, 1, H), None),
    "eight tets of two voxels": (4, lambda: kuhn_tet_box(2, 1, 1, H), [0, 1, 3, 5, 6, 7, 8, 11]),
    "one hex": (8, lambda: hex_box(1, 1, 1, H), None),
    "two hexes": (8, lambda: hex_box(2, 1, 1, H), None),
    "eight hexes": (8, lambda: hex_box(2, 2, 2, H), None),
}


@pytest.mark.parametrize("name", list(MESHES))
def test_assembled_K_equals_brute_force_sum_of_element_matrices(name):
    nv, make, keep = MESHES[name]
    m = make()
    conn = m.conn if keep is None else m.conn[keep]
    used = np.unique(conn)
    remap = -np.ones(len(m.xyz), dtype=np.int64)
    remap[used] = np.arange(len(used))
    conn = remap[conn].astype(np.int32)
    xyz = _jittered(m, seed=len(name))[used]
    p = Problem(nv, xyz, conn, TISSUE_TD)
    orc = Oracle(p)
    rng = np.random.default_rng(11)
    T = 37.0 + 30.0 * rng.random(len(xyz))
    # Eq. 13: the plain mean of the nodal conductivities, element by element
    mat = p.material
    k_e = np.zeros(len(conn))
    for e in range(len(conn)):
        s = 0.0
        for a in range(nv):
            s += mat.k0 + mat.dk * (T[conn[e, a]] - mat.T_ref)
        k_e[e] = s / nv
    Kd = np.zeros((len(xyz), len(xyz)))
    for e in range(len(conn)):
        A = _tet_matrix(xyz[conn[e]]) if nv == 4 else _hex_matrix(xyz[conn[e]])
        for a in range(nv):
            for b in range(nv):
                Kd[conn[e, a], conn[e, b]] += k_e[e] * A[a, b]
    K = orc.assemble_K(orc.element_conductivity(T))
    scale = np.abs(Kd).max()
    np.testing.assert_allclose(K.toarray(), Kd, rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(orc.conduction_load(K, T), Kd @ T, rtol=0, atol=1e-12 * scale * np.abs(T).max())
    # the brute-force matrix itself: symmetric, rows summing to zero
    np.testing.assert_allclose(Kd, Kd.T, rtol=0, atol=1e-14 * scale)
    np.testing.assert_allclose(Kd.sum(axis=1), 0.0, atol=1e-13 * scale)


def test_table_statistics_by_hand():
    """Four values 4, 1, 3, 2: median 2.5, RMS sqrt(30/4), quartiles by linear
    interpolation between order statistics at positions 0.75 and 2.25 (1.75
    and 3.25).  Five values -3, 0, 0, 5, 8: median 0, RMS sqrt(98/5), quartiles
    at positions 1 and 3 (0 and 5)."""
    s = table_stats([4.0, 1.0, 3.0, 2.0])
    assert (s["min"], s["max"], s["median"]) == (1.0, 4.0, 2.5)
    assert s["rms"] == pytest.approx(np.sqrt(7.5), rel=1e-15)
    assert s["q1"] == pytest.approx(1.75, rel=1e-15)
    assert s["q3"] == pytest.approx(3.25, rel=1e-15)
    s = table_stats([-3.0, 0.0, 0.0, 5.0, 8.0])
    assert (s["min"], s["max"], s["median"], s["q1"], s["q3"]) == (-3.0, 8.0, 0.0, 0.0, 5.0)
    assert s["rms"] == pytest.approx(np.sqrt(19.6), rel=1e-15)
    s = table_stats(np.full(7, 37.25))                  # a constant field: every statistic is the value
    assert all(v == pytest.approx(37.25, rel=1e-15) for v in s.values())
