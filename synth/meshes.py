"""Seeded synthetic meshes shaped like the paper's workloads.

The paper's liver mesh (Section 3.1.1) is not available, so these stand in:

* ``hex_box``        structured box of eight-node hexahedra (one-point elements
                     of Eq. 14), lexicographic node order, standard hex8 corner
                     order (bottom face counter-clockwise, then top face);
* ``kuhn_tet_box``   the same grid with every voxel split into six tetrahedra
                     along its main diagonal (Freudenthal/Kuhn split, conforming);
* ``tet_ellipsoid``  a voxelised ellipsoid, Kuhn-split, with every node
                     coordinate jittered independently (the tet4 workloads).

Only connectivity, coordinates and node/face sets are produced here.  Nothing
in this module computes a Jacobian, a volume, an element matrix or a load.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

# hex8 corners as (di, dj, dk) offsets, bottom face counter-clockwise then top
HEX8_CORNERS = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                         [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=np.int64)


def _kuhn_tets() -> np.ndarray:
    """The six tetrahedra of the unit voxel that share the (0,0,0)-(1,1,1)
    diagonal, as corner offsets, all with positive orientation."""
    tets = []
    for perm in itertools.permutations(range(3)):
        v = [np.zeros(3, np.int64)]
        for ax in perm:
            nxt = v[-1].copy()
            nxt[ax] += 1
            v.append(nxt)
        # permutation parity decides orientation; odd ones swap the last two corners
        inversions = sum(1 for a in range(3) for b in range(a + 1, 3) if perm[a] > perm[b])
        if inversions % 2 == 1:
            v[2], v[3] = v[3], v[2]
        tets.append(np.stack(v))
    return np.stack(tets)  # (6, 4, 3)


KUHN_TETS = _kuhn_tets()


@dataclass
class Mesh:
    elem_type: int
    xyz: np.ndarray        # (N, 3) float64
    conn: np.ndarray       # (E, nv) int32
    grid_index: np.ndarray  # (N, 3) int64 integer grid coordinates of each node


def hex_box(nx: int, ny: int, nz: int, h: float, origin=(0.0, 0.0, 0.0)) -> Mesh:
    """Box of nx*ny*nz cubes of edge h; node id = i + (nx+1)*(j + (ny+1)*k)."""
    gi, gj, gk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    grid = np.stack([gi.ravel(order="F"), gj.ravel(order="F"), gk.ravel(order="F")], axis=1)
    xyz = origin + grid * h
    ei, ej, ek = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    base = np.stack([ei.ravel(order="F"), ej.ravel(order="F"), ek.ravel(order="F")], axis=1)
    corners = base[:, None, :] + HEX8_CORNERS[None, :, :]
    conn = corners[..., 0] + (nx + 1) * (corners[..., 1] + (ny + 1) * corners[..., 2])
    return Mesh(8, xyz.astype(np.float64), conn.astype(np.int32), grid.astype(np.int64))


def kuhn_tet_box(nx: int, ny: int, nz: int, h: float, origin=(0.0, 0.0, 0.0)) -> Mesh:
    """Box of nx*ny*nz voxels, each split into the six Kuhn tetrahedra."""
    hb = hex_box(nx, ny, nz, h, origin)
    ei, ej, ek = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    base = np.stack([ei.ravel(order="F"), ej.ravel(order="F"), ek.ravel(order="F")], axis=1)
    corners = base[:, None, None, :] + KUHN_TETS[None]          # (V, 6, 4, 3)
    ids = corners[..., 0] + (nx + 1) * (corners[..., 1] + (ny + 1) * corners[..., 2])
    return Mesh(4, hb.xyz, ids.reshape(-1, 4).astype(np.int32), hb.grid_index)


def box_face_nodes(mesh: Mesh, faces=("x0", "x1", "y0", "y1", "z0", "z1")) -> np.ndarray:
    """Node ids on the named faces of a box mesh (x0 = minimum x face, ...)."""
    g = mesh.grid_index
    hi = g.max(axis=0)
    sel = np.zeros(len(g), dtype=bool)
    for f in faces:
        ax = "xyz".index(f[0])
        sel |= g[:, ax] == (0 if f[1] == "0" else hi[ax])
    return np.nonzero(sel)[0].astype(np.int32)


def hex_box_top_faces(nx: int, ny: int, nz: int) -> np.ndarray:
    """Quadrilateral faces (outward +z, counter-clockwise) on the z = max face of hex_box."""
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    i, j = i.ravel(order="F"), j.ravel(order="F")
    k = nz
    q = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
    return np.stack([a + (nx + 1) * (b + (ny + 1) * k) for a, b in q], axis=1).astype(np.int32)


def _ellipsoid_voxels(semi_axes, h):
    a = np.asarray(semi_axes, dtype=np.float64)
    n = 2 * np.ceil(a / h).astype(np.int64)        # voxels per axis, grid centred on 0
    c = [(np.arange(n[d]) + 0.5) * h - n[d] * h / 2 for d in range(3)]
    inside = ((c[0][:, None, None] / a[0]) ** 2 + (c[1][None, :, None] / a[1]) ** 2
              + (c[2][None, None, :] / a[2]) ** 2) <= 1.0
    return n, inside


def ellipsoid_node_count(semi_axes, h) -> int:
    """Number of grid nodes touched by the voxels whose centre is inside."""
    n, inside = _ellipsoid_voxels(semi_axes, h)
    touched = np.zeros(tuple(n + 1), dtype=bool)
    for d in HEX8_CORNERS:
        touched[d[0]:d[0] + n[0], d[1]:d[1] + n[1], d[2]:d[2] + n[2]] |= inside
    return int(touched.sum())


@dataclass
class EllipsoidMesh(Mesh):
    surface_nodes: np.ndarray = None   # nodes on voxel faces not shared by two inside voxels
    semi_axes: tuple = None
    h: float = 0.0


def tet_ellipsoid(semi_axes, h: float, jitter: float, seed: int) -> EllipsoidMesh:
    """Voxelise the ellipsoid sum (x_d / a_d)^2 <= 1 (a voxel is inside when its
    centre is), split each voxel into six Kuhn tetrahedra, then move every node
    coordinate by an independent U[-jitter, jitter] offset drawn from ``seed``.

    The jitter stays below half of the smallest tetrahedron height of the
    Kuhn split (h / sqrt(2) / 2 for unit voxels scaled by h) when
    jitter <= 0.2 h, so no element can invert."""
    n, inside = _ellipsoid_voxels(semi_axes, h)
    vox = np.argwhere(inside)                                   # (V, 3) in (i, j, k)
    touched = np.zeros(tuple(n + 1), dtype=bool)
    for d in HEX8_CORNERS:
        touched[d[0]:d[0] + n[0], d[1]:d[1] + n[1], d[2]:d[2] + n[2]] |= inside
    # lexicographic node numbering with x fastest
    order = np.transpose(touched, (2, 1, 0)).ravel()
    gid = -np.ones(order.size, dtype=np.int64)
    gid[order] = np.arange(int(order.sum()))
    gid = np.transpose(gid.reshape(n[2] + 1, n[1] + 1, n[0] + 1), (2, 1, 0))
    grid = np.argwhere(np.transpose(touched, (2, 1, 0)))[:, ::-1]   # (N, 3), x fastest
    corners = vox[:, None, None, :] + KUHN_TETS[None]
    conn = gid[corners[..., 0], corners[..., 1], corners[..., 2]].reshape(-1, 4)
    # surface: faces of inside voxels whose neighbour is outside
    pad = np.zeros(tuple(n + 2), dtype=bool)
    pad[1:-1, 1:-1, 1:-1] = inside
    surf = np.zeros(tuple(n + 1), dtype=bool)
    for ax in range(3):
        for side in (0, 1):
            sh = [slice(1, -1)] * 3
            sh[ax] = slice(2, None) if side else slice(0, -2)
            exposed = inside & ~pad[tuple(sh)]
            face_corners = [c for c in HEX8_CORNERS if c[ax] == side]
            for d in face_corners:
                surf[d[0]:d[0] + n[0], d[1]:d[1] + n[1], d[2]:d[2] + n[2]] |= exposed
    surface_nodes = np.sort(gid[surf]).astype(np.int32)
    origin = -n * h / 2
    rng = np.random.default_rng(seed)
    xyz = origin + grid * h + rng.uniform(-jitter, jitter, size=grid.shape)
    return EllipsoidMesh(4, xyz.astype(np.float64), conn.astype(np.int32), grid.astype(np.int64),
                         surface_nodes=surface_nodes, semi_axes=tuple(semi_axes), h=h)
