"""Host logic of the library (no GPU): internal order, node ranges, the
sliced-ELL gather and the tiles of the tiled kernel, read through the
host-only fedfem_plan_layout call.  The last test emulates the tiled kernel's
shared-memory gather in numpy with the oracle's element loads and compares
the nodal sums with the oracle's assembled K T."""
import numpy as np
import pytest

from oracle import Oracle
from synth.scenarios import cube_hex_td_convective, ellipsoid_tet_td


@pytest.fixture(scope="module")
def ff():
    from paper_1909_05098_gb300.build import build
    build()
    from paper_1909_05098_gb300 import fedfem
    return fedfem


CASES = {
    "hex": lambda: cube_hex_td_convective(n=9).problem,
    "tet": lambda: ellipsoid_tet_td(h=3e-3, axes=(0.02, 0.015, 0.012)).problem,
}


def _plan(ff, p, order, B):
    return ff.fedfem_plan_layout(p.elem_type, p.xyz, p.conn, order=order, dirichlet_nodes=p.dirichlet_nodes,
                                 faces=p.conv_faces if len(p.conv_faces) else None, tile_nodes=B)


def _decode_gather(d, nv, i):
    s, lane = i // 32, i % 32
    off, w = d["slice_off"][s], (d["slice_off"][s + 1] - d["slice_off"][s]) // 32
    ents = d["gather"][off + 32 * np.arange(w) + lane]
    return ents[ents < d["n_elems"] * nv]


@pytest.mark.parametrize("kind", ["hex", "tet"])
@pytest.mark.parametrize("order", [0, 1, 2])
def test_order_ranges_and_gather(ff, kind, order):
    p = CASES[kind]()
    nv = p.elem_type
    d = _plan(ff, p, order, 0)
    N, E = p.n_nodes, p.n_elems
    node_of, elem_of = d["node_of"], d["elem_of"]
    assert np.array_equal(np.sort(node_of), np.arange(N))
    assert np.array_equal(np.sort(elem_of), np.arange(E))
    is_dir = np.zeros(N, bool)
    is_dir[p.dirichlet_nodes] = True
    assert not is_dir[node_of[: d["n_free"]]].any() and is_dir[node_of[d["n_free"]:]].all()
    film = np.zeros(N, bool)
    if len(p.conv_faces):
        film[np.unique(p.conv_faces)] = True
    film &= ~is_dir
    assert not film[node_of[: d["n_plain"]]].any() and film[node_of[d["n_plain"]: d["n_free"]]].all()
    seen = np.zeros(E * nv, np.int32)
    for i in range(d["n_free"]):
        ents = _decode_gather(d, nv, i)
        e_int, corner = ents // nv, ents % nv
        e_in = elem_of[e_int]
        assert np.all(p.conn[e_in, corner] == node_of[i])
        assert np.all(np.diff(e_in) > 0)                # input element order fixes the sum order
        seen[e_in * nv + corner] += 1
    free_slot = ~is_dir[p.conn.ravel()]
    assert np.all(seen[free_slot] == 1) and np.all(seen[~free_slot] == 0)


def test_morton_order_is_a_z_curve_on_the_cube(ff):
    p = cube_hex_td_convective(n=8).problem
    d = _plan(ff, p, 1, 0)
    centre = p.xyz[p.conn].mean(axis=1)[d["elem_of"]]
    cell = np.floor(centre / 1e-3).astype(int)
    # every aligned group of 8 consecutive elements is a 2x2x2 block, of 64 a 4x4x4 block
    for g in (8, 64):
        blocks = cell.reshape(-1, g, 3)
        span = blocks.max(axis=1) - blocks.min(axis=1)
        assert np.all(span == round(g ** (1 / 3)) - 1)


@pytest.mark.parametrize("kind,B", [("hex", 64), ("hex", 96), ("tet", 32), ("tet", 128)])
def test_tiles_cover_and_emulated_gather_matches_oracle(ff, kind, B):
    p = CASES[kind]()
    nv = p.elem_type
    d = _plan(ff, p, 1, B)
    node_of, elem_of = d["node_of"], d["elem_of"]
    NF = d["n_free"]
    orc = Oracle(p)
    rng = np.random.default_rng(3)
    T_in = 37 + 5 * rng.random(p.n_nodes)             # input order
    k_e = orc.element_conductivity(T_in)
    Fe = np.einsum("e,enm,em->en", k_e, orc.A_e, T_in[p.conn] - T_in[p.conn[:, :1]])   # input elements
    ref = orc.conduction_load(orc.assemble_K(k_e), T_in)                                 # input nodes
    T_int = T_in[node_of]
    # internal connectivity
    conn_int = np.argsort(node_of)[p.conn[elem_of]]
    out = np.full(NF, np.nan)
    for t in range(d["n_tiles"]):
        base, own = t * B, min(B, NF - t * B)
        e0, e1 = d["tile_elem_off"][t], d["tile_elem_off"][t + 1]
        h0, h1 = d["tile_halo_off"][t], d["tile_halo_off"][t + 1]
        elems = d["tile_elems"][e0:e1]
        halo = d["tile_halo"][h0:h1]
        ne = len(elems)
        local_nodes = np.concatenate([np.arange(base, base + own), halo])
        lconn = d["tile_lconn"][e0 * nv: e1 * nv].reshape(-1, nv).astype(np.int64)
        shift = d["tile_rank_shift"]
        lconn_id, lconn_rank = lconn & ((1 << shift) - 1), lconn >> shift
        assert np.array_equal(local_nodes[lconn_id], conn_int[elems])     # local ids resolve correctly
        # every element touching an owned node is in the tile
        touching = np.nonzero(np.any((conn_int >= base) & (conn_int < base + own), axis=1))[0]
        assert np.array_equal(np.sort(elems), touching)
        Ts = T_int[local_nodes]
        assert np.allclose(Ts[lconn_id], T_int[conn_int[elems]])
        # the kernel's load table: each owned corner's load goes to row `rank`
        # of its node's column; a node sums its column in row order
        D = d["tile_degree"][t]
        table = np.zeros((max(D, 1), own))
        filled = np.zeros((max(D, 1), own), bool)
        Fe_t = Fe[elem_of[elems]]
        for j in range(ne):
            for n in range(nv):
                l, r = lconn_id[j, n], lconn_rank[j, n]
                if l < own:
                    assert r < D and not filled[r, l]                   # one load per cell
                    table[r, l] = Fe_t[j, n]
                    filled[r, l] = True
                else:
                    assert r == 0
        for l in range(own):
            ents = _decode_gather(d, nv, base + l)
            deg = len(ents)
            assert filled[:deg, l].all() and not filled[deg:, l].any()  # rows 0..deg-1, then zeros
            # row r holds the load of the node's r-th slot, in input element order
            by_rank = sorted((lconn_rank[j, n], elems[j] * nv + n) for j in range(ne) for n in range(nv)
                             if lconn_id[j, n] == l)
            assert [e for _, e in by_rank] == list(ents)
            acc = 0.0
            for r in range(D):
                acc = acc + table[r, l]
            out[base + l] = acc
    np.testing.assert_allclose(out, ref[node_of[:NF]], rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_element_groups_keep_meshes_apart(ff):
    """Two meshes occupying the same space, given as one mesh with element
    groups: the internal order must not interleave them."""
    from synth.meshes import tet_ellipsoid
    a = tet_ellipsoid((0.012, 0.01, 0.008), 2e-3, 4e-4, 1)
    b = tet_ellipsoid((0.011, 0.01, 0.009), 2e-3, 4e-4, 2)
    xyz = np.vstack([a.xyz, b.xyz])
    conn = np.vstack([a.conn, b.conn + len(a.xyz)])
    groups = np.concatenate([np.zeros(len(a.conn), np.int32), np.ones(len(b.conn), np.int32)])
    for order in (0, 1, 2):
        d = ff.fedfem_plan_layout(4, xyz, conn, order=order, groups=groups)
        g = groups[d["elem_of"]]
        assert np.all(np.diff(g) >= 0)
        node_mesh = (d["node_of"] >= len(a.xyz)).astype(int)
        assert np.all(np.diff(node_mesh) >= 0)
