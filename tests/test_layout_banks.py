"""The bank-aware element order of tet tiles (host layout, no GPU): within
each tile the elements are the same set as in sorted order, each carries the
same local ids and ranks, and a replay of the warps' shared-memory accesses
(temperature gathers at the local id, load stores at rank x (B + 1) + id;
32 consecutive elements per warp, 4-byte words in 32 banks) needs fewer
wavefronts than the sorted order: far fewer for the stores."""
import numpy as np
import pytest

from synth.scenarios import ellipsoid_tet_td


@pytest.fixture(scope="module")
def ff():
    from paper_1909_05098_gb300.build import build
    build()
    from paper_1909_05098_gb300 import fedfem
    return fedfem


def _wavefronts(words):
    """Wavefronts of each warp access: the most distinct words in one bank."""
    out = []
    for row in words:
        a = np.unique(row[row >= 0])
        if len(a):
            out.append(np.bincount(a % 32, minlength=32).max())
    return out


def test_tet_tiles_order_elements_away_from_bank_conflicts(ff):
    p = ellipsoid_tet_td(h=1.5e-3, axes=(0.03, 0.024, 0.02)).problem
    B, nv = 192, 4
    d = ff.fedfem_plan_layout(p.elem_type, p.xyz, p.conn, order=0, dirichlet_nodes=p.dirichlet_nodes, tile_nodes=B)
    eo, lc, elems = d["tile_elem_off"], d["tile_lconn"].astype(np.int64), d["tile_elems"]
    shift, NF = d["tile_rank_shift"], d["n_free"]
    got = {"gather": [], "store": []}
    ref = {"gather": [], "store": []}
    for t in range(len(eo) - 1):
        ne = eo[t + 1] - eo[t]
        codes = lc[eo[t] * nv:eo[t + 1] * nv].reshape(ne, nv)
        e = elems[eo[t]:eo[t + 1]]
        assert len(np.unique(e)) == ne                     # a permutation of the tile's elements
        srt = np.argsort(e)
        own = min(B, NF - t * B)
        for order, acc in ((np.arange(ne), got), (srt, ref)):
            c = codes[order]
            lid, rk = c & ((1 << shift) - 1), c >> shift
            store = np.where(lid < own, rk * (B + 1) + lid, -1)
            pad = -np.ones((-(-ne // 32) * 32, nv), np.int64)
            for name, w in (("gather", lid), ("store", store)):
                pad[:] = -1
                pad[:ne] = w
                for k in range(nv):
                    acc[name] += _wavefronts(pad[:, k].reshape(-1, 32))
    g, r = {k: float(np.mean(v)) for k, v in got.items()}, {k: float(np.mean(v)) for k, v in ref.items()}
    print(f"wavefronts per warp access, bank-aware order vs sorted: gather {g['gather']:.3f} vs {r['gather']:.3f}, "
          f"store {g['store']:.3f} vs {r['store']:.3f}")
    assert g["gather"] < r["gather"]
    assert g["store"] < 0.75 * r["store"]
