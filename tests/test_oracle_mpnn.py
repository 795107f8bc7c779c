"""Pins of the surrogate's FP64 reference network (the gradient oracle):
central finite differences, permutation equivariance, L-hop locality and
translation invariance."""
import numpy as np
import pytest

from oracle import mpnn
from synth.graph import mesh_edges
from synth.meshes import hex_box


def _setup(H=8, L=2, B=2, seed=0):
    m = hex_box(2, 2, 1, 1e-3)
    src, dst = mesh_edges(m.conn, len(m.xyz))
    rng = np.random.default_rng(seed)
    N = len(m.xyz)
    d = (m.xyz[dst] - m.xyz[src]) / 1e-3
    f = np.concatenate([d, np.linalg.norm(d, axis=1, keepdims=True)], axis=1)
    x = rng.normal(size=(B, N, 5))
    flat = rng.normal(size=mpnn.n_params(H, L)) * 0.5
    target = rng.normal(size=(B, N))
    mask = (rng.random(N) > 0.2).astype(float)
    return flat, x, f, src, dst, target, mask


def test_edges_of_a_hex_grid():
    m = hex_box(10, 10, 10, 1e-3)
    src, dst = mesh_edges(m.conn, len(m.xyz))
    assert len(src) == 28460                      # 26-neighbour stencil of the 11^3 grid
    assert np.all(np.diff(dst.astype(np.int64) * 10 ** 6 + src) > 0)


def test_gradient_matches_central_differences():
    H, L = 8, 2
    flat, x, f, src, dst, target, mask = _setup(H, L)
    loss, g, _ = mpnn.loss_and_grad(flat, x, f, src, dst, target, mask, H, L)
    rng = np.random.default_rng(1)
    idx = rng.choice(len(flat), 60, replace=False)
    eps = 1e-6
    for i in idx:
        p, q = flat.copy(), flat.copy()
        p[i] += eps
        q[i] -= eps
        lp = mpnn.loss_and_grad(p, x, f, src, dst, target, mask, H, L)[0]
        lq = mpnn.loss_and_grad(q, x, f, src, dst, target, mask, H, L)[0]
        fd = (lp - lq) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, np.abs(g).max()), (i, fd, g[i])


def test_permutation_equivariance():
    H, L = 8, 2
    flat, x, f, src, dst, target, mask = _setup(H, L, seed=3)
    y, _ = mpnn.forward(flat, x, f, src, dst, H, L)
    N = x.shape[1]
    perm = np.random.default_rng(4).permutation(N)       # new id of old node i is perm[i]
    inv = np.argsort(perm)
    s2, d2 = perm[src], perm[dst]
    order = np.lexsort((s2, d2))
    y2, _ = mpnn.forward(flat, x[:, inv], f[order], s2[order], d2[order], H, L)
    np.testing.assert_allclose(y2[:, perm], y, rtol=1e-12, atol=1e-12)


def _hops(src, dst, N, start):
    """Graph distance from `start` along edges src -> dst (breadth-first)."""
    dist = np.full(N, np.inf)
    dist[start] = 0
    frontier = [start]
    adj = [[] for _ in range(N)]
    for s, d in zip(src, dst):
        adj[s].append(d)
    k = 0
    while frontier:
        k += 1
        nxt = []
        for u in frontier:
            for v in adj[u]:
                if dist[v] == np.inf:
                    dist[v] = k
                    nxt.append(v)
        frontier = nxt
    return dist


@pytest.mark.parametrize("L", [1, 2, 3])
def test_l_layers_see_exactly_l_hops(L):
    """Message passing over in-edges: after L layers a node's output depends on
    the inputs within L hops and on none farther away.  Perturbing one node's
    input must change every node within L hops (generic weights) and no other."""
    H = 8
    m = hex_box(8, 1, 1, 1e-3)                         # a chain of cubes: long graph distances
    N = len(m.xyz)
    src, dst = mesh_edges(m.conn, N)
    d = (m.xyz[dst] - m.xyz[src]) / 1e-3
    f = np.concatenate([d, np.linalg.norm(d, axis=1, keepdims=True)], axis=1)
    rng = np.random.default_rng(7)
    flat = rng.normal(size=mpnn.n_params(H, L)) * 0.3        # moderate weights: no saturated SiLU
    x = rng.normal(size=(1, N, 5))
    y0, _ = mpnn.forward(flat, x, f, src, dst, H, L)
    start = 0
    x1 = x.copy()
    x1[0, start] += 0.3
    y1, _ = mpnn.forward(flat, x1, f, src, dst, H, L)
    changed = np.abs(y1[0] - y0[0]) > 1e-12
    dist = _hops(src, dst, N, start)
    assert np.all(changed[dist <= L]) and not np.any(changed[dist > L])
    assert np.any(dist > L)


def test_translation_and_rotation_of_the_mesh_change_nothing_that_they_should_not():
    """Edge inputs are relative positions: a translation leaves the output
    unchanged; a rotation by 90 degrees about z permutes the x/y edge inputs
    and so (for generic weights) does change it."""
    H, L = 8, 2
    m = hex_box(2, 2, 1, 1e-3)
    N = len(m.xyz)
    src, dst = mesh_edges(m.conn, N)

    def feats(xyz):
        d = (xyz[dst] - xyz[src]) / 1e-3
        return np.concatenate([d, np.linalg.norm(d, axis=1, keepdims=True)], axis=1)

    rng = np.random.default_rng(11)
    flat = rng.normal(size=mpnn.n_params(H, L)) * 0.5
    x = rng.normal(size=(2, N, 5))
    y, _ = mpnn.forward(flat, x, feats(m.xyz), src, dst, H, L)
    yt, _ = mpnn.forward(flat, x, feats(m.xyz + np.array([0.3, -0.2, 0.7])), src, dst, H, L)
    np.testing.assert_allclose(yt, y, rtol=1e-9, atol=1e-12)
    rot = m.xyz[:, [1, 0, 2]] * np.array([-1.0, 1.0, 1.0])
    yr, _ = mpnn.forward(flat, x, feats(rot), src, dst, H, L)
    assert np.max(np.abs(yr - y)) > 1e-6


def _hand_params(L):
    """Weights for the worked example (H = 2): with a = ln 3 every
    pre-activation below is 0 or +-a, and SiLU(a) = a sigma(a) = 3a/4,
    SiLU(-a) = -a/4, SiLU(0) = 0."""
    a = np.log(3.0)
    q = 4.0 / 3.0
    p = {
        "W_ne": np.array([[a, 0, 0, 0, 0], [0, -a, 0, 0, 0]]), "b_ne": np.zeros(2),
        "W_ee": np.array([[0, 0, 0, 0], [a, 0, 0, 0]]), "b_ee": np.zeros(2),
        # layer 0: message from the edge's second feature and the SOURCE node's first feature
        "W_e0": np.array([[0, q, 0, 0, 0, 0], [0, 0, q, 0, 0, 0]]), "b_e0": np.zeros(2),
        # node update: [h_i ; a_i] -> (q h_i0 + q a_i0, -q a_i1)
        "W_n0": np.array([[q, 0, q, 0], [0, 0, 0, -q]]), "b_n0": np.zeros(2),
        "w_d": np.array([1.0, 2.0]), "b_d": np.array([0.5]),
    }
    if L == 2:
        # layer 1 reads only the updated edge state e_1 (= 2 SiLU(a) after layer 0)
        p["W_e1"] = np.array([[0, 2.0 / 3.0, 0, 0, 0, 0], [0, 0, 0, 0, 0, 0]])
        p["b_e1"] = np.zeros(2)
        p["W_n1"] = np.array([[0, 0, q, 0], [0, 0, 0, 0]])
        p["b_n1"] = np.zeros(2)
    return mpnn.flatten({k: np.asarray(v, dtype=np.float64) for k, v in p.items()}, 2, L)


def test_forward_values_of_a_worked_example():
    """Two nodes, one edge 0 -> 1, H = 2; x_0 = e_1, x_1 = e_2, edge input
    f = e_1; a = ln 3, s = SiLU(a) = 3a/4, t = -SiLU(-a) = a/4.

      encoders:  h_0 = SiLU(a, 0) = (s, 0),  h_1 = SiLU(0, -a) = (0, -t),
                 e = SiLU(0, a) = (0, s)
      layer 0:   msg = SiLU(4/3 e_1, 4/3 h_src,0) = SiLU(a, a) = (s, s)
                 e <- e + msg = (s, 2s);  aggregate into node 1: a_1 = (s, s), a_0 = 0
                 z_0 = (4/3 s, 0) = (a, 0)       -> h_0 = (s, 0) + (s, 0) = (2s, 0)
                 z_1 = (4/3 s, -4/3 s) = (a, -a) -> h_1 = (0, -t) + (s, -t) = (s, -2t)
      decoder:   y_0 = 2s + 0.5 = 1.5a + 0.5,  y_1 = s - 4t + 0.5 = 0.5 - a/4

    With a second layer that reads only e_1 (2/3 e_1 = 4/3 s = a, so
    msg = (s, 0)) and adds 4/3 a_i0 to the first hidden unit: node 1 gets
    z = (a, 0) -> h_1 = (2s, -2t), node 0 is unchanged, so
    y = (1.5a + 0.5, 0.5a + 0.5).  A dropped residual, a message aggregated
    at the source, swapped source and destination, a missing edge update or
    a missing activation each changes one of these numbers."""
    a = np.log(3.0)
    x = np.zeros((1, 2, 5))
    x[0, 0, 0] = 1.0
    x[0, 1, 1] = 1.0
    f = np.array([[1.0, 0.0, 0.0, 0.0]])
    src, dst = np.array([0]), np.array([1])
    y1, _ = mpnn.forward(_hand_params(1), x, f, src, dst, H=2, L=1)
    np.testing.assert_allclose(y1[0], [1.5 * a + 0.5, 0.5 - 0.25 * a], rtol=1e-15, atol=1e-15)
    y2, _ = mpnn.forward(_hand_params(2), x, f, src, dst, H=2, L=2)
    np.testing.assert_allclose(y2[0], [1.5 * a + 0.5, 0.5 * a + 0.5], rtol=1e-15, atol=1e-15)
