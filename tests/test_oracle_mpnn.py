"""Pins of the surrogate's FP64 reference network (the gradient oracle):
central finite differences and permutation equivariance."""
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
