"""FP64 CPU reference of the message-passing surrogate (forward and backward).

Oracle code (test infrastructure only): the gradient oracle for the GPU
surrogate.  The paper only names neural networks as a direction for stable
dynamics (Section 4); the network below is the encode-process-decode graph
network the surrogate uses, written out plainly:

  h_i  = SiLU(W_ne x_i + b_ne)                    node encoder (5 -> H)
  e_m  = SiLU(W_ee f_m + b_ee)                    edge encoder (4 -> H)
  per layer l:
    msg_m = SiLU(W_e [e_m; h_src(m); h_dst(m)] + b_e)
    e_m  <- e_m + msg_m
    a_i   = sum of msg_m over edges m into i
    h_i  <- h_i + SiLU(W_n [h_i; a_i] + b_n)
  y_i  = w_d . h_i + b_d                          decoder (H -> 1)

Loss: mean over (scenario, node) with mask 1 of (y - target)^2.

The flat parameter layout (row-major matrices, in this order) is shared with
the GPU implementation's host interface: W_ne, b_ne, W_ee, b_ee, then per
layer W_e, b_e, W_n, b_n, then w_d, b_d.  Pinned by central finite
differences and permutation equivariance (tests/test_oracle_mpnn.py).
"""
from __future__ import annotations

import numpy as np

N_NODE_IN, N_EDGE_IN = 5, 4


def param_shapes(H: int = 64, L: int = 4):
    shapes = [("W_ne", (H, N_NODE_IN)), ("b_ne", (H,)), ("W_ee", (H, N_EDGE_IN)), ("b_ee", (H,))]
    for l in range(L):
        shapes += [(f"W_e{l}", (H, 3 * H)), (f"b_e{l}", (H,)), (f"W_n{l}", (H, 2 * H)), (f"b_n{l}", (H,))]
    shapes += [("w_d", (H,)), ("b_d", (1,))]
    return shapes


def n_params(H: int = 64, L: int = 4) -> int:
    return int(sum(np.prod(s) for _, s in param_shapes(H, L)))


def unflatten(flat, H: int = 64, L: int = 4) -> dict:
    out, o = {}, 0
    for name, shp in param_shapes(H, L):
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def flatten(p: dict, H: int = 64, L: int = 4) -> np.ndarray:
    return np.concatenate([p[name].ravel() for name, _ in param_shapes(H, L)])


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(flat, x, f, src, dst, H=64, L=4):
    """x: (B, N, 5) node inputs, f: (E, 4) edge inputs, src/dst: (E,).
    Returns y (B, N) and a cache for backward."""
    p = unflatten(flat, H, L)
    B, N, _ = x.shape
    E = len(src)
    cache = {"x": x, "f": f}
    z = x @ p["W_ne"].T + p["b_ne"]
    cache["z_ne"] = z
    h = silu(z)
    ze = f @ p["W_ee"].T + p["b_ee"]
    cache["z_ee"] = ze
    e = np.broadcast_to(silu(ze), (B, E, H)).copy()
    layers = []
    for l in range(L):
        Xe = np.concatenate([e, h[:, src], h[:, dst]], axis=2)
        z_e = Xe @ p[f"W_e{l}"].T + p[f"b_e{l}"]
        msg = silu(z_e)
        e = e + msg
        a = np.zeros((B, N, H))
        np.add.at(a, (slice(None), dst), msg)
        Xn = np.concatenate([h, a], axis=2)
        z_n = Xn @ p[f"W_n{l}"].T + p[f"b_n{l}"]
        h = h + silu(z_n)
        layers.append({"Xe": Xe, "z_e": z_e, "Xn": Xn, "z_n": z_n})
    cache["layers"] = layers
    cache["h"] = h
    y = h @ p["w_d"] + p["b_d"][0]
    return y, cache


def backward(flat, cache, dy, src, dst, H=64, L=4):
    """Gradient of sum(dy * y) with respect to the flat parameters."""
    p = unflatten(flat, H, L)
    g = {name: np.zeros(shp) for name, shp in param_shapes(H, L)}
    h = cache["h"]
    B, N, _ = h.shape
    E = len(src)
    g["w_d"] = np.einsum("bn,bnh->h", dy, h)
    g["b_d"] = np.array([dy.sum()])
    dh = dy[:, :, None] * p["w_d"]
    de = np.zeros((B, E, H))
    for l in reversed(range(L)):
        c = cache["layers"][l]
        dz_n = dh * dsilu(c["z_n"])
        g[f"W_n{l}"] = np.einsum("bnk,bnj->kj", dz_n, c["Xn"])
        g[f"b_n{l}"] = dz_n.sum(axis=(0, 1))
        dXn = dz_n @ p[f"W_n{l}"]
        dh_new = dh + dXn[:, :, :H]
        da = dXn[:, :, H:]
        dmsg = de + da[:, dst]
        dz_e = dmsg * dsilu(c["z_e"])
        g[f"W_e{l}"] = np.einsum("bmk,bmj->kj", dz_e, c["Xe"])
        g[f"b_e{l}"] = dz_e.sum(axis=(0, 1))
        dXe = dz_e @ p[f"W_e{l}"]
        de = de + dXe[:, :, :H]
        np.add.at(dh_new, (slice(None), src), dXe[:, :, H:2 * H])
        np.add.at(dh_new, (slice(None), dst), dXe[:, :, 2 * H:])
        dh = dh_new
    dz_ee = de.sum(axis=0) * dsilu(cache["z_ee"])
    g["W_ee"] = dz_ee.T @ cache["f"]
    g["b_ee"] = dz_ee.sum(axis=0)
    dz_ne = dh * dsilu(cache["z_ne"])
    g["W_ne"] = np.einsum("bnk,bnj->kj", dz_ne, cache["x"])
    g["b_ne"] = dz_ne.sum(axis=(0, 1))
    return flatten(g, H, L)


def loss_and_grad(flat, x, f, src, dst, target, mask, H=64, L=4):
    """MSE over masked entries and its parameter gradient."""
    y, cache = forward(flat, x, f, src, dst, H, L)
    m = np.broadcast_to(mask, y.shape)
    cnt = m.sum()
    r = (y - target) * m
    loss = float(np.sum(r * r) / cnt)
    dy = 2.0 * r / cnt
    return loss, backward(flat, cache, dy, src, dst, H, L), y
