"""Learned surrogate for the FED-FEM time loop, with the plain path as judge
and fallback.

The paper points to neural networks as a route to stable dynamics (Section
4) and to treatment planning as its next use (Section 5).  Here a message-
passing network (csrc/mpnn.cu, tensor-core BF16 GEMMs) learns to advance the
field by ``window`` explicit steps at once from trajectories that the plain
FED-FEM path itself generates; at inference every ``check_every`` surrogate
steps one surrogate step is re-done by the plain path from the same state,
and a scenario whose check exceeds the local error budget runs the rest of
that stretch on the plain path.

All arithmetic runs in the library's kernels; this module only arranges
device buffers (PyTorch) and calls the C ABI.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import fedfem as ff


def graph_edges(conn: np.ndarray, n_nodes: int):
    """Directed edges between nodes sharing an element, sorted by (dst, src)."""
    conn = np.asarray(conn, dtype=np.int64)
    nv = conn.shape[1]
    a = np.repeat(conn, nv, axis=1).ravel()
    b = np.tile(conn, (1, nv)).ravel()
    keep = a != b
    key = np.unique(b[keep] * n_nodes + a[keep])
    return (key % n_nodes).astype(np.int32), (key // n_nodes).astype(np.int32)


class PlainEnsemble:
    """S scenarios of one problem that differ only in their source density,
    stepped together by the plain path: copies of the mesh as element groups,
    4 scenarios per copy as lanes.  States move in and out as S x N float64
    device tensors (input node order)."""

    def __init__(self, problem, q_r: np.ndarray, stream=None, precision=ff.FP32_KAHAN, T_lo=None, T_hi=None):
        import torch
        p = problem
        self.S, self.N = q_r.shape
        self.G = math.ceil(self.S / 4)
        G, N = self.G, self.N
        xyz = np.tile(p.xyz, (G, 1))
        conn = (np.asarray(p.conn, dtype=np.int64)[None] + (np.arange(G) * N)[:, None, None]).reshape(-1, p.conn.shape[1])
        groups = np.repeat(np.arange(G, dtype=np.int32), len(p.conn))
        dn = (np.asarray(p.dirichlet_nodes, dtype=np.int64)[None] + (np.arange(G) * N)[:, None]).ravel()
        dT = np.tile(np.asarray(p.dirichlet_T, dtype=np.float64), G)
        qpad = np.zeros((4 * G, N))
        qpad[: self.S] = q_r
        self.ctx = ff.fedfem_create(0, precision, stream)
        ff.fedfem_set_mesh(self.ctx, p.elem_type, xyz, conn)
        ff.fedfem_set_element_groups(self.ctx, groups)
        ff.fedfem_set_lanes(self.ctx, 4)
        ff.apply_material(self.ctx, p.material)
        pf = p.perfusion
        ff.fedfem_set_perfusion(self.ctx, pf.w_b, pf.c_b, pf.T_a, pf.Q_m)
        ff.fedfem_set_dirichlet(self.ctx, dn, dT)
        for lane in range(4):   # lane l of copy g is scenario 4 g + l
            ff.fedfem_set_source_lane(self.ctx, lane, qpad.reshape(G, 4, N)[:, lane].ravel())
        ff.fedfem_set_tile(self.ctx, ff.KERNEL_TILED)
        self.dt_cr = ff.fedfem_precompute(self.ctx, p.T_lo if T_lo is None else T_lo, p.T_hi if T_hi is None else T_hi)
        ff.fedfem_init(self.ctx, None, float(np.asarray(p.T0).ravel()[0]))
        self._lanes = torch.empty((4, G * N), dtype=torch.float64, device="cuda")

    def set_state(self, T):
        """T: S x N float64 CUDA tensor."""
        import torch
        G, N = self.G, self.N
        full = torch.zeros((4 * G, N), dtype=torch.float64, device=T.device)
        full[: self.S] = T
        self._lanes.copy_(full.view(G, 4, N).permute(1, 0, 2).reshape(4, G * N))
        torch.cuda.synchronize()          # the context works on its own stream
        ff.fedfem_init_lanes_device(self.ctx, self._lanes.data_ptr())

    def step(self, dt, n):
        ff.fedfem_step(self.ctx, dt, n)

    def state(self):
        ff.fedfem_read_lanes_device(self.ctx, self._lanes.data_ptr())
        G, N = self.G, self.N
        return self._lanes.view(4, G, N).permute(1, 0, 2).reshape(4 * G, N)[: self.S].clone()

    def close(self):
        if self.ctx:
            ff.fedfem_destroy(self.ctx)
            self.ctx = None


class Surrogate:
    """The network plus the problem data it needs (mesh graph, Dirichlet
    mask, material laws for the inputs).  ``y`` is the change of T over
    ``window`` explicit steps in degC; Dirichlet nodes are held."""

    def __init__(self, problem, window: int = 50, layers: int = 4, max_batch: int = 64, seed: int = 0,
                 stream=None, length_scale: float | None = None):
        import torch
        p = problem
        self.p, self.window, self.max_batch = p, window, max_batch
        self.N = p.n_nodes
        src, dst = graph_edges(p.conn, self.N)
        self.n_edges = len(src)
        if length_scale is None:
            length_scale = float(np.median(np.linalg.norm(p.xyz[dst] - p.xyz[src], axis=1)))
        self.net = ff.fedfem_mpnn_create(self.N, src, dst, p.xyz, length_scale, layers=layers, max_batch=max_batch,
                                         cuda_stream=stream)
        self.n_params = ff.fedfem_mpnn_n_params(self.net)
        rng = np.random.default_rng(seed)
        H = 64
        shapes = [(H, 5), (H,), (H, 4), (H,)] + [(H, 3 * H), (H,), (H, 2 * H), (H,)] * layers
        parts = []
        for s in shapes:      # weights U(-1, 1)/sqrt(fan_in), biases 0
            parts.append(rng.uniform(-1, 1, s).ravel() / math.sqrt(s[1]) if len(s) == 2 else np.zeros(s[0]))
        parts.append(0.1 * rng.uniform(-1, 1, H) / math.sqrt(H))    # small initial decoder
        parts.append(np.zeros(1))
        params = np.concatenate(parts).astype(np.float32)
        assert params.size == self.n_params
        ff.fedfem_mpnn_set_params(self.net, params)
        D = np.zeros(self.N, dtype=np.uint8)
        D[np.asarray(p.dirichlet_nodes, dtype=np.int64)] = 1
        self.D = torch.tensor(D, device="cuda")
        self.free = torch.tensor((1 - D).astype(np.float32), device="cuda")
        m = p.material
        if m.table is not None or p.regions is not None:
            raise ValueError("the surrogate's input features take one material with linear laws")
        self.mat = (m.T_ref, m.rho0, m.drho, m.c0, m.dc, m.k0, m.dk)
        self._x = torch.empty((max_batch, self.N, 5), device="cuda")
        self._y = torch.empty((max_batch, self.N), device="cuda")

    def _features(self, T, q):
        B = T.shape[0]
        ff.fedfem_mpnn_features(self.net, B, T.data_ptr(), q.data_ptr(), self.D.data_ptr(), self.mat,
                                self._x.data_ptr())
        return self._x[:B]

    def predict(self, T, q):
        """T, q: B x N float32 CUDA tensors (any B; chunks of max_batch).
        Returns T after ``window`` steps (float32)."""
        import torch
        out = torch.empty_like(T)
        for b0 in range(0, T.shape[0], self.max_batch):
            Tb, qb = T[b0:b0 + self.max_batch].contiguous(), q[b0:b0 + self.max_batch].contiguous()
            B = Tb.shape[0]
            x = self._features(Tb, qb)
            ff.fedfem_mpnn_infer(self.net, B, x.data_ptr(), self._y.data_ptr())
            out[b0:b0 + B] = Tb + self._y[:B] * self.free
        return out

    def train(self, T_in, q, T_out, epochs: int = 2, batch: int = 32, lr: float = 1e-3, seed: int = 0,
              lr_final: float = 1e-4, log=None):
        """Minimise the mean squared error of y against T_out - T_in over free
        nodes.  Inputs: P x N float32 CUDA tensors.  Returns the loss history."""
        import torch
        P = T_in.shape[0]
        rng = np.random.default_rng(seed)
        steps = epochs * (P // batch)
        losses, it = [], 0
        t0 = time.perf_counter()
        for ep in range(epochs):
            order = torch.tensor(rng.permutation(P), device="cuda")
            for b0 in range(0, P - batch + 1, batch):
                idx = order[b0:b0 + batch]
                Tb, qb = T_in[idx].contiguous(), q[idx].contiguous()
                target = (T_out[idx] - Tb).contiguous()
                x = self._features(Tb, qb)
                loss, _ = ff.fedfem_mpnn_loss_grad(self.net, batch, x.data_ptr(), target.data_ptr(),
                                                   self.free.data_ptr())
                # cosine decay from lr to lr_final
                frac = it / max(1, steps - 1)
                ff.fedfem_mpnn_adam(self.net, lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * frac)))
                losses.append(loss)
                it += 1
                if log and it % 500 == 0:
                    log(f"epoch {ep} iter {it}/{steps} loss {np.mean(losses[-500:]):.3e} "
                        f"({time.perf_counter() - t0:.1f} s)")
        return losses

    def close(self):
        if self.net:
            ff.fedfem_mpnn_destroy(self.net)
            self.net = None


@dataclass
class RolloutResult:
    T: object                    # final temperatures, S x N float64
    wall_s: float
    checks: int
    rejected: int                # scenario-windows that fell back to the plain path
    surrogate_steps: int         # surrogate steps taken (scenario count x steps)
    max_check_error: float


def rollout(sur: Surrogate, ens: PlainEnsemble, q32, T0, dt: float, n_windows: int, check_every: int = 10,
            budget: float = 0.005):
    """Advance S scenarios by n_windows * check_every * window explicit steps.
    At the start of each stretch of ``check_every`` surrogate steps, one
    surrogate step is compared with ``window`` plain steps from the same state
    (the plain result is kept); a scenario whose difference exceeds ``budget``
    degC runs the whole stretch on the plain path."""
    import torch
    W = sur.window
    S = T0.shape[0]
    T = T0.clone()
    checks = rejected = sur_steps = 0
    worst = 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_windows):
        P1 = sur.predict(T.float(), q32).double()
        ens.set_state(T)
        ens.step(dt, W)
        R1 = ens.state()
        err = (P1 - R1).abs().amax(dim=1)
        checks += S
        worst = max(worst, float(err.max()))
        bad = ~(err <= budget)            # NaN fails too
        nbad = int(bad.sum())
        rejected += nbad
        T = R1
        if nbad:
            ens.step(dt, (check_every - 1) * W)          # plain path for the rest of the stretch
            Rp = ens.state()
        Ts = T
        good = ~bad
        if int(good.sum()):
            for _ in range(check_every - 1):
                Ts = sur.predict(Ts.float(), q32).double()
            sur_steps += int(good.sum()) * (check_every - 1)
        T = torch.where(bad[:, None], Rp, Ts) if nbad else Ts
    torch.cuda.synchronize()
    ff.fedfem_mpnn_sync(sur.net)   # a tensor-core wait that gave up is an error
    return RolloutResult(T, time.perf_counter() - t0, checks, rejected, sur_steps, worst)
