"""The GPU surrogate network (tensor-core BF16 GEMMs, FP32 accumulation)
against the FP64 CPU reference network: forward values, loss, and the
gradient of every parameter tensor (relative error <= 2e-2, cosine >= 0.999),
plus determinism and a training step that lowers the loss."""
import numpy as np
import pytest

from oracle import mpnn as ref
from synth.graph import mesh_edges
from synth.meshes import hex_box

from gpu_util import ff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    m = hex_box(10, 10, 10, 1e-3)
    N = len(m.xyz)
    src, dst = mesh_edges(m.conn, N)
    rng = np.random.default_rng(0)
    params = np.concatenate([rng.uniform(-1, 1, int(np.prod(s))) / np.sqrt(s[-1] if len(s) > 1 else 64)
                             for _, s in ref.param_shapes()]).astype(np.float32)
    B = 3
    x = rng.normal(size=(B, N, 5)).astype(np.float32)
    target = rng.normal(size=(B, N)).astype(np.float32) * 0.5
    mask = (rng.random(N) > 0.1).astype(np.float32)
    d = (m.xyz[dst] - m.xyz[src]) / 1e-3
    f = np.concatenate([d, np.linalg.norm(d, axis=1, keepdims=True)], axis=1)
    dev = torch.device("cuda", 0)
    t = {k: torch.tensor(v, device=dev) for k, v in (("x", x), ("target", target), ("mask", mask))}
    return dict(mesh=m, N=N, src=src, dst=dst, params=params, B=B, x=x, target=target, mask=mask, f=f, t=t)


def _net(s, max_batch=4):
    f = ff()
    net = f.fedfem_mpnn_create(s["N"], s["src"], s["dst"], s["mesh"].xyz, 1e-3, layers=4, max_batch=max_batch)
    f.fedfem_mpnn_set_params(net, s["params"])
    return net


def test_forward_and_gradients_match_fp64_reference(setup):
    import torch
    s = setup
    f = ff()
    net = _net(s)
    try:
        y = torch.empty((s["B"], s["N"]), device="cuda")
        f.fedfem_mpnn_forward(net, s["B"], s["t"]["x"].data_ptr(), y.data_ptr())
        loss, g = f.fedfem_mpnn_loss_grad(net, s["B"], s["t"]["x"].data_ptr(), s["t"]["target"].data_ptr(),
                                          s["t"]["mask"].data_ptr(), want_grad=True)
        assert np.array_equal(f.fedfem_mpnn_get_params(net), s["params"])
    finally:
        f.fedfem_mpnn_destroy(net)
    lref, gref, yref = ref.loss_and_grad(s["params"].astype(np.float64), s["x"].astype(np.float64), s["f"],
                                         s["src"], s["dst"], s["target"].astype(np.float64), s["mask"])
    yg = y.cpu().numpy()
    print(f"forward: max|y-yref| = {np.abs(yg - yref).max():.3e} (|yref| max {np.abs(yref).max():.2f}); "
          f"loss {loss:.6f} vs {lref:.6f}")
    assert np.abs(yg - yref).max() <= 2e-2 * max(1.0, np.abs(yref).max())
    assert abs(loss - lref) <= 2e-2 * lref
    o = 0
    for name, shp in ref.param_shapes():
        n = int(np.prod(shp))
        a, b = g[o:o + n].astype(np.float64), gref[o:o + n]
        o += n
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        cos = a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
        print(f"{name:6s} rel {rel:.2e} cos {cos:.6f}")
        assert rel <= 2e-2 and cos >= 0.999, name


def test_gradient_is_deterministic_and_adam_lowers_the_loss(setup):
    s = setup
    f = ff()
    net = _net(s)
    try:
        args = (s["B"], s["t"]["x"].data_ptr(), s["t"]["target"].data_ptr(), s["t"]["mask"].data_ptr())
        l1, g1 = f.fedfem_mpnn_loss_grad(net, *args, want_grad=True)
        l2, g2 = f.fedfem_mpnn_loss_grad(net, *args, want_grad=True)
        assert l1 == l2 and np.array_equal(g1, g2)
        losses = []
        for _ in range(60):
            l, _ = f.fedfem_mpnn_loss_grad(net, *args)
            f.fedfem_mpnn_adam(net, 1e-3)
            losses.append(l)
        print(f"training on random targets: loss {losses[0]:.4f} -> {losses[-1]:.4f}")
        assert losses[-1] < 0.9 * losses[0]
    finally:
        f.fedfem_mpnn_destroy(net)


@pytest.mark.parametrize("B", [1, 3])
def test_fused_inference_equals_training_forward(setup, B):
    """The fused inference kernels (gathered tensor-core tiles, message sums in
    the epilogue) round at the same points and sum in the same order as the
    unfused training forward, so the outputs agree exactly; both also match the
    FP64 reference within the BF16 bound of the forward test."""
    import torch
    s = setup
    f = ff()
    net = _net(s)
    try:
        x = s["t"]["x"][:B].contiguous()
        y_train = torch.empty((B, s["N"]), device="cuda")
        y_fused = torch.full((B, s["N"]), float("nan"), device="cuda")
        f.fedfem_mpnn_forward(net, B, x.data_ptr(), y_train.data_ptr())
        f.fedfem_mpnn_infer(net, B, x.data_ptr(), y_fused.data_ptr())
        f.fedfem_mpnn_sync(net)
        # a second call must not depend on state left by the first
        y_again = torch.full((B, s["N"]), float("nan"), device="cuda")
        f.fedfem_mpnn_infer(net, B, x.data_ptr(), y_again.data_ptr())
        f.fedfem_mpnn_sync(net)
    finally:
        f.fedfem_mpnn_destroy(net)
    diff = (y_fused - y_train).abs().max().item()
    print(f"fused vs training forward: max|dy| = {diff:.3e}")
    assert torch.equal(y_fused, y_again)
    assert torch.equal(y_fused, y_train), diff
    yref, _ = ref.forward(s["params"].astype(np.float64), s["x"][:B].astype(np.float64), s["f"], s["src"], s["dst"])
    assert np.abs(y_fused.cpu().numpy() - yref).max() <= 2e-2 * max(1.0, np.abs(yref).max())
