"""fedfem_step_static, the entry point for callers that may not allocate
device memory, against the ordinary context path (fedfem_step, FP64).

The caller owns every buffer (here: torch tensors); the library keeps its
temporaries in one fixed device array.  Two calls in a row must continue
each other exactly like one context that steps twice, within the FP64
tolerance of the parity tests (1e-9 degC)."""
import numpy as np
import pytest

from gpu_util import ff, max_abs

pytestmark = pytest.mark.gpu


def _gather_csr(conn, n_nodes):
    """Node -> (element, corner) slots, each row sorted by element id."""
    E, nv = conn.shape
    nodes = conn.ravel().astype(np.int64)
    slots = np.arange(E * nv, dtype=np.int64)
    order = np.lexsort((slots, nodes))          # by node, then by slot (= by element)
    row_ptr = np.zeros(n_nodes + 1, dtype=np.int64)
    np.add.at(row_ptr, nodes + 1, 1)
    return np.cumsum(row_ptr).astype(np.int32), slots[order].astype(np.int32)


def _gauss(xyz, sources):
    q = np.zeros(len(xyz))
    for s in sources:
        q += s.peak * np.exp(-np.sum((xyz - np.asarray(s.x0)) ** 2, axis=1) / (2 * s.sigma ** 2))
    return q


def test_static_entry_point_matches_context_path_on_two_calls():
    import torch
    from synth.scenarios import cube_hex_fp64
    f = ff()
    w = cube_hex_fp64()
    p = w.problem
    ref = f.Solver(p, precision=f.FP64, kernel=f.KERNEL_TWO_PHASE)
    dt = 0.5 * ref.dt_cr
    dev = torch.device("cuda", 0)
    row_ptr, slots = _gather_csr(p.conn, p.n_nodes)
    xyz = torch.tensor(p.xyz, dtype=torch.float64, device=dev).contiguous()
    conn = torch.tensor(p.conn, dtype=torch.int32, device=dev).contiguous()
    rp = torch.tensor(row_ptr, device=dev)
    sl = torch.tensor(slots, device=dev)
    qr = torch.tensor(_gauss(p.xyz, p.sources), dtype=torch.float64, device=dev)
    held = np.zeros(p.n_nodes, dtype=np.uint8)
    held[p.dirichlet_nodes] = 1
    held_t = torch.tensor(held, device=dev)
    T0 = np.full(p.n_nodes, 37.0)
    T0[p.dirichlet_nodes] = p.dirichlet_T
    T = torch.tensor(T0, dtype=torch.float64, device=dev)
    m, pf = p.material, p.perfusion
    mat = (m.T_ref, m.rho0, m.drho, m.c0, m.dc, m.k0, m.dk)
    perf = (pf.w_b, pf.c_b, pf.T_a, pf.Q_m)
    stream = torch.cuda.current_stream(dev).cuda_stream
    try:
        for call in range(2):
            f.fedfem_step_static(8, p.n_nodes, len(p.conn), xyz.data_ptr(), conn.data_ptr(), rp.data_ptr(),
                                 sl.data_ptr(), mat, perf, qr.data_ptr(), held_t.data_ptr(), dt, 150,
                                 T.data_ptr(), stream)
            ref.step(dt, 150)
            ref.sync()
            err = max_abs(T.cpu().numpy(), ref.temperature())
            print(f"call {call + 1}: max|dT| static vs context = {err:.3e}")
            assert err <= 1e-9
        assert float(T.max()) > 40.0       # the source really heated the cube
    finally:
        ref.close()


def test_static_entry_point_rejects_meshes_beyond_its_scratch():
    f = ff()
    with pytest.raises(f.FedfemError) as ei:
        f.fedfem_step_static(8, 200000, 150000, 1, 1, 1, 1, (37, 1, 0, 1, 0, 1, 0), (0, 0, 37, 0),
                             0, 0, 1.0, 1, 1, 0)
    assert ei.value.code == f.E_ARG
