"""fedfem_step_static, the entry point for callers that may not allocate
device memory, against the ordinary context path (fedfem_step, FP64) and the
FP64 CPU oracle.

The caller owns every buffer (here: torch tensors); the library keeps its
temporaries in one fixed device array.  Two calls in a row must continue
each other exactly like one context that steps twice, within the FP64
tolerance of the parity tests (1e-9 degC).  A defective mesh or gather must
come back as FEDFEM_E_MESH with the caller's temperatures untouched."""
import numpy as np
import pytest

from gpu_util import ff, max_abs

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-9


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


class _Buffers:
    """The caller's device buffers of one problem."""

    def __init__(self, p, conn=None, row_ptr=None, slots=None):
        import torch
        dev = torch.device("cuda", 0)
        conn = p.conn if conn is None else conn
        if row_ptr is None:
            row_ptr, slots = _gather_csr(p.conn, p.n_nodes)
        self.nv = conn.shape[1]
        self.n_nodes, self.n_elems = p.n_nodes, len(conn)
        self.xyz = torch.tensor(p.xyz, dtype=torch.float64, device=dev).contiguous()
        self.conn = torch.tensor(np.ascontiguousarray(conn), dtype=torch.int32, device=dev)
        self.rp = torch.tensor(row_ptr, device=dev)
        self.sl = torch.tensor(slots, device=dev)
        self.qr = torch.tensor(_gauss(p.xyz, p.sources), dtype=torch.float64, device=dev)
        held = np.zeros(p.n_nodes, dtype=np.uint8)
        held[p.dirichlet_nodes] = 1
        self.held = torch.tensor(held, device=dev)
        T0 = np.full(p.n_nodes, float(p.T0))
        T0[p.dirichlet_nodes] = p.dirichlet_T
        self.T = torch.tensor(T0, dtype=torch.float64, device=dev)
        m, pf = p.material, p.perfusion
        self.mat = (m.T_ref, m.rho0, m.drho, m.c0, m.dc, m.k0, m.dk)
        self.perf = (pf.w_b, pf.c_b, pf.T_a, pf.Q_m)
        self.stream = torch.cuda.current_stream(dev).cuda_stream

    def step(self, dt, n):
        ff().fedfem_step_static(self.nv, self.n_nodes, self.n_elems, self.xyz.data_ptr(), self.conn.data_ptr(),
                                self.rp.data_ptr(), self.sl.data_ptr(), self.mat, self.perf, self.qr.data_ptr(),
                                self.held.data_ptr(), dt, n, self.T.data_ptr(), self.stream)


def _small_tet_td():
    """Jittered Kuhn-tet box (6 x 5 x 4 voxels of 1 mm) with the ellipsoid's
    temperature-dependent k(T), c(T), perfusion, a source and Dirichlet on
    two faces."""
    from synth.meshes import box_face_nodes, kuhn_tet_box
    from synth.problem import GaussianSource, Problem
    from synth.scenarios import PERFUSION, TISSUE_TD
    m = kuhn_tet_box(6, 5, 4, 1e-3)
    rng = np.random.default_rng(7)
    xyz = m.xyz + rng.uniform(-0.2e-3, 0.2e-3, m.xyz.shape)
    dn = box_face_nodes(m, ("x0", "z0"))
    return Problem(4, xyz, m.conn, TISSUE_TD, PERFUSION,
                   sources=[GaussianSource((3e-3, 2.5e-3, 2e-3), 1.5e-3, 8e6)],
                   dirichlet_nodes=dn, dirichlet_T=np.full(len(dn), 37.0), T0=37.0, T_lo=30.0, T_hi=100.0)


def _two_calls_against_context_and_oracle(p, n_per_call, min_peak):
    from oracle import Oracle, critical_dt
    f = ff()
    ref = f.Solver(p, precision=f.FP64, kernel=f.KERNEL_TWO_PHASE)
    orc = Oracle(p)
    dt = 0.5 * critical_dt(orc)
    buf = _Buffers(p)
    T_orc = orc.initial_field()
    try:
        for call in range(2):
            buf.step(dt, n_per_call)
            ref.step(dt, n_per_call)
            ref.sync()
            T_orc = orc.run(dt, n_per_call, T_orc)
            got = buf.T.cpu().numpy()
            e_ctx, e_orc = max_abs(got, ref.temperature()), max_abs(got, T_orc)
            print(f"call {call + 1}: max|dT| static vs context = {e_ctx:.3e}, vs oracle = {e_orc:.3e}")
            assert e_ctx <= TOL_FP64
            assert e_orc <= TOL_FP64
        assert float(buf.T.max()) > min_peak     # the source really heated the mesh
    finally:
        ref.close()


def test_static_entry_point_hex8_matches_context_path_and_oracle_on_two_calls():
    from synth.scenarios import cube_hex_fp64
    _two_calls_against_context_and_oracle(cube_hex_fp64().problem, 150, 40.0)


def test_static_entry_point_tet4_td_matches_context_path_and_oracle_on_two_calls():
    _two_calls_against_context_and_oracle(_small_tet_td(), 200, 38.0)


def test_static_entry_point_leaves_T_unchanged_on_an_inverted_element():
    from synth.scenarios import cube_hex_fp64
    f = ff()
    p = cube_hex_fp64().problem
    conn = p.conn.copy()
    e = len(conn) // 2
    conn[e] = conn[e][[1, 0, 3, 2, 5, 4, 7, 6]]       # mirrored: det J < 0
    buf = _Buffers(p, conn=conn)
    buf.T += 0.25                                     # a field no step would keep
    before = buf.T.cpu().numpy()
    with pytest.raises(f.FedfemError) as ei:
        buf.step(1.0, 20)
    assert ei.value.code == f.E_MESH
    assert np.array_equal(buf.T.cpu().numpy(), before)


def test_static_entry_point_rejects_bad_indices_without_reading_through_them():
    from synth.scenarios import cube_hex_fp64
    f = ff()
    p = cube_hex_fp64().problem
    row_ptr, slots = _gather_csr(p.conn, p.n_nodes)
    cases = {}
    c = p.conn.copy()
    c[3, 2] = p.n_nodes + 5                          # corner beyond the node count
    cases["corner"] = (c, row_ptr, slots)
    s = slots.copy()
    s[10] = len(p.conn) * 8 + 100                    # slot beyond the element slots
    cases["slot"] = (p.conn, row_ptr, s)
    r = row_ptr.copy()
    r[-1] += 7                                       # gather longer than the slots
    cases["row_ptr"] = (p.conn, r, slots)
    s2 = slots.copy()
    s2[[20, 21]] = s2[[21, 20]]                      # a row out of element order
    cases["order"] = (p.conn, row_ptr, s2)
    for name, (cn, rp, sl) in cases.items():
        buf = _Buffers(p, conn=cn, row_ptr=rp, slots=sl)
        before = buf.T.cpu().numpy()
        with pytest.raises(f.FedfemError) as ei:
            buf.step(1.0, 5)
        assert ei.value.code == f.E_MESH, name
        assert np.array_equal(buf.T.cpu().numpy(), before), name
    # the shared array recovers: a good call right after the failures
    _two_calls_against_context_and_oracle(p, 20, 37.0)


def test_static_entry_point_rejects_meshes_beyond_its_scratch():
    f = ff()
    with pytest.raises(f.FedfemError) as ei:
        f.fedfem_step_static(8, 200000, 150000, 1, 1, 1, 1, (37, 1, 0, 1, 0, 1, 0), (0, 0, 37, 0),
                             0, 0, 1.0, 1, 1, 0)
    assert ei.value.code == f.E_ARG
