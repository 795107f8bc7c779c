"""Error paths of the C ABI on the GPU, checkpoint/resume, device-pointer
variants.  Failures are made on the host (bad inputs, a too-narrow range) or
with bounded device waits that are made to run out (a barrier that one block
never reaches, with a short spin limit); nothing faults or hangs the GPU."""
import copy

import numpy as np
import pytest

from oracle import Oracle, critical_dt
from synth.meshes import hex_box, kuhn_tet_box
from synth.scenarios import cube_hex_fp64, cube_hex_td_convective, ellipsoid_tet_td

from gpu_util import ff, max_abs

pytestmark = pytest.mark.gpu


def _solver(p, prec=None, **kw):
    f = ff()
    return f.Solver(p, precision=f.FP32_KAHAN if prec is None else prec, **kw)


def test_call_order_and_argument_errors():
    f = ff()
    p = cube_hex_fp64().problem
    ctx = f.fedfem_create(0, f.FP64)
    try:
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_precompute(ctx, 30, 40)
        assert e.value.code == f.E_STATE
        f.fedfem_set_mesh(ctx, 8, p.xyz, p.conn)
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_init(ctx, None, 37.0)
        assert e.value.code == f.E_STATE
        m = p.material
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_set_material(ctx, m.T_ref, -1.0, 0, m.c0, 0, m.k0, 0)
        assert e.value.code == f.E_ARG
        f.fedfem_set_material(ctx, m.T_ref, m.rho0, m.drho, m.c0, m.dc, m.k0, m.dk)
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_set_dirichlet(ctx, [0, 10 ** 6], [37.0, 37.0])
        assert e.value.code == f.E_ARG
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_precompute(ctx, 40, 30)
        assert e.value.code == f.E_ARG
        dt_cr = f.fedfem_precompute(ctx, 30, 40)
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_step(ctx, 0.5 * dt_cr, 1)
        assert e.value.code == f.E_STATE
        f.fedfem_init(ctx, None, 37.0)
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_step(ctx, 1.0001 * dt_cr, 1)
        assert e.value.code == f.E_UNSTABLE_DT
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_init(ctx, np.full(p.n_nodes, np.nan))
        assert e.value.code == f.E_ARG
        f.fedfem_step(ctx, 0.999 * dt_cr, 3)
        assert f.fedfem_sync(ctx) == 3
    finally:
        f.fedfem_destroy(ctx)


def test_inverted_element_and_unused_node_are_mesh_errors():
    f = ff()
    m = kuhn_tet_box(2, 2, 2, 1e-3)
    conn = m.conn.copy()
    conn[5, [1, 2]] = conn[5, [2, 1]]            # flip the orientation of input element 5
    ctx = f.fedfem_create(0, f.FP32_KAHAN)
    try:
        f.fedfem_set_mesh(ctx, 4, m.xyz, conn)
        f.fedfem_set_material(ctx, 37, 1000, 0, 4000, 0, 0.5, 0)
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_precompute(ctx, 30, 40)
        assert e.value.code == f.E_MESH and "element 5 " in str(e.value)
        xyz = np.vstack([m.xyz, [[1.0, 1.0, 1.0]]])
        f.fedfem_set_mesh(ctx, 4, xyz, m.conn)
        f.fedfem_set_material(ctx, 37, 1000, 0, 4000, 0, 0.5, 0)
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_precompute(ctx, 30, 40)
        assert e.value.code == f.E_MESH and f"node {len(xyz) - 1}" in str(e.value)
    finally:
        f.fedfem_destroy(ctx)


def test_range_violation_stops_every_kernel_at_the_same_step():
    f = ff()
    w = cube_hex_td_convective(n=16)
    p = copy.copy(w.problem)
    p.T_hi = 38.0                                  # the source crosses this after some steps
    dt = 0.5 * critical_dt(Oracle(p), 20.0, 38.0)
    done = {}
    for kern in (f.KERNEL_TWO_PHASE, f.KERNEL_PERSISTENT, f.KERNEL_TILED, f.KERNEL_TILED_STAGED,
                 f.KERNEL_TILED_REP):
        s = _solver(p, kernel=kern)
        try:
            s.step(dt, 400)
            rc, n = f.fedfem_sync_status(s.ctx)
            assert rc == f.E_RANGE
            done[kern] = n
            assert "left [T_lo, T_hi]" in f.fedfem_last_error(s.ctx)
            T = s.temperature()
            assert T.max() > 38.0
        finally:
            s.close()
    assert len(set(done.values())) == 1 and 0 < list(done.values())[0] < 400, done


def test_barrier_timeout_is_reported_and_the_context_recovers():
    f = ff()
    p = cube_hex_td_convective(n=24).problem
    for kern in (f.KERNEL_PERSISTENT, f.KERNEL_TILED, f.KERNEL_TILED_REP):
        s = _solver(p, kernel=kern)
        try:
            dt = 0.5 * s.dt_cr
            f.fedfem_debug_set(s.ctx, 1, 20_000_000)     # ~10 ms spin limit
            f.fedfem_debug_set(s.ctx, 2, 3)              # block 3 never arrives
            s.init()
            s.step(dt, 20)
            rc, n = f.fedfem_sync_status(s.ctx)
            assert rc == f.E_TIMEOUT, rc
            f.fedfem_debug_set(s.ctx, 2, -1)
            s.init()
            s.step(dt, 20)
            assert s.sync() == 20
        finally:
            s.close()


@pytest.mark.parametrize("prec_name", ["FP64", "FP32_KAHAN"])
def test_checkpoint_resume_is_bit_identical(prec_name):
    f = ff()
    prec = getattr(f, prec_name)
    p = ellipsoid_tet_td(h=2e-3, axes=(0.024, 0.018, 0.014)).problem
    straight = _solver(p, prec, kernel=f.KERNEL_TILED)
    try:
        dt = 0.5 * straight.dt_cr
        straight.step(dt, 87)
        straight.sync()
        ref = straight.temperature()
    finally:
        straight.close()
    a = _solver(p, prec, kernel=f.KERNEL_TILED)
    try:
        a.step(dt, 37)
        a.sync()
        state = f.fedfem_get_state(a.ctx)
    finally:
        a.close()
    b = _solver(p, prec, kernel=f.KERNEL_PERSISTENT)
    try:
        f.fedfem_set_state(b.ctx, state)
        assert b.info()["steps_done"] == 37
        b.step(dt, 50)
        assert b.sync() == 87
        assert np.array_equal(b.temperature(), ref)
        with pytest.raises(f.FedfemError):
            f.fedfem_set_state(b.ctx, state[:-8])
    finally:
        b.close()


def test_device_pointer_init_and_read():
    import torch
    f = ff()
    p = cube_hex_fp64().problem
    s = _solver(p, f.FP64)
    try:
        dev = torch.device("cuda", 0)
        T0 = torch.linspace(36.0, 38.0, p.n_nodes, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()                   # the context has its own stream
        f.fedfem_init_device(s.ctx, T0.data_ptr())
        out = torch.empty(p.n_nodes, dtype=torch.float64, device=dev)
        f.fedfem_read_temperature_device(s.ctx, out.data_ptr())
        expect = T0.cpu().numpy().copy()
        expect[p.dirichlet_nodes] = 37.0
        assert np.array_equal(out.cpu().numpy(), expect)
        assert np.array_equal(s.temperature(), expect)
    finally:
        s.close()


def test_non_finite_initial_field_is_refused_and_changes_nothing():
    """The initial field is checked on the device after its copy: one NaN or
    infinity anywhere (here the last node, and a node in the middle) gives
    E_ARG through the host and the device entry points, and the field and
    the step counter stay those of the last good init."""
    import torch
    f = ff()
    p = cube_hex_fp64().problem
    s = _solver(p, f.FP64)
    try:
        dt = 0.5 * s.dt_cr
        s.step(dt, 5)
        assert s.sync() == 5
        before = s.temperature()
        dev = torch.device("cuda", 0)
        for pos, bad in ((p.n_nodes - 1, np.nan), (p.n_nodes // 2, np.inf)):
            T0 = np.full(p.n_nodes, 37.0)
            T0[pos] = bad
            with pytest.raises(f.FedfemError) as e:
                f.fedfem_init(s.ctx, T0)
            assert e.value.code == f.E_ARG
            Td = torch.tensor(T0, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            with pytest.raises(f.FedfemError) as e:
                f.fedfem_init_device(s.ctx, Td.data_ptr())
            assert e.value.code == f.E_ARG
            assert np.array_equal(s.temperature(), before)
        s.step(dt, 3)                              # the context goes on from the last good state
        assert s.sync() == 8
    finally:
        s.close()


def test_refused_tile_size_leaves_the_context_usable():
    """A tile whose shared memory no block can hold is refused with
    E_UNSUPPORTED; the refusal must not surface as an error in later calls."""
    f = ff()
    p = cube_hex_td_convective(n=24).problem
    s = _solver(p, kernel=f.KERNEL_PERSISTENT)
    try:
        dt = 0.5 * s.dt_cr
        f.fedfem_set_tile(s.ctx, f.KERNEL_TILED_STAGED, 1024, 4096, 0)   # two stages of ~200 KB
        with pytest.raises(f.FedfemError) as e:
            s.step(dt, 5)
        assert e.value.code == f.E_UNSUPPORTED
        f.fedfem_set_tile(s.ctx, f.KERNEL_PERSISTENT)
        s.init()
        s.step(dt, 5)
        assert s.sync() == 5
    finally:
        s.close()
