"""Degenerate inputs on the GPU: a mesh of one element (one hexahedron, one
tetrahedron), insulated, heated by a source at its centre, in every kernel
against the FP64 oracle; a mesh whose every node is held (nothing to step:
the element-parallel kernels leave it as it is, the tiled kernels refuse
it); a call for zero steps."""
import numpy as np
import pytest

from oracle import Oracle, critical_dt
from synth.meshes import hex_box, kuhn_tet_box
from synth.problem import GaussianSource, Problem
from synth.scenarios import PERFUSION, TISSUE_TD

from gpu_util import ff, max_abs, run_gpu

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-9, 1e-3
H = 1e-3


def _one_element(nv):
    m = hex_box(1, 1, 1, H) if nv == 8 else kuhn_tet_box(1, 1, 1, H)
    conn = np.asarray(m.conn)[:1]
    used = np.unique(conn)
    remap = -np.ones(len(m.xyz), dtype=np.int64)
    remap[used] = np.arange(len(used))
    xyz = m.xyz[used] + np.random.default_rng(nv).uniform(-0.1 * H, 0.1 * H, (len(used), 3))
    c = xyz.mean(axis=0)
    return Problem(nv, xyz, remap[conn].astype(np.int32), TISSUE_TD, PERFUSION,
                   sources=[GaussianSource(tuple(c), 0.5e-3, 5e6)], T0=37.0, T_lo=30.0, T_hi=100.0)


@pytest.mark.parametrize("nv", [8, 4])
def test_one_element_every_kernel_against_the_oracle(nv):
    f = ff()
    p = _one_element(nv)
    orc = Oracle(p)
    dt = 0.5 * critical_dt(orc, p.T_lo, p.T_hi)
    n = 300
    ref = orc.run(dt, n)
    assert ref.max() > 37.01                       # the source heats it
    for prec, tol in ((f.FP64, TOL64), (f.FP32_KAHAN, TOL32)):
        base = None
        for kern in (f.KERNEL_TWO_PHASE, f.KERNEL_PERSISTENT, f.KERNEL_TILED, f.KERNEL_TILED_STAGED,
                     f.KERNEL_TILED_REP):
            T, _ = run_gpu(p, dt, n, prec, kernel=kern)
            err = max_abs(T, ref)
            print(f"one element nv={nv} prec {prec} kernel {kern}: max|dT| = {err:.3e}")
            assert err <= tol
            if base is None:
                base = T
            assert np.array_equal(T, base), kern


def test_every_node_held():
    f = ff()
    m = hex_box(3, 3, 3, H)
    T_dir = 37.0 + 0.125 * np.arange(len(m.xyz))   # exact in FP32 too, so the held state reads back exactly
    p = Problem(8, m.xyz, m.conn, TISSUE_TD, PERFUSION, sources=[GaussianSource((1.5e-3,) * 3, 1e-3, 5e6)],
                dirichlet_nodes=np.arange(len(m.xyz), dtype=np.int32), dirichlet_T=T_dir,
                T0=37.0, T_lo=30.0, T_hi=100.0)
    for kern in (f.KERNEL_TWO_PHASE, f.KERNEL_PERSISTENT):
        T, _ = run_gpu(p, 0.1, 20, f.FP32_KAHAN, kernel=kern)
        assert np.array_equal(T, T_dir), kern
    for kern in (f.KERNEL_TILED, f.KERNEL_TILED_STAGED, f.KERNEL_TILED_REP):
        s = f.Solver(p, precision=f.FP32_KAHAN, kernel=kern)
        try:
            with pytest.raises(f.FedfemError) as e:
                s.step(0.1, 1)
            assert e.value.code == f.E_ARG
        finally:
            s.close()


def test_zero_steps_change_nothing():
    f = ff()
    p = _one_element(8)
    s = f.Solver(p, precision=f.FP64, kernel=f.KERNEL_TILED_REP)
    try:
        before = s.temperature()
        s.step(0.01, 0)
        assert s.sync() == 0
        assert np.array_equal(s.temperature(), before)
        s.step(0.01, 5)
        assert s.sync() == 5
    finally:
        s.close()
