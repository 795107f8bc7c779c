"""The fully integrated hexahedron (2 x 2 x 2 Gauss points) on the GPU against
the FP64 oracle: the 11^3 cube and a distorted hex mesh, both precisions, the
critical step, the element-parallel kernels, and the refusals."""
import copy

import numpy as np
import pytest

from oracle import Oracle, critical_dt
from synth.meshes import box_face_nodes
from synth.scenarios import cube_hex_fp64

from gpu_util import ff, max_abs, run_gpu

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-9, 1e-3


def _problem(distorted):
    p = copy.copy(cube_hex_fp64().problem)
    p.hex_rule = "full"
    if distorted:   # interior nodes moved by up to 0.2 h (faces stay planar: Dirichlet boundary unchanged)
        rng = np.random.default_rng(5)
        xyz = p.xyz.copy()
        inner = np.ones(len(xyz), bool)
        inner[np.asarray(p.dirichlet_nodes)] = False
        xyz[inner] += rng.uniform(-0.2e-3, 0.2e-3, size=(int(inner.sum()), 3))
        p.xyz = xyz
    return p


@pytest.fixture(scope="module", params=[False, True], ids=["cube", "distorted"])
def case(request):
    p = _problem(request.param)
    orc = Oracle(p)
    dt_cr = critical_dt(orc)
    dt = 0.5 * dt_cr
    return request.param, p, dt_cr, dt, orc.run(dt, 600)


@pytest.mark.parametrize("prec_name", ["FP64", "FP32_KAHAN"])
def test_full_hex_matches_the_oracle(case, prec_name):
    distorted, p, dt_cr, dt, ref = case
    f = ff()
    T, info = run_gpu(p, dt, 600, getattr(f, prec_name))
    assert info["dt_cr"] == pytest.approx(dt_cr, rel=1e-9)
    err = max_abs(T, ref)
    one_point = copy.copy(p)
    one_point.hex_rule = "one-point"
    gap = max_abs(Oracle(one_point).run(dt, 600), ref)
    print(f"full hex ({'distorted' if distorted else 'cube'}) {prec_name}: max|dT| = {err:.3e}; "
          f"one-point vs full {gap:.3e} degC; dt_cr {dt_cr:.4f} s")
    assert gap > 1e-6                              # the rules differ on these fields
    assert err <= (TOL64 if prec_name == "FP64" else TOL32)


def test_element_parallel_kernels_agree_and_tiled_ones_refuse(case):
    _, p, _, dt, _ = case
    f = ff()
    T0, _ = run_gpu(p, dt, 200, f.FP32_KAHAN, kernel=f.KERNEL_PERSISTENT)
    T1, _ = run_gpu(p, dt, 200, f.FP32_KAHAN, kernel=f.KERNEL_TWO_PHASE)
    assert np.array_equal(T0, T1)
    for kern in (f.KERNEL_TILED, f.KERNEL_TILED_STAGED):
        s = f.Solver(p, precision=f.FP32_KAHAN, kernel=kern)
        try:
            with pytest.raises(f.FedfemError) as e:
                s.step(dt, 1)
            assert e.value.code == f.E_UNSUPPORTED
        finally:
            s.close()


def test_hex_rule_argument_is_checked():
    f = ff()
    p = copy.copy(cube_hex_fp64().problem)
    s = f.Solver(p, precision=f.FP64)
    try:
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_set_hex_integration(s.ctx, 2)
        assert e.value.code == f.E_ARG
    finally:
        s.close()
