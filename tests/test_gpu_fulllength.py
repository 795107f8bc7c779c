"""Whole runs against the FP64 oracle for the full step counts of the
workloads, at sizes the oracle steps in well under a minute:

* the temperature-dependent tet ellipsoid recipe (jittered Kuhn tets, three
  seeded Gaussian sources, perfusion, surface Dirichlet) shrunk to semi-axes
  12/9/7 mm (4,013 nodes), for the full 2e4 steps;
* the convective cube recipe (film on z = max, Dirichlet on five faces,
  temperature-dependent k and c) on 12^3 elements, for the full 1e4 steps.

Every kernel family that takes the problem runs it: FP64 within 1e-9 degC and
FP32 + Kahan within 1e-3 degC of the oracle, max over all nodes."""
import numpy as np
import pytest

from oracle import Oracle, critical_dt
from synth.scenarios import cube_hex_td_convective, ellipsoid_tet_td

from gpu_util import ff, max_abs

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-9, 1e-3


def _oracle_run(w):
    orc = Oracle(w.problem)
    dt = 0.5 * critical_dt(orc)
    return dt, orc.run(dt, w.n_steps)


@pytest.fixture(scope="module")
def ellipsoid_small():
    w = ellipsoid_tet_td(axes=(0.012, 0.009, 0.007))
    assert w.n_steps == 20000
    return (w,) + _oracle_run(w)


@pytest.fixture(scope="module")
def cube_small():
    w = cube_hex_td_convective(n=12)
    assert w.n_steps == 10000
    return (w,) + _oracle_run(w)


def _gpu(p, dt, n, prec, kernel, block=0, tile=0):
    f = ff()
    s = f.Solver(p, precision=prec)
    try:
        f.fedfem_set_tile(s.ctx, kernel, block, tile, 0)
        s.step(dt, n)
        assert s.sync() == n
        return s.temperature()
    finally:
        s.close()


def _check(label, w, dt, ref, configs):
    f = ff()
    for prec, tol in ((f.FP64, TOL64), (f.FP32_KAHAN, TOL32)):
        for kern, blk, B in configs(prec):
            T = _gpu(w.problem, dt, w.n_steps, prec, kern, blk, B)
            err = max_abs(T, ref)
            print(f"{label} {w.n_steps} steps prec {prec} kernel {kern}/{blk}/{B}: max|dT| = {err:.3e} "
                  f"(max T {ref.max():.2f})")
            assert err <= tol


def test_small_ellipsoid_full_2e4_steps(ellipsoid_small):
    w, dt, ref = ellipsoid_small
    f = ff()
    assert ref.max() > 45.0                      # the sources heat well above body temperature

    def configs(prec):
        out = [(f.KERNEL_PERSISTENT, 0, 0), (f.KERNEL_TILED, 0, 0), (f.KERNEL_TILED_STAGED, 0, 0)]
        out.append((f.KERNEL_TILED_REP, 0, 0))
        return out
    _check("ellipsoid 12/9/7 mm", w, dt, ref, configs)


def test_small_convective_cube_full_1e4_steps(cube_small):
    w, dt, ref = cube_small
    f = ff()
    assert ref.max() > 40.0

    def configs(prec):
        out = [(f.KERNEL_PERSISTENT, 0, 0), (f.KERNEL_TILED, 0, 0), (f.KERNEL_TILED_STAGED, 0, 0)]
        out.append((f.KERNEL_TILED_REP, 0, 0 if prec == f.FP64 else 512))
        return out
    _check("convective cube 12^3", w, dt, ref, configs)
