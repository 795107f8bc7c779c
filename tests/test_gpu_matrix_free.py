"""Matrix-free tet4 geometry (fedfem_set_matrix_free): the tiled kernels
recompute each element's matrix from its nodes' coordinates every step
instead of reading the pre-computed one (Eq. 15-16).

* Against the FP64 oracle on the reduced tet ellipsoid recipe for the full
  2e4 steps (FP32 + Kahan, 1e-3 degC), and on the 1 mm ellipsoid at sampled
  nodes (the oracle's dependency cones);
* the two kernels that take it, at any tile size, agree bit for bit, and
  differ from the stored-matrix path only by the FP32 rounding of the
  recomputed matrices;
* the refusals (FP64 state, hex8, kernels without it)."""
import copy

import numpy as np
import pytest

from oracle import Oracle, critical_dt, sampled_run
from synth.scenarios import cube_hex_fp64, ellipsoid_tet_td

from gpu_util import ff, max_abs

pytestmark = pytest.mark.gpu

TOL32 = 1e-3


def _run(p, dt, n, kernel, mf=True, tile=0, T0=None, prec=None):
    f = ff()
    s = f.Solver(p, precision=f.FP32_KAHAN if prec is None else prec, matrix_free=mf)
    try:
        f.fedfem_set_tile(s.ctx, kernel, 0, tile, 0)
        if T0 is not None:
            s.init(T0)
        s.step(dt, n)
        assert s.sync() == n
        return s.temperature(), s.info()
    finally:
        s.close()


@pytest.fixture(scope="module")
def small():
    w = ellipsoid_tet_td(axes=(0.012, 0.009, 0.007))
    orc = Oracle(w.problem)
    dt = 0.5 * critical_dt(orc)
    return w, dt, orc.run(dt, w.n_steps)


def test_matrix_free_full_2e4_steps_against_the_oracle(small):
    w, dt, ref = small
    f = ff()
    out = {}
    for kern in (f.KERNEL_TILED, f.KERNEL_TILED_STAGED):
        T, info = _run(w.problem, dt, w.n_steps, kern)
        err = max_abs(T, ref)
        print(f"matrix-free kernel {kern}: max|dT| vs oracle after {w.n_steps} steps = {err:.3e} "
              f"(max T {ref.max():.2f})")
        assert err <= TOL32
        out[kern] = T
    assert np.array_equal(out[f.KERNEL_TILED], out[f.KERNEL_TILED_STAGED])
    for kern, B in ((f.KERNEL_TILED, 64), (f.KERNEL_TILED_STAGED, 96)):   # other tilings: the same bits
        T, _ = _run(w.problem, dt, 500, kern, tile=B)
        T0, _ = _run(w.problem, dt, 500, f.KERNEL_TILED_STAGED)
        assert np.array_equal(T, T0), (kern, B)


def test_matrix_free_differs_from_stored_matrices_by_rounding_only(small):
    w, dt, _ = small
    f = ff()
    a, ia = _run(w.problem, dt, 1000, f.KERNEL_TILED_STAGED, mf=True)
    b, ib = _run(w.problem, dt, 1000, f.KERNEL_TILED_STAGED, mf=False)
    d = max_abs(a, b)
    print(f"matrix-free vs stored matrices after 1000 steps: {d:.3e}; algorithmic bytes "
          f"{ia['algorithmic_bytes_per_step']} vs {ib['algorithmic_bytes_per_step']}")
    assert 0.0 < d < 1e-4
    assert ia["algorithmic_bytes_per_step"] < ib["algorithmic_bytes_per_step"]


def test_matrix_free_full_size_ellipsoid_sampled_oracle():
    w = ellipsoid_tet_td()
    p = copy.copy(w.problem)
    rng = np.random.default_rng(31)
    T0 = 37.0 + 8.0 * rng.random(p.n_nodes)
    T0[p.dirichlet_nodes] = 37.0
    p.T0 = T0
    dt = 0.5 * critical_dt(w.problem)
    samples = rng.choice(p.n_nodes, 150, replace=False)
    ref = sampled_run(p, dt, 3, samples)
    f = ff()
    for kern in (f.KERNEL_TILED, f.KERNEL_TILED_STAGED):
        T, _ = _run(p, dt, 3, kern, T0=T0)
        err = max_abs(T[samples], ref)
        print(f"1 mm ellipsoid, matrix-free kernel {kern}: sampled max|dT| = {err:.3e}")
        assert err <= TOL32


def test_matrix_free_refusals():
    f = ff()
    w = ellipsoid_tet_td(axes=(0.006, 0.005, 0.004))
    p = w.problem
    for kern in (f.KERNEL_PERSISTENT, f.KERNEL_TWO_PHASE, f.KERNEL_TILED_REP):
        s = f.Solver(p, precision=f.FP32_KAHAN, matrix_free=True)
        try:
            f.fedfem_set_tile(s.ctx, kern, 0, 0, 0)
            with pytest.raises(f.FedfemError) as ei:
                s.step(0.01, 1)
            assert ei.value.code == f.E_UNSUPPORTED, kern
        finally:
            s.close()
    s = f.Solver(p, precision=f.FP64, matrix_free=True)
    try:
        with pytest.raises(f.FedfemError) as ei:
            s.step(0.01, 1)
        assert ei.value.code == f.E_UNSUPPORTED
    finally:
        s.close()
    ctx = f.fedfem_create(0, f.FP32_KAHAN, None)
    try:
        h = cube_hex_fp64().problem
        f.fedfem_set_mesh(ctx, 8, h.xyz, h.conn)
        with pytest.raises(f.FedfemError) as ei:
            f.fedfem_set_matrix_free(ctx, True)
        assert ei.value.code == f.E_UNSUPPORTED
    finally:
        f.fedfem_destroy(ctx)
