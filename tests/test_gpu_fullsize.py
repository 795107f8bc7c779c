"""Parity at the workloads' full sizes, in the launch configurations the bench
uses.  The oracle cannot step 2 million nodes, so it computes a few steps at
sampled nodes (oracle/sampled.py: the exact dependency cone of each sample);
the full step counts are compared against the FP64 GPU path, which the
smaller tests pin to the oracle at 1e-9 degC.  Inputs and dt always come from
the seeded generators and the oracle, never from the GPU path."""
import copy

import numpy as np
import pytest

from oracle import Oracle, critical_dt, sampled_run
from synth.scenarios import cube_hex_td_convective, ellipsoid_tet_td

from gpu_util import ff, max_abs

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-9, 1e-3


def _random_T0(p, seed, lo=37.0, hi=45.0):
    rng = np.random.default_rng(seed)
    return lo + (hi - lo) * rng.random(p.n_nodes)


def _run(p, dt, n, prec, kernel, T0=None, tile_nodes=0):
    f = ff()
    s = f.Solver(p, precision=prec)
    try:
        f.fedfem_set_tile(s.ctx, kernel, 0, tile_nodes, 0)
        if T0 is not None:
            s.init(T0)
        s.step(dt, n)
        assert s.sync() == n
        return s.temperature(), s.info()
    finally:
        s.close()


@pytest.fixture(scope="module")
def cube128():
    from oracle.box_spectrum import critical_dt_hex_box
    w = cube_hex_td_convective(n=128)
    # the cube's own critical step, by separation of variables (equal to the dense
    # solver's on small boxes, tests/test_oracle_dtcr.py)
    dt = 0.5 * critical_dt_hex_box(w.problem, 128, 1e-3)
    return w, dt


def test_cube128_dt_cr_matches_oracle(cube128):
    w, dt = cube128
    f = ff()
    s = f.Solver(w.problem, precision=f.FP32_KAHAN)
    try:
        print(f"cube128 dt_cr GPU {s.dt_cr:.12g} oracle {2 * dt:.12g}")
        assert s.dt_cr == pytest.approx(2 * dt, rel=1e-8)
    finally:
        s.close()


@pytest.fixture(scope="module")
def ellipsoid():
    w = ellipsoid_tet_td()
    dt = 0.5 * critical_dt(w.problem)
    return w, dt


def _kernels(prec=None):
    """Kernel and tile size pairs; the replicated-row kernel with the bench's
    512-node tiles in FP32 (its FP64 build has 256-thread rows: default tiles)."""
    f = ff()
    rep_B = 0 if prec == f.FP64 else 512
    return [(f.KERNEL_PERSISTENT, 0), (f.KERNEL_TILED, 0), (f.KERNEL_TILED_STAGED, 384), (f.KERNEL_TILED_REP, rep_B)]


def test_cube128_sampled_oracle_parity(cube128):
    w, dt = cube128
    p = copy.copy(w.problem)
    p.T0 = _random_T0(p, 11)
    rng = np.random.default_rng(12)
    N = p.n_nodes
    top = np.nonzero(np.isclose(p.xyz[:, 2], p.xyz[:, 2].max()))[0]
    centre = np.argsort(np.sum((p.xyz - 0.064) ** 2, axis=1))[:40]
    samples = np.unique(np.concatenate([rng.choice(N, 200, replace=False), rng.choice(top, 40), centre]))
    n = 5
    ref = sampled_run(p, dt, n, samples)
    f = ff()
    for prec, tol in ((f.FP64, TOL64), (f.FP32_KAHAN, TOL32)):
        for kern, B in _kernels(prec):
            T, info = _run(p, dt, n, prec, kern, T0=p.T0, tile_nodes=B)
            err = max_abs(T[samples], ref)
            print(f"cube128 prec {prec} kernel {kern}: sampled max|dT| = {err:.3e}")
            assert err <= tol


def test_cube128_fp32_kahan_vs_fp64_after_1e4_steps(cube128):
    w, dt = cube128
    f = ff()
    T64, _ = _run(w.problem, dt, w.n_steps, f.FP64, f.KERNEL_PERSISTENT)
    T32, _ = _run(w.problem, dt, w.n_steps, f.FP32_KAHAN, f.KERNEL_TILED_STAGED, tile_nodes=384)
    Tp, _ = _run(w.problem, dt, w.n_steps, f.FP32_PLAIN, f.KERNEL_TILED)
    e32, ep = max_abs(T32, T64), max_abs(Tp, T64)
    print(f"cube128 1e4 steps: FP32+Kahan vs FP64 {e32:.3e}, plain FP32 {ep:.3e}, max T {T64.max():.2f}")
    assert e32 <= TOL32
    assert T64.max() > 45.0


def test_cube128_uniform_field_bit_unchanged(cube128):
    w, dt = cube128
    p = copy.copy(w.problem)
    p.sources = []
    p.conv_T_inf = 37.0
    f = ff()
    for kern, B in _kernels(f.FP32_KAHAN):
        T, _ = _run(p, dt, 50, f.FP32_KAHAN, kern, tile_nodes=B)
        assert np.all(T == 37.0), kern


def test_ellipsoid_sampled_oracle_parity(ellipsoid):
    w, dt = ellipsoid
    p = copy.copy(w.problem)
    p.T0 = _random_T0(p, 21)
    p.T0[p.dirichlet_nodes] = 37.0
    rng = np.random.default_rng(22)
    samples = rng.choice(p.n_nodes, 150, replace=False)
    n = 3
    ref = sampled_run(p, dt, n, samples)
    f = ff()
    for prec, tol in ((f.FP64, TOL64), (f.FP32_KAHAN, TOL32)):
        for kern, B in ((f.KERNEL_PERSISTENT, 0), (f.KERNEL_TILED, 0), (f.KERNEL_TILED_REP, 0)):
            T, _ = _run(p, dt, n, prec, kern, T0=p.T0, tile_nodes=B)
            err = max_abs(T[samples], ref)
            print(f"ellipsoid prec {prec} kernel {kern}: sampled max|dT| = {err:.3e}")
            assert err <= tol


def test_ellipsoid_dt_cr_matches_oracle(ellipsoid):
    w, dt = ellipsoid
    f = ff()
    s = f.Solver(w.problem, precision=f.FP32_KAHAN)
    try:
        assert s.dt_cr == pytest.approx(2 * dt, rel=1e-8)
        print(f"ellipsoid dt_cr GPU {s.dt_cr:.12g} oracle {2 * dt:.12g}, Lanczos {s.info()['lanczos_iterations']}")
    finally:
        s.close()


def test_ellipsoid_fp32_kahan_vs_fp64_after_2e4_steps(ellipsoid):
    w, dt = ellipsoid
    f = ff()
    T64, _ = _run(w.problem, dt, w.n_steps, f.FP64, f.KERNEL_PERSISTENT)
    T32, _ = _run(w.problem, dt, w.n_steps, f.FP32_KAHAN, f.KERNEL_TILED)
    Tp, _ = _run(w.problem, dt, w.n_steps, f.FP32_PLAIN, f.KERNEL_TILED)
    e32, ep = max_abs(T32, T64), max_abs(Tp, T64)
    print(f"ellipsoid 2e4 steps: FP32+Kahan vs FP64 {e32:.3e}, plain FP32 {ep:.3e}, max T {T64.max():.2f}")
    assert e32 <= TOL32
    assert e32 < ep
