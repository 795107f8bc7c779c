"""Tabulated (piecewise-linear) property laws on the GPU against the FP64
oracle: every kernel, both precisions, hex and tet meshes, scenario lanes,
the critical step, the two-point table as the linear laws of Section 3.1.6,
and the argument checks of fedfem_set_material_table."""
import copy

import numpy as np
import pytest

from oracle import Oracle, critical_dt
from synth.problem import Material
from synth.scenarios import cube_hex_fp64, ellipsoid_tet_td, planning_batch

from gpu_util import ff, max_abs, run_gpu

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-9, 1e-3
# kinks at 40 and 46 degC; the heated regions cross both and, on the tet
# mesh, run past the last point (the extended end interval)
TAB = Material.tabulated((30.0, 40.0, 46.0, 70.0), (1060.0, 1050.0, 1030.0, 1000.0),
                         (3600.0, 3700.0, 3500.0, 3300.0), (0.50, 0.56, 0.70, 0.74))


def _problem(mesh):
    if mesh == "hex":
        p = copy.copy(cube_hex_fp64().problem)
    else:
        p = copy.copy(ellipsoid_tet_td(h=1.5e-3, axes=(0.024, 0.018, 0.014), n_steps=1200).problem)
    p.material = TAB
    p.T_lo, p.T_hi = 0.0, 200.0
    return p


@pytest.fixture(scope="module", params=["hex", "tet"])
def case(request):
    p = _problem(request.param)
    orc = Oracle(p)
    dt_cr = critical_dt(orc, p.T_lo, p.T_hi)
    dt = 0.5 * dt_cr
    n = 800
    return request.param, p, dt_cr, dt, n, orc.run(dt, n)


@pytest.mark.parametrize("prec_name", ["FP64", "FP32_KAHAN"])
def test_tabulated_laws_match_the_oracle(case, prec_name):
    mesh, p, dt_cr, dt, n, ref = case
    f = ff()
    T, info = run_gpu(p, dt, n, getattr(f, prec_name))
    assert info["dt_cr"] == pytest.approx(dt_cr, rel=1e-9)
    err = max_abs(T, ref)
    print(f"table {mesh} {p.n_nodes} nodes {prec_name}: max|dT| = {err:.3e}, T in [{ref.min():.2f}, {ref.max():.2f}]")
    assert ref.max() > 46.0                        # both kinks crossed
    assert err <= (TOL64 if prec_name == "FP64" else TOL32)


def test_every_kernel_gives_the_same_field(case):
    mesh, p, _, dt, _, _ = case
    f = ff()
    T0, _ = run_gpu(p, dt, 200, f.FP32_KAHAN, kernel=f.KERNEL_PERSISTENT)
    for kern in (f.KERNEL_TWO_PHASE, f.KERNEL_TILED, f.KERNEL_TILED_STAGED):
        T, _ = run_gpu(p, dt, 200, f.FP32_KAHAN, kernel=kern)
        assert np.array_equal(T, T0), (mesh, kern)


@pytest.mark.parametrize("prec_name", ["FP64", "FP32_KAHAN"])
def test_two_point_table_is_bit_identical_to_the_linear_laws(prec_name):
    """Section 3.1.6's laws given as a two-point table run the table kernels;
    their interval, value and slope are those of the linear laws, so the
    fields agree bit for bit."""
    f = ff()
    p = copy.copy(cube_hex_fp64().problem)
    lin = Material.from_two_points(37.0, 65.0, (1040.0, 1000.0), (3600.0, 3700.0), (0.5, 0.6))
    p.material = lin
    dt = 0.5 * critical_dt(Oracle(p))
    T_lin, i_lin = run_gpu(p, dt, 300, getattr(f, prec_name))
    p.material = Material.tabulated((37.0, 65.0), (1040.0, 1000.0), (3600.0, 3700.0), (0.5, 0.6))
    T_tab, i_tab = run_gpu(p, dt, 300, getattr(f, prec_name))
    assert i_tab["dt_cr"] == pytest.approx(i_lin["dt_cr"], rel=1e-14)
    assert np.array_equal(T_tab, T_lin)


@pytest.mark.parametrize("kernel_name", ["KERNEL_TILED", "KERNEL_TILED_STAGED"])
def test_table_with_scenario_lanes_equals_single_runs(kernel_name):
    f = ff()
    meshes = [pm.problems for pm in planning_batch(n_meshes=2, n_scenarios=4, n_range=(900, 3000), base_seed=11)]
    for scen in meshes:
        for i, q in enumerate(scen):
            q = copy.copy(q)
            q.material = TAB
            q.T_lo, q.T_hi = 0.0, 200.0
            scen[i] = q
    b = f.Batch(meshes, kernel=getattr(f, kernel_name))
    try:
        dt = 0.5 * b.dt_cr
        f.fedfem_step(b.ctx, dt, 150)
        assert f.fedfem_sync(b.ctx) == 150
        for g, scen in enumerate(meshes):
            for s_i in (0, 3):
                s = f.Solver(scen[s_i], precision=f.FP32_KAHAN, kernel=f.KERNEL_PERSISTENT)
                try:
                    s.step(dt, 150)
                    s.sync()
                    assert np.array_equal(b.temperature(g, s_i), s.temperature()), (g, s_i)
                finally:
                    s.close()
        ref = Oracle(meshes[0][1]).run(dt, 150)
        assert max_abs(b.temperature(0, 1), ref) <= TOL32
    finally:
        b.close()


def test_table_arguments_are_checked():
    f = ff()
    p = _problem("hex")
    s = f.Solver(p, precision=f.FP32_KAHAN)
    try:
        for args in [((37.0,), (1.0,), (1.0,), (1.0,)),                      # one point
                     (tuple(range(9)), (1.0,) * 9, (1.0,) * 9, (1.0,) * 9),   # nine points
                     ((37.0, 37.0), (1.0, 1.0), (1.0, 1.0), (1.0, 1.0)),    # not increasing
                     ((37.0, 65.0), (0.0, 1.0), (1.0, 1.0), (1.0, 1.0)),    # rho at the first point
                     ((37.0, np.nan), (1.0, 1.0), (1.0, 1.0), (1.0, 1.0))]:
            with pytest.raises(f.FedfemError) as e:
                f.fedfem_set_material_table(s.ctx, *args)
            assert e.value.code == f.E_ARG, args
        # c falls to zero near 66 degC: positive at both points, not on [0, 100]
        f.fedfem_set_material_table(s.ctx, (37.0, 50.0), (1000.0, 1000.0), (3600.0, 2000.0), (0.5, 0.5))
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_precompute(s.ctx, 0.0, 100.0)
        assert e.value.code == f.E_RANGE
        assert f.fedfem_precompute(s.ctx, 0.0, 60.0) > 0.0
    finally:
        s.close()


# eight points (the most a table takes): six kinks between 38 and 48 degC,
# slopes changing sign, all inside the range the heated cube crosses
TAB8 = Material.tabulated((30.0, 38.0, 40.0, 42.0, 44.0, 46.0, 48.0, 70.0),
                          (1060.0, 1058.0, 1050.0, 1052.0, 1040.0, 1035.0, 1030.0, 1000.0),
                          (3600.0, 3650.0, 3700.0, 3640.0, 3560.0, 3500.0, 3480.0, 3300.0),
                          (0.50, 0.52, 0.56, 0.55, 0.62, 0.70, 0.69, 0.74))


def test_eight_point_table_every_kink_every_kernel():
    """Every interior point of the largest table is a kink the field crosses:
    FP64 within 1e-9 and FP32+Kahan within 1e-3 of the oracle, all kernels
    the same bits."""
    f = ff()
    p = copy.copy(cube_hex_fp64().problem)
    p.material = TAB8
    p.T_lo, p.T_hi = 0.0, 200.0
    orc = Oracle(p)
    dt = 0.5 * critical_dt(orc, p.T_lo, p.T_hi)
    n = 800
    ref = orc.run(dt, n)
    assert ref.max() > 48.0                         # the last interior kink is crossed
    for prec, tol in ((f.FP64, TOL64), (f.FP32_KAHAN, TOL32)):
        base = None
        for kern in (f.KERNEL_PERSISTENT, f.KERNEL_TWO_PHASE, f.KERNEL_TILED, f.KERNEL_TILED_STAGED,
                     f.KERNEL_TILED_REP):
            T, _ = run_gpu(p, dt, n, prec, kernel=kern)
            err = max_abs(T, ref)
            print(f"eight-point table prec {prec} kernel {kern}: max|dT| = {err:.3e}")
            assert err <= tol
            if base is None:
                base = T
            assert np.array_equal(T, base), kern


def test_field_below_the_first_table_point_extrapolates_the_first_interval():
    """A table that starts above the initial 37 degC (points at 40, 45 and 60
    degC): most of the cube stays below its first point for the whole run,
    where every property follows the first interval's line, and the heated
    centre crosses into and past the table; FP64 and FP32+Kahan against the
    oracle, every kernel the same bits."""
    f = ff()
    p = copy.copy(cube_hex_fp64().problem)
    p.material = Material.tabulated((40.0, 45.0, 60.0), (1050.0, 1040.0, 1020.0), (3700.0, 3650.0, 3500.0),
                                    (0.55, 0.60, 0.66))
    p.T_lo, p.T_hi = 0.0, 200.0
    orc = Oracle(p)
    dt = 0.5 * critical_dt(orc, p.T_lo, p.T_hi)
    n = 800
    ref = orc.run(dt, n)
    assert ref.min() < 40.0 < 45.0 < ref.max()      # below the table and past its interior point
    for prec, tol in ((f.FP64, TOL64), (f.FP32_KAHAN, TOL32)):
        base = None
        for kern in (f.KERNEL_PERSISTENT, f.KERNEL_TILED_STAGED, f.KERNEL_TILED_REP):
            T, _ = run_gpu(p, dt, n, prec, kernel=kern)
            err = max_abs(T, ref)
            print(f"table above T0, prec {prec} kernel {kern}: max|dT| = {err:.3e}")
            assert err <= tol
            if base is None:
                base = T
            assert np.array_equal(T, base), kern
