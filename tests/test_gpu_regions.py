"""Heterogeneous tissue (element regions with their own laws, perfusion and
metabolic heat) on the GPU against the FP64 oracle: hex and tet meshes, both
precisions, every kernel, scenario lanes, and the argument checks of
fedfem_set_regions."""
import copy

import numpy as np
import pytest

from oracle import Oracle, critical_dt
from synth.problem import Material, Perfusion
from synth.scenarios import cube_hex_fp64, ellipsoid_tet_td, planning_batch

from gpu_util import ff, max_abs, run_gpu

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-9, 1e-3
LIVER = Material(T_ref=37.0, rho0=1060.0, drho=-0.5, c0=3600.0, dc=4.0, k0=0.52, dk=0.0015)
TUMOUR = Material(T_ref=35.0, rho0=1045.0, drho=-0.8, c0=3750.0, dc=6.0, k0=0.60, dk=0.0030)
VESSEL = Material.constant(1050.0, 3617.0, 0.50)
PERF = (Perfusion(w_b=0.5, c_b=3617.0, T_a=37.0, Q_m=400.0),
        Perfusion(w_b=0.2, c_b=3617.0, T_a=37.0, Q_m=800.0),
        Perfusion(w_b=8.0, c_b=3617.0, T_a=37.0, Q_m=0.0))


def _with_regions(p, centre, radius):
    """A tumour ball (region 1) with a perfused shell (region 2) in liver (region 0)."""
    p = copy.copy(p)
    c = p.xyz[np.asarray(p.conn)].mean(axis=1)
    d = np.linalg.norm(c - np.asarray(centre), axis=1)
    p.regions = np.where(d < radius, 1, np.where(d < 1.6 * radius, 2, 0)).astype(np.int32)
    p.region_materials = (LIVER, TUMOUR, VESSEL)
    p.region_perfusion = PERF
    return p


def _problem(mesh):
    if mesh == "hex":
        return _with_regions(cube_hex_fp64().problem, (5e-3, 5e-3, 5e-3), 2.0e-3)
    p = ellipsoid_tet_td(h=1.5e-3, axes=(0.024, 0.018, 0.014), n_steps=1200).problem
    return _with_regions(p, p.sources[0].x0, 4e-3)


@pytest.fixture(scope="module", params=["hex", "tet"])
def case(request):
    p = _problem(request.param)
    assert {0, 1, 2} <= set(np.unique(p.regions))
    orc = Oracle(p)
    dt_cr = critical_dt(orc)
    dt = 0.5 * dt_cr
    n = 600
    return request.param, p, dt_cr, dt, n, orc.run(dt, n)


@pytest.mark.parametrize("prec_name", ["FP64", "FP32_KAHAN"])
def test_regions_match_the_oracle(case, prec_name):
    mesh, p, dt_cr, dt, n, ref = case
    f = ff()
    T, info = run_gpu(p, dt, n, getattr(f, prec_name))
    assert info["dt_cr"] == pytest.approx(dt_cr, rel=1e-9)
    err = max_abs(T, ref)
    print(f"regions {mesh} {p.n_nodes} nodes {prec_name}: max|dT| = {err:.3e}, max T {ref.max():.2f}")
    assert ref.max() > 40.0
    assert err <= (TOL64 if prec_name == "FP64" else TOL32)


def test_every_kernel_gives_the_same_field(case):
    mesh, p, _, dt, _, _ = case
    f = ff()
    T0, _ = run_gpu(p, dt, 200, f.FP32_KAHAN, kernel=f.KERNEL_PERSISTENT)
    for kern in (f.KERNEL_TWO_PHASE, f.KERNEL_TILED, f.KERNEL_TILED_STAGED):
        T, _ = run_gpu(p, dt, 200, f.FP32_KAHAN, kernel=kern)
        assert np.array_equal(T, T0), (mesh, kern)


def test_one_material_in_every_region_is_the_homogeneous_problem():
    f = ff()
    p = copy.copy(cube_hex_fp64().problem)
    dt = 0.5 * critical_dt(Oracle(p))
    T_plain, i_plain = run_gpu(p, dt, 300, f.FP64)
    q = copy.copy(p)
    q.regions = (np.arange(len(p.conn)) % 3).astype(np.int32)
    q.region_materials = (p.material,) * 3
    q.region_perfusion = (p.perfusion,) * 3
    T_reg, i_reg = run_gpu(q, dt, 300, f.FP64)
    assert i_reg["dt_cr"] == pytest.approx(i_plain["dt_cr"], rel=1e-12)
    assert max_abs(T_reg, T_plain) <= 1e-11


@pytest.mark.parametrize("kernel_name", ["KERNEL_TILED", "KERNEL_TILED_STAGED"])
def test_regions_with_scenario_lanes_equal_single_runs(kernel_name):
    f = ff()
    meshes = [pm.problems for pm in planning_batch(n_meshes=2, n_scenarios=4, n_range=(900, 3000), base_seed=5)]
    for scen in meshes:
        centre = scen[0].xyz.mean(axis=0)
        for i, q in enumerate(scen):
            scen[i] = _with_regions(q, centre, 3e-3)
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
        ref = Oracle(meshes[1][2]).run(dt, 150)
        assert max_abs(b.temperature(1, 2), ref) <= TOL32
    finally:
        b.close()


def test_region_arguments_are_checked():
    f = ff()
    p = _problem("hex")
    s = f.Solver(p, precision=f.FP32_KAHAN)
    try:
        E = len(p.conn)
        bad = [((), (), np.zeros(E)),                                        # no region
               ((LIVER,) * 17, PERF[:1] * 17, np.zeros(E)),                   # 17 regions
               ((LIVER, TUMOUR), PERF[:2], np.full(E, 2)),                    # id out of range
               ((LIVER, TUMOUR), PERF[:2], np.full(E, -1)),
               ((Material.constant(0.0, 3600.0, 0.5),), PERF[:1], np.zeros(E)),
               ((LIVER,), (Perfusion(w_b=-1.0, c_b=3617.0, T_a=37.0),), np.zeros(E))]
        for mats, perf, reg in bad:
            with pytest.raises(f.FedfemError) as e:
                f.fedfem_set_regions(s.ctx, mats, perf, reg)
            assert e.value.code == f.E_ARG, (len(mats), reg[:1])
        # rho c of region 1 reaches zero inside [0, 100]
        hot = Material(T_ref=37.0, rho0=1000.0, drho=0.0, c0=3600.0, dc=-60.0, k0=0.5, dk=0.0)
        f.fedfem_set_regions(s.ctx, (LIVER, hot), PERF[:2], (np.arange(E) % 2).astype(np.int32))
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_precompute(s.ctx, 0.0, 100.0)
        assert e.value.code == f.E_RANGE
        assert f.fedfem_precompute(s.ctx, 0.0, 80.0) > 0.0
    finally:
        s.close()
