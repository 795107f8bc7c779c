"""Pins of the oracle's heterogeneous tissue: elements in regions with their
own laws, perfusion and metabolic heat (the element-wise properties that the
finite element form allows).

The pins: one material in every region is the homogeneous problem; the
region weights partition the lumped volume; a two-material Dirichlet bar has
the series-resistance steady state; a uniform block whose regions share the
ratios beta/C and Q/C stays uniform and relaxes geometrically; the
critical-step scale against brute force, and stability at 0.9 of it."""
import copy

import numpy as np
import pytest

from oracle import Oracle, critical_dt
from oracle.critical_dt import region_scale
from synth.meshes import box_face_nodes, hex_box, kuhn_tet_box
from synth.problem import Material, Perfusion, Problem
from synth.scenarios import cube_hex_fp64

H = 1e-3
LIVER = Material(T_ref=37.0, rho0=1060.0, drho=-0.5, c0=3600.0, dc=4.0, k0=0.52, dk=0.0015)
TUMOUR = Material(T_ref=37.0, rho0=1045.0, drho=-0.8, c0=3750.0, dc=6.0, k0=0.60, dk=0.0030)


def _centroids(p):
    return p.xyz[np.asarray(p.conn)].mean(axis=1)


def test_one_material_in_every_region_is_the_homogeneous_problem():
    w = cube_hex_fp64()
    p = copy.copy(w.problem)
    base = Oracle(p).run(0.5 * critical_dt(Oracle(p)), 200)
    q = copy.copy(p)
    q.regions = (np.arange(len(p.conn)) % 3).astype(np.int32)
    q.region_materials = (p.material,) * 3
    q.region_perfusion = (p.perfusion,) * 3
    orc = Oracle(q)
    assert critical_dt(orc) == pytest.approx(critical_dt(Oracle(p)), rel=1e-12)
    np.testing.assert_allclose(orc.run(0.5 * critical_dt(Oracle(p)), 200), base, rtol=0, atol=1e-11)


def test_region_weights_partition_the_lumped_volume():
    m = kuhn_tet_box(5, 4, 3, H)
    p = Problem(m.elem_type, m.xyz, m.conn, LIVER)
    p.regions = (_centroids(p)[:, 0] > 2.2 * H).astype(np.int32)
    p.region_materials = (LIVER, TUMOUR)
    p.region_perfusion = (Perfusion(), Perfusion())
    orc = Oracle(p)
    np.testing.assert_allclose(orc.W[0] + orc.W[1], orc.V, rtol=1e-14)
    assert np.sum(orc.W[1]) == pytest.approx(np.sum(orc.V_e[p.regions == 1]), rel=1e-13)
    assert np.count_nonzero((orc.W[0] > 0) & (orc.W[1] > 0)) > 0          # interface nodes share


def test_two_material_bar_has_the_series_resistance_steady_state():
    """Constant k1 on the left half, k2 on the right, Dirichlet ends: the
    heat flow is the same through every element, so the nodal temperatures are
    linear in x on each half with slopes in the ratio k2 : k1."""
    n = 8
    m = hex_box(n, 1, 1, H)
    k1, k2 = 0.4, 1.2
    mats = (Material.constant(1060.0, 3600.0, k1), Material.constant(1000.0, 3000.0, k2))
    left, right = box_face_nodes(m, ("x0",)), box_face_nodes(m, ("x1",))
    T1, T2 = 37.0, 65.0
    p = Problem(m.elem_type, m.xyz, m.conn, mats[0], dirichlet_nodes=np.concatenate([left, right]),
                dirichlet_T=np.concatenate([np.full(4, T1), np.full(4, T2)]), T0=40.0)
    p.regions = (_centroids(p)[:, 0] > n * H / 2).astype(np.int32)
    p.region_materials = mats
    p.region_perfusion = (Perfusion(), Perfusion())
    orc = Oracle(p)
    T = orc.run(0.9 * critical_dt(orc), 8000)
    x = m.grid_index[:, 0] * H
    L = n * H
    q = (T2 - T1) / (0.5 * L / k1 + 0.5 * L / k2)          # heat flow per unit area
    expect = np.where(x <= L / 2, T1 + q * x / k1, T1 + q * (L / 2) / k1 + q * (x - L / 2) / k2)
    np.testing.assert_allclose(T, expect, rtol=0, atol=1e-10)


def test_uniform_block_with_matched_regions_relaxes_geometrically():
    """Region 2 has twice region 1's rho c, w_b c_b and Q_m, so every node has
    the same beta_i / C_i and Q_i / C_i: an insulated block at a uniform
    temperature stays uniform (no conduction) and follows
    T^n = T_inf + (T0 - T_inf)(1 - dt beta/C)^n, T_inf = T_a + Q_m / (w_b c_b)."""
    m = kuhn_tet_box(4, 4, 4, H)
    m1 = Material.constant(1000.0, 3000.0, 0.5)
    m2 = Material.constant(1200.0, 5000.0, 0.9)            # rho c = 2 x 3.0e6
    pf1 = Perfusion(w_b=10.0, c_b=3600.0, T_a=37.0, Q_m=2.0e4)
    pf2 = Perfusion(w_b=20.0, c_b=3600.0, T_a=37.0, Q_m=4.0e4)
    p = Problem(m.elem_type, m.xyz, m.conn, m1, perfusion=pf1, T0=30.0)
    c = _centroids(p)
    p.regions = (np.linalg.norm(c - 2 * H, axis=1) < 1.3 * H).astype(np.int32)
    assert 0 < p.regions.sum() < len(p.regions)
    p.region_materials = (m1, m2)
    p.region_perfusion = (pf1, pf2)
    orc = Oracle(p)
    dt, n = 0.5 * critical_dt(orc), 400
    T = orc.run(dt, n)
    rate = pf1.w_b * pf1.c_b / (m1.rho0 * m1.c0)
    T_inf = pf1.T_a + pf1.Q_m / (pf1.w_b * pf1.c_b)
    expect = T_inf + (30.0 - T_inf) * (1 - dt * rate) ** n
    np.testing.assert_allclose(T, expect, rtol=0, atol=1e-11)


@pytest.mark.parametrize("lo,hi", [(0.0, 100.0), (30.0, 60.0)])
def test_region_scale_against_brute_force(lo, hi):
    T = np.linspace(lo, hi, 200001)
    k = np.maximum(LIVER.k0 + LIVER.dk * (T - 37.0), TUMOUR.k0 + TUMOUR.dk * (T - 37.0))
    rc = np.minimum((LIVER.rho0 + LIVER.drho * (T - 37.0)) * (LIVER.c0 + LIVER.dc * (T - 37.0)),
                    (TUMOUR.rho0 + TUMOUR.drho * (T - 37.0)) * (TUMOUR.c0 + TUMOUR.dc * (T - 37.0)))
    brute = max(1.0, k.max() / LIVER.k0) * max(1.0, LIVER.rho0 * LIVER.c0 / rc.min())
    assert region_scale((LIVER, TUMOUR), lo, hi) == pytest.approx(brute, rel=1e-8)


def test_tumour_in_liver_is_stable_at_the_bounded_step():
    """Runs at 0.9 of the bounded critical step stay bounded, hottest at the
    source; at three times that step they blow up, so the bound is not
    vacuous."""
    w = cube_hex_fp64()
    p = copy.copy(w.problem)
    c = _centroids(p)
    p.regions = (np.linalg.norm(c - 5e-3, axis=1) < 2.5e-3).astype(np.int32)
    p.region_materials = (LIVER, TUMOUR)
    p.region_perfusion = (Perfusion(w_b=0.5, c_b=3617.0, T_a=37.0, Q_m=400.0),
                          Perfusion(w_b=0.2, c_b=3617.0, T_a=37.0, Q_m=800.0))
    orc = Oracle(p)
    dt = critical_dt(orc)
    T = orc.run(0.9 * dt, 600)
    assert np.all(np.isfinite(T)) and 37.0 <= T.min() and T.max() < 80.0
    assert T[np.argmin(np.sum((p.xyz - 5e-3) ** 2, axis=1))] == pytest.approx(T.max())
    with np.errstate(over="ignore", invalid="ignore"):
        Tb = orc.run(3.0 * dt, 600)
    assert not np.all(np.abs(Tb) < 1e3)
