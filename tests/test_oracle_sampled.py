"""The sampled-node oracle (used for parity at sizes too large to step whole)
must agree with the whole-mesh oracle at the samples."""
import numpy as np

from oracle import Oracle, critical_dt, sampled_run
from synth.scenarios import cube_hex_td_convective, ellipsoid_tet_td


def test_sampled_run_equals_full_run_hex():
    w = cube_hex_td_convective(n=14)
    p = w.problem
    dt = 0.5 * critical_dt(p)
    full = Oracle(p).run(dt, 6)
    rng = np.random.default_rng(1)
    samples = rng.choice(p.n_nodes, 40, replace=False)
    samples = np.concatenate([samples, [p.n_nodes - 1, np.argmax(p.xyz[:, 2])]])
    np.testing.assert_allclose(sampled_run(p, dt, 6, samples), full[samples], rtol=0, atol=1e-12)


def test_sampled_run_equals_full_run_tet():
    w = ellipsoid_tet_td(h=2.5e-3, axes=(0.02, 0.015, 0.012))
    p = w.problem
    dt = 0.5 * critical_dt(p)
    full = Oracle(p).run(dt, 4)
    rng = np.random.default_rng(2)
    samples = rng.choice(p.n_nodes, 30, replace=False)
    np.testing.assert_allclose(sampled_run(p, dt, 4, samples), full[samples], rtol=0, atol=1e-12)


def test_sampled_run_equals_full_run_for_the_variants():
    """Regions (cut with the sub-mesh), tabulated laws, the full hex rule and
    uniform lumping (whose V / N stays that of the whole mesh)."""
    import copy
    from synth.problem import Material, Perfusion
    w = cube_hex_td_convective(n=20)
    base = w.problem
    rng = np.random.default_rng(3)
    samples = rng.choice(base.n_nodes, 4, replace=False)
    tab = copy.copy(base)
    tab.material = Material.tabulated((30.0, 40.0, 46.0, 70.0), (1060.0, 1050.0, 1030.0, 1000.0),
                                      (3600.0, 3700.0, 3500.0, 3300.0), (0.50, 0.56, 0.70, 0.74))
    reg = copy.copy(base)
    cen = base.xyz[np.asarray(base.conn)].mean(axis=1)
    reg.regions = (np.linalg.norm(cen - cen.mean(axis=0), axis=1) < 6e-3).astype(np.int32)
    reg.region_materials = (base.material, Material.constant(1045.0, 3750.0, 0.6))
    reg.region_perfusion = (base.perfusion, Perfusion(w_b=1.0, c_b=3617.0, T_a=37.0, Q_m=500.0))
    full = copy.copy(base)
    full.hex_rule = "full"
    uni = copy.copy(base)
    uni.lumping = "uniform"
    uni.perfusion = Perfusion(w_b=26.6, c_b=3617.0, T_a=39.0, Q_m=33800.0)   # away from T0, so beta matters
    for p in (tab, reg, full, uni):
        dt = 0.5 * critical_dt(p)
        ref = Oracle(p).run(dt, 4)
        np.testing.assert_allclose(sampled_run(p, dt, 4, samples), ref[samples], rtol=0, atol=1e-12)
