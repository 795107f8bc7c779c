"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (max |dT| over all nodes): FP64 1e-9 degC, FP32 + Kahan 1e-3 degC.
"""
import copy

import numpy as np
import pytest

from oracle import Oracle, critical_dt, eq20_error
from synth.scenarios import cube_hex_fp64, cube_hex_td_convective, ellipsoid_tet_td

from gpu_util import ff, max_abs, run_gpu

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-9, 1e-3


@pytest.fixture(scope="module")
def cube():
    w = cube_hex_fp64()
    orc = Oracle(w.problem)
    dt_cr = critical_dt(orc)
    dt = 0.5 * dt_cr
    return w, orc, dt_cr, dt, orc.run(dt, w.n_steps)


def test_cube_fp64_2000_steps(cube):
    w, orc, dt_cr, dt, ref = cube
    f = ff()
    T, info = run_gpu(w.problem, dt, w.n_steps, f.FP64)
    assert info["dt_cr"] == pytest.approx(dt_cr, rel=1e-9)
    err = max_abs(T, ref)
    print(f"cube FP64 2000 steps: max|dT| = {err:.3e}, Eq.20 = {eq20_error(ref, T):.3e}, "
          f"Lanczos iterations {info['lanczos_iterations']}")
    assert err <= TOL64


def test_cube_fp32_kahan_and_plain(cube):
    w, orc, dt_cr, dt, ref = cube
    f = ff()
    Tk, _ = run_gpu(w.problem, dt, w.n_steps, f.FP32_KAHAN)
    Tp, _ = run_gpu(w.problem, dt, w.n_steps, f.FP32_PLAIN)
    ek, ep = max_abs(Tk, ref), max_abs(Tp, ref)
    print(f"cube FP32+Kahan max|dT| = {ek:.3e}; FP32 plain (negative control) = {ep:.3e}")
    assert ek <= TOL32
    assert ek < ep


def test_every_kernel_and_order_is_bit_identical(cube):
    w, orc, dt_cr, dt, ref = cube
    f = ff()
    for prec in (f.FP64, f.FP32_KAHAN):
        base, _ = run_gpu(w.problem, dt, 300, prec, order=f.ORDER_MORTON, kernel=f.KERNEL_PERSISTENT)
        for order in (f.ORDER_INPUT, f.ORDER_MORTON, f.ORDER_RCM):
            for kernel in (f.KERNEL_TWO_PHASE, f.KERNEL_PERSISTENT, f.KERNEL_TILED, f.KERNEL_TILED_STAGED,
                           f.KERNEL_TILED_REP):
                T, _ = run_gpu(w.problem, dt, 300, prec, order=order, kernel=kernel)
                assert np.array_equal(T, base), (prec, order, kernel)


@pytest.mark.parametrize("n_steps", [1, 2, 7])
def test_tiled_kernel_odd_even_steps_and_tets(n_steps):
    """The tiled kernels double-buffer T; any step count must leave the same
    state as the other kernels, for hex and tet meshes, several tile sizes
    (some larger than the block, so threads own more than one node) and every
    block size the staged kernel is built for."""
    f = ff()
    for w in (cube_hex_td_convective(n=14), ellipsoid_tet_td(h=2e-3, axes=(0.024, 0.018, 0.014))):
        p = w.problem
        dt = 0.5 * critical_dt(Oracle(p))
        base, _ = run_gpu(p, dt, n_steps, f.FP32_KAHAN, kernel=f.KERNEL_PERSISTENT)
        # hex tiles larger than the block (threads own two nodes); tets (about 24
        # elements per node) with smaller tiles so that the load table fits
        big = ((f.KERNEL_TILED_STAGED, 0, 1000), (f.KERNEL_TILED_STAGED, 1024, 1280),
               (f.KERNEL_TILED_REP, 0, 512)) if p.elem_type == 8 else \
              ((f.KERNEL_TILED_STAGED, 1024, 200), (f.KERNEL_TILED_REP, 256, 128))
        # the replicated-row kernel: default tiles, tiles smaller than the block, 256 threads
        rep = ((f.KERNEL_TILED_REP, 0, 0), (f.KERNEL_TILED_REP, 0, 96), (f.KERNEL_TILED_REP, 256, 72))
        for kern, blk, B in ((f.KERNEL_TILED, 0, 0), (f.KERNEL_TILED, 0, 64), (f.KERNEL_TILED, 0, 160),
                             (f.KERNEL_TILED_STAGED, 0, 0), (f.KERNEL_TILED_STAGED, 0, 96),
                             (f.KERNEL_TILED_STAGED, 256, 72)) + rep + big:
            s = f.Solver(p, precision=f.FP32_KAHAN)
            try:
                f.fedfem_set_tile(s.ctx, kern, blk, B, 0)
                s.step(dt, n_steps)
                assert s.sync() == n_steps
                assert np.array_equal(s.temperature(), base), (p.elem_type, kern, blk, B, n_steps)
                s.step(dt, 3)        # continue after an odd/even count
                s.sync()
            finally:
                s.close()


@pytest.mark.parametrize("prec_name", ["FP64", "FP32_KAHAN"])
def test_small_tet_ellipsoid_td(prec_name):
    w = ellipsoid_tet_td(h=1.5e-3, axes=(0.024, 0.018, 0.014), n_steps=1500)
    p = w.problem
    orc = Oracle(p)
    dt = 0.5 * critical_dt(orc)
    ref = orc.run(dt, w.n_steps)
    f = ff()
    T, info = run_gpu(p, dt, w.n_steps, getattr(f, prec_name))
    assert info["dt_cr"] == pytest.approx(critical_dt(orc), rel=1e-9)
    err = max_abs(T, ref)
    print(f"tet ellipsoid {p.n_nodes} nodes {prec_name}: max|dT| = {err:.3e}, max T = {ref.max():.2f}")
    assert err <= (TOL64 if prec_name == "FP64" else TOL32)


@pytest.mark.parametrize("prec_name", ["FP64", "FP32_KAHAN"])
def test_small_convective_cube_td(prec_name):
    w = cube_hex_td_convective(n=12)
    p = w.problem
    orc = Oracle(p)
    dt = 0.5 * critical_dt(orc)
    ref = orc.run(dt, 800)
    f = ff()
    T, _ = run_gpu(p, dt, 800, getattr(f, prec_name))
    err = max_abs(T, ref)
    print(f"convective cube 12^3 {prec_name}: max|dT| = {err:.3e}")
    assert err <= (TOL64 if prec_name == "FP64" else TOL32)


def test_uniform_field_bit_unchanged_on_gpu():
    w = cube_hex_td_convective(n=20)
    p = copy.copy(w.problem)
    p.sources = []
    p.conv_T_inf = 37.0
    f = ff()
    for prec in (f.FP64, f.FP32_KAHAN, f.FP32_PLAIN):
        for kernel in (f.KERNEL_TWO_PHASE, f.KERNEL_PERSISTENT, f.KERNEL_TILED, f.KERNEL_TILED_STAGED,
                       f.KERNEL_TILED_REP):
            T, _ = run_gpu(p, 1.0, 200, prec, kernel=kernel)
            assert np.all(T == 37.0), (prec, kernel)


@pytest.mark.parametrize("prec_name", ["FP64", "FP32_KAHAN"])
@pytest.mark.parametrize("mesh", ["tet", "hex"])
def test_section_3_1_6_laws_with_density_varying(prec_name, mesh):
    """The temperature-dependent variant the paper verifies (Section 3.1.6,
    Table 5): rho, c and k all linear in T through their 37 and 65 degC values
    (rho falls from 1040 to 1000 kg/m^3), on a tet and a hex mesh."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    g = g["td_properties_sec_3_1_6"]
    from synth.problem import Material
    mat = Material.from_two_points(g["T1"], g["T2"], tuple(g["rho"]), tuple(g["c"]), tuple(g["k"]))
    assert mat.drho != 0.0
    if mesh == "tet":
        w = ellipsoid_tet_td(h=1.5e-3, axes=(0.024, 0.018, 0.014), n_steps=1200)
    else:
        w = cube_hex_td_convective(n=12)
    p = copy.copy(w.problem)
    p.material = mat
    orc = Oracle(p)
    dt = 0.5 * critical_dt(orc)
    ref = orc.run(dt, 800)
    f = ff()
    T, info = run_gpu(p, dt, 800, getattr(f, prec_name))
    assert info["dt_cr"] == pytest.approx(critical_dt(orc), rel=1e-9)
    err = max_abs(T, ref)
    print(f"Section 3.1.6 laws, {mesh} {p.n_nodes} nodes {prec_name}: max|dT| = {err:.3e}, max T = {ref.max():.2f}")
    assert err <= (TOL64 if prec_name == "FP64" else TOL32)
