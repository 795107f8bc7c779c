"""Hourglass-stabilised one-point hexahedron on the GPU against the FP64
oracle (oracle/elements.py: hex8_hourglass), on the 11^3 cube and on a
distorted hex mesh (interior nodes moved by up to 0.2 h, so the hourglass
weights are not zero), in every kernel family, plus its critical step and the
behaviour it exists for: an hourglass-shaped disturbance of an insulated block
decays with the stabilisation and stays forever without it."""
import copy

import numpy as np
import pytest

from oracle import Oracle, critical_dt
from synth.scenarios import cube_hex_fp64

from gpu_util import ff, max_abs

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-9, 1e-3
EPS = 0.2


def _distorted(p, seed=5, amount=0.2):
    q = copy.copy(p)
    rng = np.random.default_rng(seed)
    h = 1e-3
    interior = np.ones(p.n_nodes, dtype=bool)
    interior[p.dirichlet_nodes] = False
    q.xyz = p.xyz.copy()
    q.xyz[interior] += rng.uniform(-amount * h, amount * h, (int(interior.sum()), 3))
    return q


def _hg(p):
    q = copy.copy(p)
    q.hex_rule = "hourglass"
    q.hourglass_eps = EPS
    return q


@pytest.fixture(scope="module", params=["cube", "distorted"])
def case(request):
    p = cube_hex_fp64().problem
    if request.param == "distorted":
        p = _distorted(p)
    p = _hg(p)
    orc = Oracle(p)
    dt = 0.5 * critical_dt(orc)
    return request.param, p, orc, dt, orc.run(dt, 600)


def _run(p, dt, n, prec, kernel, block=0, tile=0):
    f = ff()
    s = f.Solver(p, precision=prec)
    try:
        f.fedfem_set_tile(s.ctx, kernel, block, tile, 0)
        s.step(dt, n)
        assert s.sync() == n
        return s.temperature(), s.dt_cr
    finally:
        s.close()


def test_hourglass_matches_the_oracle_in_every_kernel(case):
    name, p, orc, dt, ref = case
    f = ff()
    for prec, tol in ((f.FP64, TOL64), (f.FP32_KAHAN, TOL32)):
        base = None
        for kern in (f.KERNEL_TWO_PHASE, f.KERNEL_PERSISTENT, f.KERNEL_TILED, f.KERNEL_TILED_STAGED,
                     f.KERNEL_TILED_REP):
            T, dt_cr = _run(p, dt, 600, prec, kern)
            err = max_abs(T, ref)
            print(f"hourglass {name} prec {prec} kernel {kern}: max|dT| = {err:.3e}")
            assert err <= tol
            assert dt_cr == pytest.approx(critical_dt(orc), rel=1e-9)
            if base is None:
                base = T
            assert np.array_equal(T, base), kern            # every kernel gives the same bits


def test_hourglass_mode_decays_only_with_stabilisation():
    """An insulated 10^3 hex block (no Dirichlet, no sources, no perfusion)
    started from 37 degC plus a small x-y checkerboard (the hourglass pattern
    s_x s_y repeated over the grid): the one-point rule leaves it untouched
    (zero energy), the stabilised rule smooths it away; both keep the mean."""
    from synth.meshes import hex_box
    from synth.problem import Perfusion, Problem
    from synth.scenarios import TISSUE_CONST
    m = hex_box(10, 10, 10, 1e-3)
    g = m.grid_index
    T0 = 37.0 + 0.5 * (-1.0) ** (g[:, 0] + g[:, 1])
    p = Problem(8, m.xyz, m.conn, TISSUE_CONST, Perfusion(), T0=T0, T_lo=30.0, T_hi=45.0)
    f = ff()
    dt = 0.5 * critical_dt(Oracle(_hg(p)))
    plain, _ = _run(p, dt, 400, f.FP64, f.KERNEL_TILED_REP)
    stab, _ = _run(_hg(p), dt, 400, f.FP64, f.KERNEL_TILED_REP)
    amp_plain = np.max(np.abs(plain - 37.0))
    amp_stab = np.max(np.abs(stab - 37.0))
    print(f"checkerboard amplitude after 400 steps: plain {amp_plain:.3e}, stabilised {amp_stab:.3e}")
    assert amp_plain == pytest.approx(0.5, rel=1e-9)
    assert amp_stab < 0.05
    ref = Oracle(_hg(p)).run(dt, 400)
    assert max_abs(stab, ref) <= TOL64


def test_hourglass_refusals():
    f = ff()
    p = cube_hex_fp64().problem
    s = f.Solver(p, precision=f.FP64)
    try:
        with pytest.raises(f.FedfemError):
            f.fedfem_set_hourglass_control(s.ctx, -1.0)
    finally:
        s.close()
    q = _hg(p)
    q.hex_rule = "full"
    ctx = f.fedfem_create(0, f.FP64, None)
    try:
        f.fedfem_set_mesh(ctx, 8, q.xyz, q.conn)
        f.fedfem_set_hourglass_control(ctx, 0.1)
        f.fedfem_set_hex_integration(ctx, f.HEX_FULL)
        f.apply_material(ctx, q.material)
        with pytest.raises(f.FedfemError) as ei:
            f.fedfem_precompute(ctx, 30.0, 100.0)
        assert ei.value.code == f.E_UNSUPPORTED
    finally:
        f.fedfem_destroy(ctx)
