"""Uniform V/N lumping of perfusion and metabolic heat (the form of the
paper's verification runs, Sections 3.1.3-3.1.4) on the GPU against the FP64
oracle, and its refusals."""
import copy

import numpy as np
import pytest

from oracle import Oracle, critical_dt
from synth.problem import Perfusion
from synth.scenarios import cube_hex_fp64, ellipsoid_tet_td

from gpu_util import ff, max_abs, run_gpu

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-9, 1e-3


def _problem(mesh):
    if mesh == "hex":
        p = copy.copy(cube_hex_fp64().problem)
    else:
        p = copy.copy(ellipsoid_tet_td(h=1.5e-3, axes=(0.024, 0.018, 0.014), n_steps=1200).problem)
    p.lumping = "uniform"
    p.perfusion = Perfusion(w_b=26.6, c_b=3617.0, T_a=39.0, Q_m=33800.0)   # Sections 3.1.3-3.1.4
    return p


@pytest.mark.parametrize("mesh", ["hex", "tet"])
def test_uniform_lumping_matches_the_oracle(mesh):
    p = _problem(mesh)
    orc = Oracle(p)
    dt_cr = critical_dt(orc)
    dt = 0.5 * dt_cr
    ref = orc.run(dt, 500)
    element = copy.copy(p)
    element.lumping = "element"
    gap = max_abs(Oracle(element).run(dt, 500), ref)
    f = ff()
    for prec_name, kern in [("FP64", "KERNEL_PERSISTENT"), ("FP32_KAHAN", "KERNEL_PERSISTENT"),
                            ("FP32_KAHAN", "KERNEL_TILED_STAGED")]:
        T, info = run_gpu(p, dt, 500, getattr(f, prec_name), kernel=getattr(f, kern))
        assert info["dt_cr"] == pytest.approx(dt_cr, rel=1e-9)
        err = max_abs(T, ref)
        print(f"uniform lumping {mesh} {prec_name} {kern}: max|dT| = {err:.3e}; element vs uniform {gap:.3e} degC")
        assert err <= (TOL64 if prec_name == "FP64" else TOL32)
    assert gap > 1e-6


def test_uniform_lumping_refusals():
    f = ff()
    p = copy.copy(cube_hex_fp64().problem)
    s = f.Solver(p, precision=f.FP64)
    try:
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_set_lumping(s.ctx, 2)
        assert e.value.code == f.E_ARG
        f.fedfem_set_lumping(s.ctx, f.LUMP_UNIFORM)
        E = len(p.conn)
        f.fedfem_set_regions(s.ctx, (p.material, p.material), (p.perfusion, p.perfusion),
                             (np.arange(E) % 2).astype(np.int32))
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_precompute(s.ctx, 0.0, 100.0)
        assert e.value.code == f.E_UNSUPPORTED
    finally:
        s.close()
