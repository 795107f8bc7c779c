"""Time-varying sources (Algorithm 1's per-step load update; the two-stage
heating and relaxation of Section 3.1.5) and the CEM43 thermal dose on the
GPU, against the FP64 oracle, across every kernel, with scenario lanes and
through a checkpoint."""
import copy

import numpy as np
import pytest

from oracle import Oracle, critical_dt
from synth.scenarios import cube_hex_fp64, planning_batch

from gpu_util import ff, max_abs

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-9, 1e-3
N_STEPS = 400


@pytest.fixture(scope="module")
def two_stage():
    """The 11^3 cube heated for 400 s, then relaxing (about half the run each)."""
    w = cube_hex_fp64()
    p = copy.copy(w.problem)
    p.schedule_end = np.array([400.0, 1e30])
    p.schedule_factor = np.array([1.0, 0.0])
    orc = Oracle(p)
    dt = 0.5 * critical_dt(orc)
    T, D = orc.run(dt, N_STEPS, dose=True)
    return p, dt, T, D


def _run(p, dt, prec, kernel=None, n=N_STEPS):
    f = ff()
    kw = {} if kernel is None else {"kernel": kernel}
    s = f.Solver(p, precision=prec, dose=True, **kw)
    try:
        s.step(dt, n)
        assert s.sync() == n
        return s.temperature(), s.dose()
    finally:
        s.close()


@pytest.mark.parametrize("prec_name", ["FP64", "FP32_KAHAN"])
def test_two_stage_heating_and_dose_match_the_oracle(two_stage, prec_name):
    p, dt, T_ref, D_ref = two_stage
    f = ff()
    T, D = _run(p, dt, getattr(f, prec_name))
    err = max_abs(T, T_ref)
    rel = np.max(np.abs(D - D_ref) / D_ref)
    print(f"two-stage {prec_name}: max|dT| = {err:.3e} (max T {T_ref.max():.2f} at the end), "
          f"dose max {D_ref.max():.3e} min, max rel dose error {rel:.2e}")
    assert T_ref.max() < 43.0 < Oracle(p).run(dt, N_STEPS // 2).max()   # the source was on, then off
    if prec_name == "FP64":
        assert err <= TOL64 and rel <= 1e-12
    else:
        assert err <= TOL32 and rel <= 1e-4


def test_every_kernel_gives_the_same_field_and_dose(two_stage):
    p, dt, _, _ = two_stage
    f = ff()
    T0, D0 = _run(p, dt, f.FP32_KAHAN, f.KERNEL_PERSISTENT, n=150)
    for kern in (f.KERNEL_TWO_PHASE, f.KERNEL_TILED, f.KERNEL_TILED_STAGED):
        T, D = _run(p, dt, f.FP32_KAHAN, kern, n=150)
        assert np.array_equal(T, T0) and np.array_equal(D, D0), kern


def test_checkpoint_carries_the_dose(two_stage):
    p, dt, _, _ = two_stage
    f = ff()
    T_straight, D_straight = _run(p, dt, f.FP64, f.KERNEL_TILED, n=300)
    a = f.Solver(p, precision=f.FP64, dose=True, kernel=f.KERNEL_TILED)
    try:
        a.step(dt, 170)
        a.sync()
        state = f.fedfem_get_state(a.ctx)
    finally:
        a.close()
    b = f.Solver(p, precision=f.FP64, dose=True, kernel=f.KERNEL_PERSISTENT)
    try:
        f.fedfem_set_state(b.ctx, state)
        b.step(dt, 130)
        assert b.sync() == 300
        assert np.array_equal(b.temperature(), T_straight)
        assert np.array_equal(b.dose(), D_straight)
    finally:
        b.close()


@pytest.mark.parametrize("kernel_name", ["KERNEL_TILED", "KERNEL_TILED_STAGED"])
def test_schedule_and_dose_with_scenario_lanes_equal_single_runs(kernel_name):
    f = ff()
    meshes = [pm.problems for pm in planning_batch(n_meshes=2, n_scenarios=4, n_range=(900, 3000), base_seed=7)]
    sched = (np.array([30.0, 1e30]), np.array([1.0, 0.25]))
    b = f.Batch(meshes, kernel=getattr(f, kernel_name), schedule=sched, dose=True)
    try:
        dt = 0.5 * b.dt_cr
        f.fedfem_step(b.ctx, dt, 120)
        assert f.fedfem_sync(b.ctx) == 120
        for g, scen in enumerate(meshes):
            for s_i in (0, 3):
                p = copy.copy(scen[s_i])
                p.schedule_end, p.schedule_factor = sched
                s = f.Solver(p, precision=f.FP32_KAHAN, kernel=f.KERNEL_PERSISTENT, dose=True)
                try:
                    s.step(dt, 120)
                    s.sync()
                    assert np.array_equal(b.temperature(g, s_i), s.temperature()), (g, s_i)
                    assert np.array_equal(b.dose(g, s_i), s.dose()), (g, s_i)
                finally:
                    s.close()
    finally:
        b.close()


def test_unsupported_combinations_are_refused(two_stage):
    p, dt, _, _ = two_stage
    f = ff()
    s = f.Solver(p, precision=f.FP32_KAHAN)
    try:
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_capture_graph(s.ctx, dt, 10)
        assert e.value.code == f.E_UNSUPPORTED
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_set_source_schedule(s.ctx, [2.0, 1.0], [1.0, 0.0])
        assert e.value.code == f.E_ARG
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_read_dose(s.ctx)
        assert e.value.code == f.E_STATE
    finally:
        s.close()
    meshes = [pm.problems for pm in planning_batch(n_meshes=1, n_scenarios=2, n_range=(900, 1200), base_seed=3)]
    b = f.Batch(meshes, dose=True)
    try:
        with pytest.raises(f.FedfemError) as e:
            f.fedfem_read_dose(b.ctx, 4)
        assert e.value.code == f.E_ARG
    finally:
        b.close()


ARR = ("arrhenius", 7.39e39, 2.577e5)   # liver coagulation parameters often used


@pytest.fixture(scope="module")
def two_stage_damage(two_stage):
    p, dt, _, _ = two_stage
    T, D = Oracle(p).run(dt, N_STEPS, dose=ARR)
    return p, dt, T, D


@pytest.mark.parametrize("prec_name", ["FP64", "FP32_KAHAN"])
def test_arrhenius_damage_matches_the_oracle(two_stage_damage, prec_name):
    p, dt, T_ref, D_ref = two_stage_damage
    f = ff()
    s = f.Solver(p, precision=getattr(f, prec_name), dose=ARR)
    try:
        s.step(dt, N_STEPS)
        assert s.sync() == N_STEPS
        T, D = s.temperature(), s.dose()
    finally:
        s.close()
    rel = np.max(np.abs(D - D_ref) / D_ref)
    print(f"Arrhenius {prec_name}: Omega in [{D_ref.min():.3e}, {D_ref.max():.3e}], max rel error {rel:.2e}")
    assert D_ref.max() > 1.0                      # the heated core coagulates
    if prec_name == "FP64":
        assert max_abs(T, T_ref) <= TOL64 and rel <= 1e-12
    else:
        assert max_abs(T, T_ref) <= TOL32 and rel <= 1e-4


def test_arrhenius_is_the_same_in_every_kernel_and_arguments_are_checked(two_stage):
    p, dt, _, _ = two_stage
    f = ff()
    out = []
    for kern in (f.KERNEL_PERSISTENT, f.KERNEL_TWO_PHASE, f.KERNEL_TILED, f.KERNEL_TILED_STAGED):
        s = f.Solver(p, precision=f.FP32_KAHAN, kernel=kern, dose=ARR)
        try:
            s.step(dt, 150)
            s.sync()
            out.append(s.dose())
            if kern == f.KERNEL_PERSISTENT:
                for args in [(2, 1.0, 1.0), (f.DOSE_ARRHENIUS, 0.0, 1.0), (f.DOSE_ARRHENIUS, 1.0, -1.0),
                             (f.DOSE_ARRHENIUS, float("inf"), 1.0)]:
                    with pytest.raises(f.FedfemError) as e:
                        f.fedfem_set_dose_model(s.ctx, *args)
                    assert e.value.code == f.E_ARG, args
        finally:
            s.close()
    for D in out[1:]:
        assert np.array_equal(D, out[0])
