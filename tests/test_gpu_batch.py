"""Batched planning runs (scenario lanes x element groups, one launch) and
CUDA-graph replay.  A batched run must be bit-identical to the same run
stepped alone; one run is also checked against the FP64 oracle."""
import numpy as np
import pytest

from oracle import Oracle
from synth.scenarios import planning_batch

from gpu_util import ff, max_abs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_batch():
    return planning_batch(n_meshes=3, n_scenarios=4, n_range=(900, 4000), base_seed=100)


@pytest.mark.parametrize("kernel_name", ["KERNEL_TILED", "KERNEL_TILED_STAGED"])
def test_batched_runs_equal_single_runs(small_batch, kernel_name):
    f = ff()
    meshes = [pm.problems for pm in small_batch]
    b = f.Batch(meshes, kernel=getattr(f, kernel_name))
    try:
        dt = 0.5 * b.dt_cr
        f.fedfem_step(b.ctx, dt, 150)
        assert f.fedfem_sync(b.ctx) == 150
        for g, scen in enumerate(meshes):
            for s_i, p in enumerate(scen):
                s = f.Solver(p, precision=f.FP32_KAHAN, kernel=f.KERNEL_PERSISTENT)
                try:
                    assert dt < s.dt_cr
                    s.step(dt, 150)
                    s.sync()
                    single = s.temperature()
                finally:
                    s.close()
                got = b.temperature(g, s_i)
                assert np.array_equal(got, single), (g, s_i, max_abs(got, single))
                assert got.max() > 37.5          # every lane saw its own source
    finally:
        b.close()


def test_batched_run_matches_oracle(small_batch):
    f = ff()
    meshes = [pm.problems for pm in small_batch]
    b = f.Batch(meshes)
    try:
        dt = 0.5 * b.dt_cr
        f.fedfem_step(b.ctx, dt, 300)
        f.fedfem_sync(b.ctx)
        for g, s_i in ((0, 3), (2, 1)):
            ref = Oracle(meshes[g][s_i]).run(dt, 300)
            err = max_abs(b.temperature(g, s_i), ref)
            print(f"batch mesh {g} scenario {s_i}: max|dT| vs oracle = {err:.3e}")
            assert err <= 1e-3
    finally:
        b.close()


def test_graph_replay_equals_direct_steps(small_batch):
    f = ff()
    p = small_batch[0].problems[0]
    for kern in (f.KERNEL_PERSISTENT, f.KERNEL_TILED):
        direct = f.Solver(p, kernel=kern)
        graph = f.Solver(p, kernel=kern)
        try:
            dt = 0.5 * direct.dt_cr
            direct.step(dt, 120)
            direct.sync()
            f.fedfem_capture_graph(graph.ctx, dt, 40)
            for _ in range(3):
                f.fedfem_replay_graph(graph.ctx)
            assert graph.sync() == 120
            assert np.array_equal(graph.temperature(), direct.temperature())
        finally:
            direct.close()
            graph.close()
    meshes = [pm.problems for pm in small_batch]
    b1, b2 = f.Batch(meshes), f.Batch(meshes)
    try:
        dt = 0.5 * b1.dt_cr
        f.fedfem_step(b1.ctx, dt, 60)
        f.fedfem_capture_graph(b2.ctx, dt, 20)
        for _ in range(3):
            f.fedfem_replay_graph(b2.ctx)
        f.fedfem_sync(b1.ctx)
        f.fedfem_sync(b2.ctx)
        for lane in range(4):
            assert np.array_equal(f.fedfem_read_temperature_lane(b1.ctx, lane),
                                  f.fedfem_read_temperature_lane(b2.ctx, lane))
    finally:
        b1.close()
        b2.close()
