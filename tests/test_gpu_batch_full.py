"""The full batched-planning workload on the GPU: 64 seeded ellipsoid tet
meshes of uneven size (5k-170k nodes, 3.49M in all) x 4 source scenarios,
256 runs in one context, in the launch configuration the bench's autotuner
picks.  Sampled runs -- the largest and the smallest mesh and four others --
must be bit-identical to the same run stepped alone, and within 1e-3 degC of
the FP64 run of that problem."""
import numpy as np
import pytest

from synth.scenarios import planning_batch

from gpu_util import ff, max_abs

pytestmark = pytest.mark.gpu

N_STEPS = 200


def test_full_planning_batch_sampled_runs():
    from paper_1909_05098_gb300.autotune import tune
    f = ff()
    batch = planning_batch()
    meshes = [pm.problems for pm in batch]
    assert len(meshes) == 64 and all(len(s) == 4 for s in meshes)
    sizes = [s[0].n_nodes for s in meshes]
    b = f.Batch(meshes)
    try:
        dt = 0.5 * b.dt_cr
        tuned = tune(b, dt, use_cache=False, steps=20)
        print(f"batch kernel {tuned['kernel']} block {tuned['block']} tile {tuned['tile_nodes']}")
        f.fedfem_step(b.ctx, dt, N_STEPS)
        assert f.fedfem_sync(b.ctx) == N_STEPS
        rng = np.random.default_rng(4)
        picks = [int(np.argmax(sizes)), int(np.argmin(sizes))] + [int(g) for g in rng.choice(64, 4, replace=False)]
        for g in picks:
            s_i = int(rng.integers(4))
            p = meshes[g][s_i]
            got = b.temperature(g, s_i)
            single = f.Solver(p, precision=f.FP32_KAHAN, kernel=f.KERNEL_PERSISTENT)
            ref = f.Solver(p, precision=f.FP64, kernel=f.KERNEL_PERSISTENT)
            try:
                assert dt < single.dt_cr
                single.step(dt, N_STEPS)
                ref.step(dt, N_STEPS)
                single.sync()
                ref.sync()
                alone, T64 = single.temperature(), ref.temperature()
            finally:
                single.close()
                ref.close()
            err = max_abs(got, T64)
            print(f"mesh {g} ({sizes[g]} nodes) scenario {s_i}: max|dT| vs FP64 {err:.3e}, max T {T64.max():.2f}")
            assert np.array_equal(got, alone), (g, s_i, max_abs(got, alone))
            assert err <= 1e-3
    finally:
        b.close()
