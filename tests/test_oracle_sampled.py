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
