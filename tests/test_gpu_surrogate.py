"""Surrogate workflow on the GPU: training data from the plain path lowers the
training loss; an untrained (or badly perturbed) network fails every check,
so the fallback reproduces the plain path exactly."""
import numpy as np
import pytest

from synth.scenarios import cube_hex_fp64, source_density, surrogate_sources

from gpu_util import ff

pytestmark = pytest.mark.gpu


def test_fallback_reproduces_plain_path_and_training_lowers_loss():
    import torch
    ff()
    from paper_1909_05098_gb300.surrogate import PlainEnsemble, Surrogate, rollout
    p = cube_hex_fp64().problem
    src = surrogate_sources(24, seed=3)
    q = source_density(p.xyz, src)
    ens = PlainEnsemble(p, q)
    try:
        dt = 0.5 * ens.dt_cr
        W = 50
        T0 = torch.full((len(src), p.n_nodes), 37.0, dtype=torch.float64, device="cuda")
        ens.set_state(T0)
        states = [T0.float()]
        for _ in range(8):
            ens.step(dt, W)
            states.append(ens.state().float())
        T_plain_20 = ens.state()
        sur = Surrogate(p, window=W, max_batch=16, seed=1)
        try:
            S = torch.stack(states, 1)
            T_in = S[:, :-1].reshape(-1, p.n_nodes).contiguous()
            T_out = S[:, 1:].reshape(-1, p.n_nodes).contiguous()
            q32 = torch.tensor(q, dtype=torch.float32, device="cuda")
            q_in = q32[:, None, :].expand(-1, 8, -1).reshape(-1, p.n_nodes).contiguous()
            # a corrupted network (decoder bias +5 degC) fails every check: result == plain path
            good = ff().fedfem_mpnn_get_params(sur.net)
            bad = good.copy()
            bad[-1] = 5.0
            ff().fedfem_mpnn_set_params(sur.net, bad)
            res = rollout(sur, ens, q32, T0, dt, n_windows=2, check_every=4, budget=1e-4)
            ff().fedfem_mpnn_set_params(sur.net, good)
            assert res.rejected == res.checks == 2 * len(src)
            # re-initialising the plain path from (hi + lo) can re-split a Kahan pair that sits on a
            # rounding tie, so the fallback matches the uninterrupted run to FP32+Kahan accuracy
            d = float((res.T - T_plain_20).abs().max())
            print(f"fallback vs uninterrupted plain run: max |dT| = {d:.3e}")
            assert d <= 1e-5
            e_untrained = rollout(sur, ens, q32, T0, dt, n_windows=1, check_every=2, budget=1e9).max_check_error
            losses = sur.train(T_in, q_in, T_out, epochs=12, batch=16, lr=2e-3)
            e_trained = rollout(sur, ens, q32, T0, dt, n_windows=1, check_every=2, budget=1e9).max_check_error
            # an unbounded budget accepts every finite check: surrogate steps are taken, no NaN
            res = rollout(sur, ens, q32, T0, dt, n_windows=2, check_every=4, budget=1e9)
            print(f"loss {np.mean(losses[:5]):.3e} -> {np.mean(losses[-5:]):.3e}; first-window check error "
                  f"{e_untrained:.3f} -> {e_trained:.3f} degC")
            assert np.mean(losses[-5:]) < 0.3 * np.mean(losses[:5])
            assert res.rejected == 0 and res.surrogate_steps == 2 * 3 * len(src)
            assert bool(torch.isfinite(res.T).all())
            assert e_trained < e_untrained
        finally:
            sur.close()
    finally:
        ens.close()
