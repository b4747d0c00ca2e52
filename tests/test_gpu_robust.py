"""GPU parity of the robust losses (ba_options.loss: 1 Huber, 2 Cauchy; IRLS weights
rho'(|r|^2) at the linearisation point) against the oracle's loss="huber"/"cauchy",
on data with gross outliers (5 % of the pixels moved by +-40 px).

Bars: final cost within 1e-4 relative (mixed) or 1e-8 (plain FP64), the same LM
iteration count, PCG counts of the early steps within 2.
"""
import dataclasses

import numpy as np
import pytest

from oracle import ba_oracle as O
from paper_2605_30583_gb300 import synth

pytestmark = pytest.mark.gpu
OPTS = dict(max_lm_iters=10, max_pcg_iters=50)
LOSS = {"huber": 1, "cauchy": 2}


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_30583_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _outliers(p, seed, frac=0.05, size=40.0):
    rng = np.random.default_rng(seed)
    px = p.pixels.copy()
    idx = rng.choice(p.n_obs, int(frac * p.n_obs), replace=False)
    px[idx] += size * rng.choice([-1.0, 1.0], size=(len(idx), 2))
    return dataclasses.replace(p, pixels=px)


@pytest.mark.parametrize("loss", ["huber", "cauchy"])
@pytest.mark.parametrize("pcg_kernel", [0, 1, 2])
def test_robust_solve_matches_oracle(B, loss, pcg_kernel):
    prob = synth.round_to_f32(_outliers(synth.make_config("tiny", seed=61), 1))
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels)
    p.set_params(prob.cams_init, prob.pts_init)
    res = p.solve(loss=LOSS[loss], loss_scale=2.0, pcg_kernel=pcg_kernel, **OPTS)
    ref = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels,
                     O.LMOptions(loss=loss, loss_scale=2.0, **OPTS))
    assert res.status == 0 and res.lm_iters == ref.lm_iters
    assert abs(res.initial_cost - ref.initial_cost) <= 1e-6 * ref.initial_cost
    assert abs(res.final_cost - ref.final_cost) <= 1e-4 * ref.final_cost, (res.final_cost, ref.final_cost)
    for h, o in zip(res.history[:3], ref.history[:3]):
        assert abs(h["pcg_iters"] - o["pcg_iters"]) <= 2 and h["accepted"] == o["accepted"]


@pytest.mark.parametrize("loss", ["huber", "cauchy"])
def test_robust_fp64_matches_oracle(B, loss):
    prob = _outliers(synth.make_config("tiny", seed=62), 2)
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels, precision="fp64")
    p.set_params(prob.cams_init, prob.pts_init)
    res = p.solve(loss=LOSS[loss], loss_scale=2.0, **OPTS)
    ref = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels,
                     O.LMOptions(loss=loss, loss_scale=2.0, **OPTS))
    assert res.status == 0 and res.lm_iters == ref.lm_iters
    assert abs(res.final_cost - ref.final_cost) <= 1e-8 * ref.final_cost, (res.final_cost, ref.final_cost)
    for h, o in zip(res.history[:3], ref.history[:3]):
        assert abs(h["pcg_iters"] - o["pcg_iters"]) <= 1 and h["accepted"] == o["accepted"]


def test_robust_loss_is_rejected_by_the_batched_mode(B):
    probs = synth.make_batch(2, seed=63000, cams=(5, 6), pts=(200, 220))
    b = B.Batch(probs)
    b.set_params(np.concatenate([q.cams_init for q in probs]), np.concatenate([q.pts_init for q in probs]))
    with pytest.raises(B.BAError) as e:
        b.solve(loss=1)
    assert e.value.status == 6


def test_evaluate_after_a_robust_solve_is_the_squared_cost(B):
    prob = synth.round_to_f32(_outliers(synth.make_config("tiny", seed=64), 3))
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels)
    p.set_params(prob.cams_init, prob.pts_init)
    p.solve(loss=2, loss_scale=2.0, max_lm_iters=2)
    p.set_params(prob.cams_init, prob.pts_init)
    F, _, _ = p.evaluate()
    ref = O.cost(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels)
    assert abs(F - ref) <= 1e-6 * ref
