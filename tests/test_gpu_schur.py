"""GPU parity of the Schur-complement solver (ba_options.solver = 1): PCG on the camera
Schur complement S = H'cc - Hcp H'pp^-1 Hpc with block-Jacobi on the camera blocks and
the points back-substituted, against the oracle's solver="schur".

Bars as for the default solver: final LM cost within 1e-4 relative (mixed), the same
LM iteration count, PCG counts of the early LM steps within 2.
"""
import dataclasses

import numpy as np
import pytest

from oracle import ba_oracle as O
from paper_2605_30583_gb300 import synth

pytestmark = pytest.mark.gpu
OPTS = dict(max_lm_iters=10, max_pcg_iters=50)


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_30583_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _check(res, ref, tol=1e-4):
    assert res.status == 0 and res.lm_iters == ref.lm_iters
    assert abs(res.final_cost - ref.final_cost) <= tol * ref.final_cost, (res.final_cost, ref.final_cost)
    for h, o in zip(res.history[:3], ref.history[:3]):
        assert abs(h["pcg_iters"] - o["pcg_iters"]) <= 2 and h["accepted"] == o["accepted"], (h, o)


@pytest.mark.parametrize("use_graph", [1, 2, 0])
def test_schur_solve_matches_oracle(B, use_graph):
    prob = synth.round_to_f32(synth.make_config("tiny", seed=71))
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels)
    p.set_params(prob.cams_init, prob.pts_init)
    res = p.solve(solver=1, use_graph=use_graph, **OPTS)
    ref = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels,
                     O.LMOptions(solver="schur", **OPTS))
    _check(res, ref)


def test_schur_with_retraction_and_robust_loss(B):
    prob = synth.make_config("tiny", seed=72)
    rng = np.random.default_rng(0)
    px = prob.pixels.copy()
    idx = rng.choice(prob.n_obs, prob.n_obs // 20, replace=False)
    px[idx] += 40.0 * rng.choice([-1.0, 1.0], size=(len(idx), 2))
    prob = synth.round_to_f32(dataclasses.replace(prob, pixels=px))
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels)
    p.set_params(prob.cams_init, prob.pts_init)
    res = p.solve(solver=1, rotation_update=1, loss=1, loss_scale=2.0, **OPTS)
    ref = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels,
                     O.LMOptions(solver="schur", rotation_update="retraction", loss="huber", loss_scale=2.0, **OPTS))
    _check(res, ref)


def test_schur_on_the_medium_workload_reaches_the_oracle_cost(B):
    """The medium workload, 20 LM x <= 50 PCG: the Schur solver reaches the cost the
    FP64 oracle's default solver reaches (same optimum, within 1e-4)."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_lm_medium.json")))["fp64"]
    prob = synth.make_config("medium")
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels)
    p.set_params(prob.cams_init, prob.pts_init)
    res = p.solve(solver=1)
    assert res.status == 0
    assert abs(res.final_cost - gold["final_cost"]) <= 1e-4 * gold["final_cost"], (res.final_cost, gold["final_cost"])


def test_schur_is_rejected_for_the_fp64_form(B):
    prob = synth.make_config("tiny", seed=73)
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels, precision="fp64")
    p.set_params(prob.cams_init, prob.pts_init)
    with pytest.raises(B.BAError) as e:
        p.solve(solver=1)
    assert e.value.status == 6
