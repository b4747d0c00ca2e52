"""GPU parity of the plain all-FP64 form against the FP64 oracle.

Both sides compute in FP64 on identical inputs, so the tolerances follow FP64 rounding:
residuals and Jacobian blocks to 1e-11 relative (a pixel of ~500 px after ~30
operations), the normal operator to 1e-10, and final LM costs to 1e-8 relative (the
two trajectories differ only by summation order inside PCG).
"""
import json
import os

import numpy as np
import pytest

from oracle import ba_oracle as O
from paper_2605_30583_gb300 import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_30583_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _problem(B, prob):
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels, precision="fp64")
    p.set_params(prob.cams_init, prob.pts_init)
    return p


def test_fp64_residuals_and_jacobian(B):
    prob = synth.make_config("tiny", seed=31)
    p = _problem(B, prob)
    cost, r, J = p.evaluate(residuals=True, jacobian=True)
    ref_r, Jc, Jp = O.jacobian_blocks(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels)
    r = r.cpu().numpy()
    J = J.cpu().numpy()
    assert np.linalg.norm(r - ref_r) <= 1e-11 * np.linalg.norm(ref_r)
    assert abs(cost - 0.5 * float(np.sum(ref_r ** 2))) <= 1e-11 * cost
    err_c = np.linalg.norm(J[:, :, :9] - Jc, axis=(1, 2)) / np.linalg.norm(Jc, axis=(1, 2))
    err_p = np.linalg.norm(J[:, :, 9:] - Jp, axis=(1, 2)) / np.linalg.norm(Jp, axis=(1, 2))
    assert err_c.max() < 1e-11 and err_p.max() < 1e-11, (err_c.max(), err_p.max())


def test_fp64_normal_operator(B):
    import torch
    prob = synth.make_config("tiny", seed=32)
    p = _problem(B, prob)
    p.evaluate()
    lin = O.linearize(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels)
    D = O.damping_diag(lin.J)
    rng = np.random.default_rng(2)
    n = 9 * prob.n_cams + 3 * prob.n_pts
    for mu in (0.0, 0.01, 2.0):
        v = rng.standard_normal(n)
        out, vav = p.apply_normal(mu, torch.from_numpy(v))
        ref = O.normal_matvec(lin, D, mu, v)
        assert np.linalg.norm(out.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)
        assert abs(vav - v @ ref) <= 1e-10 * abs(v @ ref)


@pytest.mark.parametrize("use_graph", [1, 2, 0])
def test_fp64_lm_solve_matches_oracle(B, use_graph):
    prob = synth.make_config("tiny", seed=33)
    opts = dict(max_lm_iters=10, max_pcg_iters=50)
    res = _problem(B, prob).solve(use_graph=use_graph, **opts)
    ref = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels, O.LMOptions(**opts))
    assert res.status == 0 and res.lm_iters == ref.lm_iters
    assert abs(res.initial_cost - ref.initial_cost) <= 1e-11 * ref.initial_cost
    assert abs(res.final_cost - ref.final_cost) <= 1e-8 * ref.final_cost, (res.final_cost, ref.final_cost)
    # FP64 on both sides: the PCG iteration counts of the early LM steps agree exactly
    for h, o in zip(res.history[:3], ref.history[:3]):
        assert abs(h["pcg_iters"] - o["pcg_iters"]) <= 1
        assert h["accepted"] == o["accepted"]


def test_fp64_tiny_matches_stored_oracle_cost(B):
    """The tiny workload (16 cameras, 1,000 points), 20 LM x 50 PCG, against the stored
    oracle result written by tests/golden/make_golden.py."""
    gold = json.load(open(os.path.join(GOLDEN, "oracle_lm_tiny.json")))["fp64"]
    prob = synth.make_config("tiny")
    res = _problem(B, prob).solve(max_lm_iters=20, max_pcg_iters=50)
    assert prob.n_obs == gold["n_obs"]
    assert abs(res.final_cost - gold["final_cost"]) <= 1e-8 * gold["final_cost"]


def test_mixed_and_fp64_agree_on_final_cost(B):
    prob = synth.round_to_f32(synth.make_config("tiny", seed=34))
    a = _problem(B, prob).solve(max_lm_iters=12)
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels)
    p.set_params(prob.cams_init, prob.pts_init)
    b = p.solve(max_lm_iters=12)
    assert abs(a.final_cost - b.final_cost) <= 1e-4 * a.final_cost
