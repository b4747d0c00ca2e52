"""GPU parity of the tangent-space rotation update (ba_options.rotation_update = 1):
rotations step as R <- Exp(d) R(w) with the Jacobian taken w.r.t. d (the paper's Pose3
update, Sec. VI-A), against the oracle's rotation_update="retraction".

Bars as for the additive update: final LM cost within 1e-4 relative (mixed) or 1e-8
(plain FP64), the same LM iteration count, PCG counts of the early LM steps within 2.
"""
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


def _oracle(prob, **kw):
    return O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels,
                      O.LMOptions(rotation_update="retraction", **kw))


@pytest.mark.parametrize("use_graph,pcg_kernel", [(1, 0), (2, 1), (0, 0)])
def test_retraction_solve_matches_oracle(B, use_graph, pcg_kernel):
    prob = synth.round_to_f32(synth.make_config("tiny", seed=51))
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels)
    p.set_params(prob.cams_init, prob.pts_init)
    res = p.solve(use_graph=use_graph, pcg_kernel=pcg_kernel, rotation_update=1, **OPTS)
    ref = _oracle(prob, **OPTS)
    assert res.status == 0 and res.lm_iters == ref.lm_iters
    assert abs(res.final_cost - ref.final_cost) <= 1e-4 * ref.final_cost, (res.final_cost, ref.final_cost)
    for h, o in zip(res.history[:3], ref.history[:3]):
        assert abs(h["pcg_iters"] - o["pcg_iters"]) <= 2 and h["accepted"] == o["accepted"]
    # the returned parameters carry the composed rotations: they reproduce the final cost
    c, q = p.get_params()
    F = O.cost(c, q, prob.cam_idx, prob.pt_idx, prob.pixels)
    assert abs(F - res.final_cost) <= 1e-5 * res.final_cost


@pytest.mark.parametrize("use_graph", [1, 0])
def test_retraction_fp64_matches_oracle(B, use_graph):
    prob = synth.make_config("tiny", seed=52)
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels, precision="fp64")
    p.set_params(prob.cams_init, prob.pts_init)
    res = p.solve(use_graph=use_graph, rotation_update=1, **OPTS)
    ref = _oracle(prob, **OPTS)
    assert res.status == 0 and res.lm_iters == ref.lm_iters
    assert abs(res.final_cost - ref.final_cost) <= 1e-8 * ref.final_cost, (res.final_cost, ref.final_cost)
    for h, o in zip(res.history[:3], ref.history[:3]):
        assert abs(h["pcg_iters"] - o["pcg_iters"]) <= 1 and h["accepted"] == o["accepted"]
    c, q = p.get_params()
    ref_c, ref_q = O.unpack(ref.x, prob.n_cams)
    # same gauge and start, FP64 on both sides: the rotations themselves agree
    assert np.allclose(c[:, 0:3], ref_c[:, 0:3], atol=1e-6)


def test_retraction_batch_matches_oracle(B):
    probs = [synth.round_to_f32(q) for q in synth.make_batch(6, seed=53000, cams=(5, 15), pts=(200, 800))]
    b = B.Batch(probs)
    b.set_params(np.concatenate([q.cams_init for q in probs]), np.concatenate([q.pts_init for q in probs]))
    res = b.solve(rotation_update=1, **OPTS)
    for q, r in zip(probs, res):
        ref = _oracle(q, **OPTS)
        assert r.status == 0 and r.lm_iters == ref.lm_iters
        assert abs(r.final_cost - ref.final_cost) <= 1e-4 * ref.final_cost


def test_evaluate_stays_additive_after_a_retraction_solve(B):
    prob = synth.round_to_f32(synth.make_config("tiny", seed=54))
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels)
    p.set_params(prob.cams_init, prob.pts_init)
    p.solve(rotation_update=1, max_lm_iters=2)
    p.set_params(prob.cams_init, prob.pts_init)
    _, _, J = p.evaluate(jacobian=True)
    _, Jc, _ = O.jacobian_blocks(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels)
    J = J.cpu().numpy()
    err = np.linalg.norm(J[:, :, :9] - Jc, axis=(1, 2)) / np.linalg.norm(Jc, axis=(1, 2))
    assert err.max() < 1e-4
