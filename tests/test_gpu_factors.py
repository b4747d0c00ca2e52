"""Pose factors (relative-pose factors between cameras) on the GPU against the oracle.

Inputs are rounded to FP32 (parameters, pixels); the measurements stay FP64 on both
sides.  Bars as for the reprojection-only path: cost 1e-5 relative, normal operator
1e-4 relative, final LM cost 1e-4 relative, same LM iteration count.
"""
import numpy as np
import pytest

from oracle import ba_oracle as O
from paper_2605_30583_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_30583_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _case(seed=3, pairs="chain+skip", n_cams=None):
    kw = dict(seed=seed) if n_cams is None else dict(seed=seed, n_cams=n_cams)
    prob = synth.round_to_f32(synth.make_config("tiny", **kw))
    fa, fb, meas, sq = synth.make_pose_factors(prob, pairs=pairs, seed=seed)
    sq = 4.0 * sq   # weigh the factors up against the many observations
    return prob, (fa, fb, meas, sq), O.PoseFactors(fa, fb, meas, sq)


def _problem(B, prob, fac):
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels, pose_factors=fac)
    p.set_params(prob.cams_init, prob.pts_init)
    return p


def test_cost_with_factors_matches_oracle(B):
    prob, fac, f = _case()
    p = _problem(B, prob, fac)
    cost, _, _ = p.evaluate()
    ref = O.cost(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels) + \
        O.pose_factor_cost(prob.cams_init, f)
    assert O.pose_factor_cost(prob.cams_init, f) > 0.01 * ref   # the factors weigh in
    assert abs(cost - ref) <= 1e-5 * ref, (cost, ref)


def test_normal_operator_with_factors_matches_oracle(B):
    import torch
    prob, fac, f = _case(seed=9)
    p = _problem(B, prob, fac)
    p.evaluate()
    lin = O.linearize(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels, factors=f)
    D = O.damping_diag(lin.J)
    rng = np.random.default_rng(0)
    n = 9 * prob.n_cams + 3 * prob.n_pts
    for mu in (0.0, 0.01, 3.0):
        v = rng.standard_normal(n).astype(np.float32).astype(np.float64)
        out, vav = p.apply_normal(mu, torch.from_numpy(v))
        ref = O.normal_matvec(lin, D, mu, v)
        out = out.double().cpu().numpy()
        assert np.linalg.norm(out - ref) <= 1e-4 * np.linalg.norm(ref)
        assert abs(vav - v @ ref) <= 1e-4 * abs(v @ ref)
        # the camera part alone (where the factors act)
        nc = 9 * prob.n_cams
        assert np.linalg.norm(out[:nc] - ref[:nc]) <= 1e-4 * np.linalg.norm(ref[:nc])


# (use_graph, pcg_kernel): persistent two-exchange, one kernel per PCG step, persistent
# one-exchange, under the default graph, the unrolled graph and host launches
MODES = [(1, 0), (1, 1), (1, 2), (2, 0), (0, 1)]


@pytest.mark.parametrize("use_graph,pcg_kernel", MODES)
def test_solve_with_factors_matches_oracle(B, use_graph, pcg_kernel):
    prob, fac, f = _case(seed=11)
    p = _problem(B, prob, fac)
    opts = dict(max_lm_iters=12, max_pcg_iters=50)
    res = p.solve(use_graph=use_graph, pcg_kernel=pcg_kernel, **opts)
    ref = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels, O.LMOptions(**opts),
                     factors=f)
    assert res.status == 0
    assert res.lm_iters == ref.lm_iters
    assert abs(res.initial_cost - ref.initial_cost) <= 1e-5 * ref.initial_cost
    assert abs(res.final_cost - ref.final_cost) <= 1e-4 * ref.final_cost, (res.final_cost, ref.final_cost)
    for h, o in zip(res.history[:3], ref.history[:3]):
        assert abs(h["pcg_iters"] - o["pcg_iters"]) <= 2, (h, o)
    # the parameters on the device reproduce the reported cost
    c, q = p.get_params()
    F = O.cost(c, q, prob.cam_idx, prob.pt_idx, prob.pixels) + O.pose_factor_cost(c, f)
    assert abs(F - res.final_cost) <= 1e-5 * res.final_cost


def test_factors_with_retraction_and_robust_loss(B):
    prob, fac, f = _case(seed=13)
    opts = dict(max_lm_iters=10, max_pcg_iters=50)
    p = _problem(B, prob, fac)
    res = p.solve(rotation_update=1, loss=1, loss_scale=2.0, **opts)
    ref = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels,
                     O.LMOptions(rotation_update="retraction", loss="huber", loss_scale=2.0, **opts), factors=f)
    assert res.status == 0 and res.lm_iters == ref.lm_iters
    assert abs(res.final_cost - ref.final_cost) <= 1e-4 * ref.final_cost, (res.final_cost, ref.final_cost)


def test_exact_factors_pull_to_ground_truth(B):
    """Exact relative poses and noise-free pixels: the optimum has zero cost."""
    prob = synth.round_to_f32(synth.make_problem(8, 600, ("poisson", 3.0), "nearest", seed=21, noise_px=0.0))
    fa, fb, meas, sq = synth.make_pose_factors(prob, pairs="chain", noise=False)
    p = _problem(B, prob, (fa, fb, meas, sq))
    res = p.solve(max_lm_iters=30)
    assert res.status == 0
    assert res.final_cost < 1e-6 * res.initial_cost


def test_many_factors_more_than_ctas(B):
    """More factors than CTAs of the persistent kernel, factors on unobserved cameras."""
    prob = synth.round_to_f32(synth.make_config("tiny", seed=17, n_cams=40))
    fa, fb, meas, sq = synth.make_pose_factors(prob, pairs="chain+skip", seed=17)
    f = O.PoseFactors(fa, fb, meas, sq)
    opts = dict(max_lm_iters=8, max_pcg_iters=50)
    for k in (0, 2):
        p = _problem(B, prob, (fa, fb, meas, sq))
        res = p.solve(pcg_kernel=k, **opts)
        ref = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels, O.LMOptions(**opts),
                         factors=f)
        assert res.status == 0
        assert abs(res.final_cost - ref.final_cost) <= 1e-4 * ref.final_cost, (k, res.final_cost, ref.final_cost)


def test_rejections(B):
    prob, fac, f = _case()
    with pytest.raises(B.BAError) as e:
        B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels, precision="fp64",
                  pose_factors=fac)
    assert e.value.status == 6   # not implemented
    p = _problem(B, prob, fac)
    with pytest.raises(B.BAError) as e:
        p.solve(solver=1)
    assert e.value.status == 6   # not implemented


def test_cameras_held_only_by_factors_or_by_nothing(B):
    """Camera 3 loses its observations and is held by pose factors alone; camera 5 loses
    its observations and has no factor (its block is mu D alone, its step stays zero)."""
    base = synth.make_config("tiny", seed=23, n_cams=12)
    keep = (base.cam_idx != 3) & (base.cam_idx != 5)
    counts = np.bincount(base.pt_idx[keep], minlength=base.n_pts)
    live = counts >= 2                          # points that keep two views
    keep &= live[base.pt_idx]
    new_id = np.cumsum(live) - 1
    prob = synth.round_to_f32(synth.Problem(base.n_cams, int(live.sum()), base.cam_idx[keep],
                                            new_id[base.pt_idx[keep]].astype(np.uint32), base.pixels[keep],
                                            base.cams_init, base.pts_init[live], base.cams_gt, base.pts_gt[live],
                                            "tiny-holes"))
    assert not np.any(prob.cam_idx == 3) and not np.any(prob.cam_idx == 5)
    fa, fb, meas, sq = synth.make_pose_factors(prob, pairs="chain", seed=23)
    sel = (fa != 5) & (fb != 5)
    fac = (fa[sel], fb[sel], meas[sel], sq[sel])
    f = O.PoseFactors(*fac)
    opts = dict(max_lm_iters=10, max_pcg_iters=50)
    ref = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels, O.LMOptions(**opts),
                     factors=f)
    for k in (0, 1, 2):
        p = _problem(B, prob, fac)
        res = p.solve(pcg_kernel=k, **opts)
        assert res.status == 0 and res.lm_iters == ref.lm_iters
        assert abs(res.final_cost - ref.final_cost) <= 1e-4 * ref.final_cost, (k, res.final_cost, ref.final_cost)
        c, _ = p.get_params()
        np.testing.assert_allclose(c[5], prob.cams_init[5], rtol=0, atol=1e-6)   # untouched
        assert np.abs(c[3] - prob.cams_init[3]).max() > 1e-5                     # moved by its factors
