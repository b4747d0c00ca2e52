"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Inputs are rounded to FP32 first, so both sides see bit-identical parameters and
pixels and only arithmetic differs.  Tolerances (derived from FP32 arithmetic):
  * residuals: |r_gpu - r_ref|_2 <= 1e-5 |r_ref|_2 at the initial point, and per
    element |dr| <= 2e-4 px + 1e-5 |r| (a pixel of ~500 px carries an FP32 rounding
    of ~3e-5 px per operation);
  * Jacobian blocks, normal operator: relative 2-norm error <= 1e-5 / 1e-4, and the
    operator per entry: |q_i - ref_i| <= 1e-4 s_i with s = |J|^T |J v| + mu D |v|, the
    sum of the magnitudes of the terms that make up entry i (an FP32 sum of terms
    carries an error of a few ulp of that scale, whatever their cancellation), so a
    wrong block anywhere shows up at its own entries;
  * final LM cost: relative error <= 1e-4.
"""
import dataclasses

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


def _problem(B, prob, precision="mixed"):
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels, precision=precision)
    p.set_params(prob.cams_init, prob.pts_init)
    return p


def _ragged(seed=3):
    # 1000 points = 3 full tiles of 256 plus a ragged tail of 232
    return synth.round_to_f32(synth.make_config("tiny", seed=seed))


def test_residuals_match_oracle(B):
    prob = _ragged()
    p = _problem(B, prob)
    cost, r, _ = p.evaluate(residuals=True)
    r = r.double().cpu().numpy()
    ref = O.residuals(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels)
    assert np.linalg.norm(r - ref) <= 1e-5 * np.linalg.norm(ref)
    assert np.all(np.abs(r - ref) <= 2e-4 + 1e-5 * np.abs(ref))
    ref_cost = 0.5 * float(np.sum(ref * ref))
    assert abs(cost - ref_cost) <= 1e-5 * ref_cost


def test_double_float_residuals_are_the_oracle_residuals_rounded(B):
    """Residual arithmetic of the mixed form.  Default (double-float, ~48 bits): each
    residual is the oracle's FP64 residual rounded to FP32, so it is within half an ulp
    of itself plus the double-float error (a few 2^-48 of the ~500 px terms): bound
    1.2e-7 |r| + 1e-8 px.  residual_precision 0 (FP32 arithmetic): the ~500 px terms
    carry ~1e-4 px of error, so the same bound fails and the FP32 bar of the other tests
    (2e-4 px + 1e-5 |r|) holds."""
    prob = _ragged(19)
    ref = O.residuals(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels)
    p = _problem(B, prob)
    _, r, _ = p.evaluate(residuals=True)
    err = np.abs(r.double().cpu().numpy() - ref)
    assert np.all(err <= 1.2e-7 * np.abs(ref) + 1e-8), err.max()
    p.solve(max_lm_iters=0, residual_precision=0)   # writes the options
    _, r32, _ = p.evaluate(residuals=True)
    err32 = np.abs(r32.double().cpu().numpy() - ref)
    assert np.all(err32 <= 2e-4 + 1e-5 * np.abs(ref))
    assert err32.max() > 10 * err.max()


def test_jacobian_matches_oracle(B):
    prob = _ragged(5)
    p = _problem(B, prob)
    _, _, J = p.evaluate(jacobian=True)
    J = J.double().cpu().numpy()
    _, Jc, Jp = O.jacobian_blocks(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels)
    err_c = np.linalg.norm(J[:, :, :9] - Jc, axis=(1, 2)) / np.linalg.norm(Jc, axis=(1, 2))
    err_p = np.linalg.norm(J[:, :, 9:] - Jp, axis=(1, 2)) / np.linalg.norm(Jp, axis=(1, 2))
    assert err_c.max() < 1e-5, err_c.max()
    assert err_p.max() < 1e-5, err_p.max()


def _with_repeats(prob, n_rep, seed):
    """The problem with n_rep observations repeated (same camera and point, the pixel
    moved by up to a pixel): a camera that sees a point twice."""
    rng = np.random.default_rng(seed)
    pick = rng.choice(prob.n_obs, size=n_rep, replace=False)
    px = prob.pixels[pick] + rng.uniform(-1.0, 1.0, size=(n_rep, 2))
    return synth.round_to_f32(dataclasses.replace(
        prob, cam_idx=np.concatenate([prob.cam_idx, prob.cam_idx[pick]]),
        pt_idx=np.concatenate([prob.pt_idx, prob.pt_idx[pick]]), pixels=np.concatenate([prob.pixels, px])))


@pytest.mark.parametrize("repeats", [0, 300])
def test_normal_operator_matches_oracle(B, repeats):
    """repeats = 0: the tile operator's warps add point sums into private copies;
    repeats > 0: repeated (camera, point) observations, which sit next to each other in
    a camera run, make it keep one copy with atomics."""
    import torch
    prob = _ragged(9)
    if repeats:
        prob = _with_repeats(prob, repeats, seed=4)
    p = _problem(B, prob)
    p.evaluate()
    lin = O.linearize(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels)
    D = O.damping_diag(lin.J)
    rng = np.random.default_rng(0)
    n = 9 * prob.n_cams + 3 * prob.n_pts
    for mu in (0.0, 0.01, 3.0):
        v = rng.standard_normal(n).astype(np.float32).astype(np.float64)
        out, vav = p.apply_normal(mu, torch.from_numpy(v))
        ref = O.normal_matvec(lin, D, mu, v)
        out = out.double().cpu().numpy()
        assert np.linalg.norm(out - ref) <= 1e-4 * np.linalg.norm(ref)
        Ja = abs(lin.J)
        scale = Ja.T @ (Ja @ np.abs(v)) + mu * D * np.abs(v)
        err = np.abs(out - ref) / scale
        assert err.max() <= 1e-4, (mu, int(err.argmax()), err.max())
        assert abs(vav - v @ ref) <= 1e-4 * abs(v @ ref)
        # adjointness of the operator: <A v, w> = <v, A w>
        w = rng.standard_normal(n).astype(np.float32).astype(np.float64)
        out_w, _ = p.apply_normal(mu, torch.from_numpy(w))
        a, b = float(out @ w), float(v @ out_w.double().cpu().numpy())
        assert abs(a - b) <= 1e-4 * (abs(a) + abs(b))


def test_lm_solve_with_repeated_observations_matches_oracle(B):
    prob = _with_repeats(_ragged(13), 400, seed=6)
    ref = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels,
                     O.LMOptions(max_lm_iters=10, max_pcg_iters=50))
    p = _problem(B, prob)
    res = p.solve(max_lm_iters=10, max_pcg_iters=50)
    assert res.status == 0
    assert abs(res.final_cost - ref.final_cost) <= 1e-4 * ref.final_cost, (res.final_cost, ref.final_cost)


def test_lm_solve_with_a_tile_beyond_the_shared_memory_sort(B):
    """90 cameras that all see the same 256 points: one tile of 23,040 observations, more
    than the 16,384 the bind sorts per tile in shared memory, so the observation order
    comes from the global sort; the solve (both PCG forms' inputs, the tile operator)
    still follows the oracle."""
    prob = synth.round_to_f32(synth.make_problem(90, 256, ("poisson", 1000.0), "uniform", seed=51))
    assert prob.n_obs > 16384
    ref = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels,
                     O.LMOptions(max_lm_iters=8, max_pcg_iters=50))
    for precision, tol in (("mixed", 1e-4), ("fp64", 1e-8)):
        p = _problem(B, prob, precision)
        res = p.solve(max_lm_iters=8, max_pcg_iters=50)
        assert res.status == 0
        assert abs(res.final_cost - ref.final_cost) <= tol * ref.final_cost, (precision, res.final_cost, ref.final_cost)
        p.close()


# (use_graph, pcg_kernel): conditional-loop graph / unrolled graph / host-launched
# sequence, with the persistent PCG kernel (0: two exchanges per iteration, 2: one),
# or separate kernels per PCG step (1: textbook recurrences, 3: one reduction a step)
MODES = [(g, k) for g in (1, 2, 0) for k in (0, 1, 2, 3)]


@pytest.mark.parametrize("use_graph,pcg_kernel", MODES)
def test_lm_solve_matches_oracle(B, use_graph, pcg_kernel):
    prob = _ragged(11)
    p = _problem(B, prob)
    opts = dict(max_lm_iters=12, max_pcg_iters=50)
    res = p.solve(use_graph=use_graph, pcg_kernel=pcg_kernel, **opts)
    ref = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels, O.LMOptions(**opts))
    assert res.status == 0
    assert res.lm_iters == ref.lm_iters
    assert abs(res.initial_cost - ref.initial_cost) <= 1e-5 * ref.initial_cost
    assert abs(res.final_cost - ref.final_cost) <= 1e-4 * ref.final_cost, (res.final_cost, ref.final_cost)
    # accepted steps strictly decrease the cost
    for h in res.history:
        if h["accepted"]:
            assert h["cost_new"] < h["cost"]
    # the parameters on the device reproduce the reported cost
    c, q = p.get_params()
    assert abs(O.cost(c, q, prob.cam_idx, prob.pt_idx, prob.pixels) - res.final_cost) <= 1e-5 * res.final_cost


def test_all_launch_modes_agree(B):
    prob = _ragged(13)
    res = [_problem(B, prob).solve(use_graph=g, pcg_kernel=k, max_lm_iters=8) for g, k in MODES]
    ref = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels,
                     O.LMOptions(max_lm_iters=8))
    for r in res:
        assert r.status == 0 and r.lm_iters == res[0].lm_iters
        assert abs(r.final_cost - res[0].final_cost) <= 1e-6 * res[0].final_cost
        # While the cost still falls well above the FP32 noise floor (the first LM
        # steps), each PCGNR solve takes the oracle's iteration count to within 2;
        # later steps sit at the noise floor, where the counts are not comparable.
        for h, o in zip(r.history[:4], ref.history[:4]):
            assert abs(h["pcg_iters"] - o["pcg_iters"]) <= 2, (h, o)


def test_pcg_step_matches_oracle_at_tight_tolerance(B):
    """One LM step with a tight CG tolerance: same PCGNR iteration count, same model
    decrease L = -g^T h - |J h|^2 / 2 (to FP32 accuracy), for both PCG forms."""
    prob = _ragged(13)
    opts = dict(max_lm_iters=1, pcg_rel_tol=1e-6, max_pcg_iters=200)
    ref = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels, O.LMOptions(**opts))
    for k in (0, 1, 2, 3):
        r = _problem(B, prob).solve(pcg_kernel=k, **opts)
        h, o = r.history[0], ref.history[0]
        assert abs(h["pcg_iters"] - o["pcg_iters"]) <= 2
        assert abs(h["model_decrease"] - o["model_decrease"]) <= 1e-5 * o["model_decrease"]
        assert abs(h["cost_new"] - o["cost_new"]) <= 1e-5 * o["cost_new"]


def test_repeated_solves_reuse_the_graph(B):
    prob = _ragged(17)
    p = _problem(B, prob)
    r1 = p.solve(max_lm_iters=5)
    p.set_params(prob.cams_init, prob.pts_init)
    r2 = p.solve(max_lm_iters=5)
    # switching the PCG form rebuilds the cached graph
    p.set_params(prob.cams_init, prob.pts_init)
    r3 = p.solve(max_lm_iters=5, pcg_kernel=1)
    assert abs(r3.final_cost - r1.final_cost) <= 1e-6 * r1.final_cost
    assert abs(r1.final_cost - r2.final_cost) <= 1e-6 * r1.final_cost
    # zero LM iterations: nothing changes, final cost = initial cost
    p.set_params(prob.cams_init, prob.pts_init)
    r0 = p.solve(max_lm_iters=0)
    assert r0.lm_iters == 0 and r0.final_cost == r0.initial_cost


def test_noise_free_ground_truth_has_zero_cost(B):
    prob = synth.make_problem(16, 300, ("poisson", 3.0), "uniform", seed=21, noise_px=0.0, perturb=False)
    prob = synth.round_to_f32(prob)
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels)
    p.set_params(prob.cams_gt.astype(np.float32), prob.pts_gt.astype(np.float32))
    cost, r, _ = p.evaluate(residuals=True)
    ref = O.residuals(prob.cams_gt.astype(np.float32).astype(np.float64),
                      prob.pts_gt.astype(np.float32).astype(np.float64), prob.cam_idx, prob.pt_idx, prob.pixels)
    # FP32 ulp of a ~500 px pixel is ~3e-5 px; the rounded inputs leave a residual of that order
    assert np.abs(r.double().cpu().numpy() - ref).max() < 2e-4


def test_single_tile_and_heavy_point(B):
    """One point seen by every camera (a 40-observation run in a tile) and tiny tiles.

    The problem is underdetermined (360 camera parameters against 5 points), so LM does
    not converge on it and the cost after 5 iterations depends on where each PCG solve
    stopped.  The textbook recurrences (pcg_kernel 0, 1) stop where the oracle's do and
    match it at the 1e-4 bar.  The default one-exchange form with residual replacement
    runs on until its true residual meets the tolerance (104 oracle PCG iterations
    against ~140) and is held to 1e-3."""
    prob = synth.make_problem(40, 5, ("poisson", 60.0), "uniform", seed=4)
    prob = synth.round_to_f32(prob)
    p = _problem(B, prob)
    cost, r, J = p.evaluate(residuals=True, jacobian=True)
    ref = O.residuals(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels)
    assert np.linalg.norm(r.double().cpu().numpy() - ref) <= 1e-5 * np.linalg.norm(ref)
    refs = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels,
                      O.LMOptions(max_lm_iters=5))
    for k, bar in ((0, 1e-4), (1, 1e-4), (2, 1e-3)):
        p.set_params(prob.cams_init, prob.pts_init)
        res = p.solve(max_lm_iters=5, pcg_kernel=k)
        assert res.status == 0 and res.lm_iters == 5
        assert abs(res.final_cost - refs.final_cost) <= bar * refs.final_cost, (k, res.final_cost, refs.final_cost)


def test_problems_bound_side_by_side_keep_working(B):
    """Several problems bound at once, larger first: each keeps its own launch shape
    (the persistent kernel's shared-memory limit is per function and must only grow)."""
    # 60,000 points = 235 tiles: more tiles than SMs, so its CTAs hold several tiles
    big = synth.round_to_f32(synth.make_problem(40, 60000, ("poisson", 4.0), "nearest", seed=61))
    small = synth.round_to_f32(synth.make_config("tiny", seed=62))
    opts = dict(max_lm_iters=3, max_pcg_iters=30)
    pb = _problem(B, big)
    ps = _problem(B, small)      # bound after the big one
    rb = pb.solve(**opts)
    rs = ps.solve(**opts)
    for prob, r in ((big, rb), (small, rs)):
        ref = O.ba_solve(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels, O.LMOptions(**opts))
        assert r.status == 0
        assert abs(r.final_cost - ref.final_cost) <= 1e-4 * ref.final_cost
