"""The large workload (13,000 cameras, 4.5M points, ~29M observations, 2+Geometric(4.4)
views, nearest-camera visibility) at full size, checked where the oracle can follow:

* residuals of a random sample of observations against the oracle's, one by one;
* the damped normal operator on sampled points and cameras against the oracle's blocks
  restricted to those nodes' observations;
* the full LM solve against the plain all-FP64 GPU form of the same algorithm, which
  stands in for the oracle at this size (it matches the oracle to 1e-8 on the tiny
  workload and to ~1e-14 on the medium one; the oracle itself would need hours here):
  the workload's own 20-iteration budget at the first step, and a 500-iteration solve
  whose end point and continuation are held to the 1e-4 bar.
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


@pytest.fixture(scope="module")
def large():
    return synth.round_to_f32(synth.make_config("large"))


@pytest.fixture(scope="module")
def mixed(B, large):
    p = B.Problem(large.n_cams, large.n_pts, large.cam_idx, large.pt_idx, large.pixels)
    p.set_params(large.cams_init, large.pts_init)
    return p


def test_large_sampled_residuals(mixed, large):
    assert large.n_obs > 28_000_000
    _, r, _ = mixed.evaluate(residuals=True)
    rng = np.random.default_rng(0)
    S = rng.choice(large.n_obs, 20000, replace=False)
    rs = r.cpu().numpy()[S].astype(np.float64)
    ref = O.residuals(large.cams_init, large.pts_init, large.cam_idx[S], large.pt_idx[S], large.pixels[S])
    err = np.abs(rs - ref)
    assert np.all(err <= 2e-4 + 1e-5 * np.abs(ref)), err.max()
    assert np.linalg.norm(rs - ref) <= 1e-5 * np.linalg.norm(ref)


def _node_blocks(large, obs):
    _, Jc, Jp = O.jacobian_blocks(large.cams_init, large.pts_init, large.cam_idx[obs], large.pt_idx[obs],
                                  large.pixels[obs])
    return Jc, Jp


def test_large_sampled_normal_operator(B, mixed, large):
    import torch
    mixed.evaluate()
    n = 9 * large.n_cams + 3 * large.n_pts
    rng = np.random.default_rng(1)
    v = rng.standard_normal(n)
    mu = 0.01
    out, _ = mixed.apply_normal(mu, torch.from_numpy(v.astype(np.float32)))
    q = out.cpu().numpy().astype(np.float64)
    vf = v.astype(np.float32).astype(np.float64)
    vc = vf[: 9 * large.n_cams].reshape(-1, 9)
    vp = vf[9 * large.n_cams:].reshape(-1, 3)
    clamp = lambda d: np.clip(d, 1e-6, 1e32)
    got, ref, scale = [], [], []
    # sampled points: all their observations
    order = np.argsort(large.pt_idx, kind="stable")
    starts = np.searchsorted(large.pt_idx[order], np.arange(large.n_pts + 1))
    for p in rng.choice(large.n_pts, 300, replace=False):
        obs = order[starts[p]:starts[p + 1]]
        Jc, Jp = _node_blocks(large, obs)
        t = np.einsum("oij,oj->oi", Jc, vc[large.cam_idx[obs]]) + np.einsum("oij,j->oi", Jp, vp[p])
        D = clamp(np.einsum("oij,oij->j", Jp, Jp))
        ref.append(np.einsum("oij,oi->j", Jp, t) + mu * D * vp[p])
        ta = np.einsum("oij,oj->oi", np.abs(Jc), np.abs(vc[large.cam_idx[obs]])) + \
            np.einsum("oij,j->oi", np.abs(Jp), np.abs(vp[p]))
        scale.append(np.einsum("oij,oi->j", np.abs(Jp), ta) + mu * D * np.abs(vp[p]))
        got.append(q[9 * large.n_cams + 3 * p: 9 * large.n_cams + 3 * p + 3])
    # sampled cameras with modest observation counts
    counts = np.bincount(large.cam_idx, minlength=large.n_cams)
    cand = np.flatnonzero((counts > 0) & (counts < 4000))
    for c in rng.choice(cand, 4, replace=False):
        obs = np.flatnonzero(large.cam_idx == c)
        Jc, Jp = _node_blocks(large, obs)
        t = np.einsum("oij,j->oi", Jc, vc[c]) + np.einsum("oij,oj->oi", Jp, vp[large.pt_idx[obs]])
        D = clamp(np.einsum("oij,oij->j", Jc, Jc))
        ref.append(np.einsum("oij,oi->j", Jc, t) + mu * D * vc[c])
        ta = np.einsum("oij,j->oi", np.abs(Jc), np.abs(vc[c])) + \
            np.einsum("oij,oj->oi", np.abs(Jp), np.abs(vp[large.pt_idx[obs]]))
        scale.append(np.einsum("oij,oi->j", np.abs(Jc), ta) + mu * D * np.abs(vc[c]))
        got.append(q[9 * c: 9 * c + 9])
    got = np.concatenate(got)
    ref = np.concatenate(ref)
    scale = np.concatenate(scale)
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref), np.linalg.norm(got - ref) / np.linalg.norm(ref)
    # per entry, against the sum of the magnitudes of its terms (see test_gpu_parity)
    err = np.abs(got - ref) / scale
    assert err.max() <= 1e-4, err.max()


def test_large_solve_against_fp64_form(B, mixed, large):
    """The workload's own budget (20 LM x <= 50 PCG) on both forms.

    At this size 20 LM iterations do not converge: both forms end a few per cent above
    the noise floor and are still descending.  Their trajectories separate after the
    first step, because PCG stops at its 50-iteration cap and a truncated Krylov iterate
    depends on rounding: FP32 and FP64 steps differ by ~1e-4, which changes the next rho
    and mu.  So the first LM step is compared at the parity bar, and the end of the solve
    by where each form stands (statuses, monotone costs, both near the noise floor, and
    within 1 % of each other)."""
    opts = dict(max_lm_iters=20, max_pcg_iters=50)
    mixed.set_params(large.cams_init, large.pts_init)
    a = mixed.solve(**opts)
    q = B.Problem(large.n_cams, large.n_pts, large.cam_idx, large.pt_idx, large.pixels, precision="fp64")
    q.set_params(large.cams_init, large.pts_init)
    b = q.solve(**opts)
    q.close()
    assert a.status == 0 and b.status == 0 and a.lm_iters == 20 and b.lm_iters == 20
    assert abs(a.initial_cost - b.initial_cost) <= 1e-6 * b.initial_cost
    # first step: same PCG iteration count, same accepted cost
    ha, hb = a.history[0], b.history[0]
    assert ha["accepted"] and hb["accepted"] and ha["pcg_iters"] == hb["pcg_iters"]
    assert abs(ha["cost_new"] - hb["cost_new"]) <= 1e-4 * hb["cost_new"]
    for r in (a, b):
        costs = [h["cost"] for h in r.history] + [r.final_cost]
        assert all(x >= y for x, y in zip(costs, costs[1:]))
    floor = 0.5 * (2 * large.n_obs - 9 * large.n_cams - 3 * large.n_pts + 7)   # chi^2 level at the optimum
    assert floor < a.final_cost < 1.1 * floor and floor < b.final_cost < 1.1 * floor, (a.final_cost, b.final_cost)


def test_large_long_solve_tracks_the_fp64_form_at_the_bar(B, mixed, large):
    """The mixed form over a long budget, checked by the plain FP64 form.

    This workload does not converge in any budget a test can afford: its points are seen
    by their 2-6 nearest cameras of a dense ring, along nearly parallel rays (parallax
    ~1e-3 rad), so their depths are barely constrained and LM with block-Jacobi PCG crawls
    along those directions (the FP64 form crawls at the same rate).  What is checked:

    * 500 LM iterations (<= 500 PCG each) lower the cost monotonically, status 0;
    * the mixed form's own cost at its end point is the true cost: the FP64 form
      evaluates the same parameters within 1e-9 (double-float residuals; with FP32
      residuals LM exploits their ~1e-4 px errors along the flat directions and the two
      evaluations part by up to ~3e-4);
    * from that end point, 20 more LM iterations of each form (fresh solves, same
      options) reach costs within the 1e-4 bar of each other: the mixed form keeps
      tracking FP64 in the hard tail, not only at the first step;
    * 2F / dof, dof = m - n + 7 (the chi^2 statistic of the maximum-likelihood fit, n
      minus the 7-dimensional similarity gauge), is within 1 % of 1.  (It sits ~0.2 %
      below: for nearly degenerate two-view points the linear count of degrees of
      freedom overstates what the fit leaves in the residuals, so the +-4 sigma band of
      the linear model, 0.04 %, does not apply.)"""
    mixed.set_params(large.cams_init, large.pts_init)
    a = mixed.solve(max_lm_iters=500, max_pcg_iters=500)
    assert a.status == 0 and a.lm_iters == 500
    costs = [h["cost"] for h in a.history] + [a.final_cost]
    assert all(x >= y for x, y in zip(costs, costs[1:]))
    c, q = mixed.get_params()
    f = B.Problem(large.n_cams, large.n_pts, large.cam_idx, large.pt_idx, large.pixels, precision="fp64")
    f.set_params(c, q)
    b = f.solve(max_lm_iters=20, max_pcg_iters=500)
    f.close()
    assert b.status == 0
    assert abs(b.initial_cost - a.final_cost) <= 1e-9 * a.final_cost, (b.initial_cost, a.final_cost)
    mixed.set_params(c, q)
    a2 = mixed.solve(max_lm_iters=20, max_pcg_iters=500)
    assert a2.status == 0
    assert abs(a2.initial_cost - b.initial_cost) <= 1e-9 * b.initial_cost
    assert abs(a2.final_cost - b.final_cost) <= 1e-4 * b.final_cost, (a2.final_cost, b.final_cost)
    dof = 2 * large.n_obs - 9 * large.n_cams - 3 * large.n_pts + 7
    for r in (a, a2, b):
        assert abs(2.0 * r.final_cost / dof - 1.0) <= 0.01, r.final_cost
