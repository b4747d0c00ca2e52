"""Failure paths of a real solve, made on the host and ended by bounded waits: nothing
faults, traps or hangs the GPU.

* Non-finite parameters reach BA_ERR_NUMERIC through the device status word (the first
  linearisation finds a non-finite cost and stops the LM loop).
* A grid-wide wait limit of 0 ms (ba_options.wait_timeout_ms) makes the persistent PCG
  kernel give up at its first barrier: the solve reports BA_ERR_TIMEOUT, every CTA has
  left the kernel, and the next solve with the default limit succeeds on the same
  problem and context.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("where", ["point", "focal", "rotation"])
@pytest.mark.parametrize("pcg_kernel", [0, 1])
def test_non_finite_parameters_report_numeric(B, where, pcg_kernel):
    prob = synth.round_to_f32(synth.make_config("tiny", seed=71))
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels)
    cams, pts = prob.cams_init.copy(), prob.pts_init.copy()
    if where == "point":
        pts[17, 1] = np.nan
    elif where == "focal":
        cams[3, 6] = np.inf
    else:
        cams[5, 0] = np.nan
    p.set_params(cams, pts)
    res = p.solve(max_lm_iters=5, pcg_kernel=pcg_kernel)
    assert res.status == 4, res.status            # BA_ERR_NUMERIC from the device
    assert res.lm_iters == 0
    # the same problem solves once the parameters are finite again
    p.set_params(prob.cams_init, prob.pts_init)
    ok = p.solve(max_lm_iters=5, pcg_kernel=pcg_kernel)
    assert ok.status == 0 and ok.final_cost < ok.initial_cost
    p.close()


def test_grid_wait_limit_runs_out_in_a_real_solve_and_the_next_solve_succeeds(B):
    # 60,000 points = 235 tiles over one CTA per SM: the CTAs reach the first barrier at
    # different times, so a 0 ms limit runs out there
    prob = synth.round_to_f32(synth.make_problem(40, 60000, ("poisson", 4.0), "nearest", seed=73))
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels)
    p.set_params(prob.cams_init, prob.pts_init)
    ref = p.solve(max_lm_iters=3, max_pcg_iters=30)
    assert ref.status == 0
    p.set_params(prob.cams_init, prob.pts_init)
    out = p.solve(max_lm_iters=3, max_pcg_iters=30, wait_timeout_ms=0)
    assert out.status == 5, out.status            # BA_ERR_TIMEOUT
    p.set_params(prob.cams_init, prob.pts_init)
    again = p.solve(max_lm_iters=3, max_pcg_iters=30)
    assert again.status == 0
    assert abs(again.final_cost - ref.final_cost) <= 1e-6 * ref.final_cost
    p.close()


def test_wait_limit_option_is_validated(B):
    prob = synth.round_to_f32(synth.make_config("tiny", seed=75))
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels)
    p.set_params(prob.cams_init, prob.pts_init)
    for bad in (-1, 60001):
        with pytest.raises(B.BAError):
            p.solve(max_lm_iters=1, wait_timeout_ms=bad)
    p.close()
