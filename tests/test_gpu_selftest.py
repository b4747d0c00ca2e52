"""Failure detection without a GPU fault: the bounded grid wait gives up and the
context stays usable (the wait simply runs out; nothing faults or traps)."""
import time

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


@pytest.mark.parametrize("grid", [1, 8, 64])
def test_grid_wait_gives_up_and_the_context_survives(B, grid):
    t0 = time.perf_counter()
    gave_up, err = B.selftest_wait_timeout(grid=grid, timeout_ms=50)
    dt = time.perf_counter() - t0
    assert gave_up == grid and err == 1
    assert 0.05 <= dt < 2.0, dt
    # the same process solves a problem afterwards
    prob = synth.round_to_f32(synth.make_config("tiny", seed=3))
    p = B.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels)
    p.set_params(prob.cams_init, prob.pts_init)
    res = p.solve(max_lm_iters=3)
    assert res.status == 0 and res.final_cost < res.initial_cost


def test_selftest_rejects_bad_arguments(B):
    with pytest.raises(B.BAError):
        B.selftest_wait_timeout(grid=0)
    with pytest.raises(B.BAError):
        B.selftest_wait_timeout(grid=1, timeout_ms=5000)
