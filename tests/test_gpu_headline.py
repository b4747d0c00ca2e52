"""The headline medium workload (1,000 cameras, 200,000 points, 1,199,169 observations)
solved with the default solver against the FP64 oracle's stored run.

The stored run (tests/golden/oracle_lm_medium.json, written by make_golden.py from the
oracle alone) takes 20 LM iterations of at most 50 PCGNR iterations each, initial trust
region 100 and CG tolerance 1e-3 (Sec. VI), on the same FP32-rounded inputs.  The GPU
runs the same budget with the default options (persistent PCG kernel, conditional-loop
graph mode): its final cost must be the oracle's within 1e-4 relative (the parity bar
for final costs), it must take the same number of LM iterations, and every accepted
step must lower the cost.
"""
import json
import os

import pytest

from paper_2605_30583_gb300 import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_lm_medium.json")


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
def medium():
    return synth.round_to_f32(synth.make_config("medium"))


@pytest.mark.parametrize("pcg_kernel", [0, 1])
def test_medium_default_solve_matches_oracle(B, medium, pcg_kernel):
    ref = json.load(open(GOLDEN))["fp32_inputs"]
    assert ref["n_obs"] == medium.n_obs and ref["options"] == {"max_lm_iters": 20, "max_pcg_iters": 50}
    p = B.Problem(medium.n_cams, medium.n_pts, medium.cam_idx, medium.pt_idx, medium.pixels)
    p.set_params(medium.cams_init, medium.pts_init)
    opts = B.default_options(pcg_kernel=pcg_kernel)     # 20 LM x <= 50 PCG, TR0 = 100, tol 1e-3
    assert opts.max_lm_iters == 20 and opts.max_pcg_iters == 50 and opts.use_graph == 1
    res = p.solve(opts)
    assert res.status == 0
    assert res.lm_iters == ref["lm_iters"]
    assert abs(res.initial_cost - ref["initial_cost"]) <= 1e-5 * ref["initial_cost"]
    assert abs(res.final_cost - ref["final_cost"]) <= 1e-4 * ref["final_cost"], (res.final_cost, ref["final_cost"])
    for h in res.history:
        if h["accepted"]:
            assert h["cost_new"] < h["cost"]
    # the first step, far above the noise floor, follows the oracle's closely
    h0, o0 = res.history[0], ref["history"][0]
    assert h0["accepted"] and abs(h0["pcg_iters"] - o0["pcg_iters"]) <= 2
    assert abs(h0["cost_new"] - o0["cost_new"]) <= 1e-4 * o0["cost_new"]
    p.close()
