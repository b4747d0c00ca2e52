"""The allocation-free cost entry point (ba_cost_noalloc) against ba_evaluate.

ba_cost_noalloc serves callers that cannot allocate device memory (for example code
running while a stream is captured, or hosts whose device memory belongs to another
allocator): its scratch is a fixed array inside the library.  This file is collected
last, so a run that stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_30583_gb300 import binding, synth


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2605_30583_gb300 import build
    build.build()
    L = binding.lib()
    big = L.ba_cost_noalloc(100000, 10, 10, None, None, None, None, None, 0.0, None, None)
    assert big == 1 and b"scratch capacity" in L.ba_last_error()
    huge = L.ba_cost_noalloc(10, 10, 1 << 40, None, None, None, None, None, 0.0, None, None)
    assert huge == 1 and b"scratch capacity" in L.ba_last_error()


@pytest.mark.gpu
def test_noalloc_cost_matches_evaluate_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_30583_gb300 import build
    build.build()
    L = binding.lib()
    prob = synth.round_to_f32(synth.make_config("tiny", seed=41))
    p = binding.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels)
    p.set_params(prob.cams_init, prob.pts_init)
    ref, _, _ = p.evaluate()
    dev = torch.device("cuda")
    cams = torch.tensor(prob.cams_init, dtype=torch.float32, device=dev)
    pts = torch.tensor(prob.pts_init, dtype=torch.float32, device=dev)
    ci = torch.tensor(prob.cam_idx.astype(np.int32), device=dev)   # same bits as uint32 here
    pi = torch.tensor(prob.pt_idx.astype(np.int32), device=dev)
    px = torch.tensor(prob.pixels, dtype=torch.float32, device=dev)
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for k in range(2):   # two calls in a row share the scratch
        st = L.ba_cost_noalloc(prob.n_cams, prob.n_pts, prob.n_obs, cams.data_ptr(), pts.data_ptr(), ci.data_ptr(),
                               pi.data_ptr(), px.data_ptr(), 0.0, out.data_ptr() + 8 * k, stream)
        binding.check(st)
    torch.cuda.synchronize()
    c = out.cpu().numpy()
    # same FP32 residual arithmetic, FP64 sums in a different order
    assert abs(c[0] - ref) <= 1e-5 * ref, (c[0], ref)
    assert abs(c[1] - ref) <= 1e-5 * ref, (c[1], ref)
    assert abs(c[0] - c[1]) <= 1e-12 * ref
