"""The allocation-free cost entry point (ba_cost_noalloc) against the FP64 oracle.

ba_cost_noalloc serves callers that cannot allocate device memory (for example code
running while a stream is captured, or hosts whose device memory belongs to another
allocator): its scratch is a fixed array inside the library.  This file is collected
last, so a run that stops at the first failure has already run every other test.

Tolerance: the residuals are FP32 (inputs rounded to FP32 first, so only arithmetic
differs) and the sum is FP64; the cost then agrees with the oracle's FP64 cost to
1e-5 relative, the bar the evaluation parity tests use.
"""
import numpy as np
import pytest

from oracle import ba_oracle as O
from paper_2605_30583_gb300 import binding, synth


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2605_30583_gb300 import build
    build.build()
    L = binding.lib()
    big = L.ba_cost_noalloc(100000, 10, 10, None, None, None, None, None, 0.0, None, None)
    assert big == 1 and b"scratch capacity" in L.ba_last_error()
    huge = L.ba_cost_noalloc(10, 10, 1 << 40, None, None, None, None, None, 0.0, None, None)
    assert huge == 1 and b"scratch capacity" in L.ba_last_error()


def _device_inputs(prob, torch):
    dev = torch.device("cuda")
    return dict(cams=torch.tensor(prob.cams_init, dtype=torch.float32, device=dev),
                pts=torch.tensor(prob.pts_init, dtype=torch.float32, device=dev),
                ci=torch.tensor(prob.cam_idx.astype(np.int32), device=dev),   # same bits as uint32 here
                pi=torch.tensor(prob.pt_idx.astype(np.int32), device=dev),
                px=torch.tensor(prob.pixels, dtype=torch.float32, device=dev))


def _call(L, prob, t, eps, out, k, stream, n_obs=None):
    st = L.ba_cost_noalloc(prob.n_cams, prob.n_pts, prob.n_obs if n_obs is None else n_obs, t["cams"].data_ptr(),
                           t["pts"].data_ptr(), t["ci"].data_ptr(), t["pi"].data_ptr(), t["px"].data_ptr(),
                           float(eps), out.data_ptr() + 8 * k, stream)
    binding.check(st)


@pytest.mark.gpu
@pytest.mark.parametrize("shape", ["tiny", "multi_block"])
def test_noalloc_cost_matches_oracle_on_consecutive_calls(shape):
    """Three calls in a row (they share the scratch and its ticket) agree with the
    oracle's cost and with ba_evaluate; the multi-block case spans 15 blocks of 1,024
    observations and 300 cameras, so the last-block reduction and the ticket reset
    between calls are exercised; an eps_depth > 0 call follows the oracle's d_safe."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_30583_gb300 import build
    build.build()
    L = binding.lib()
    if shape == "tiny":
        prob = synth.round_to_f32(synth.make_config("tiny", seed=41))
    else:
        prob = synth.round_to_f32(synth.make_problem(300, 3000, ("poisson", 3.0), "uniform", seed=43))
        assert prob.n_obs > 14 * 1024
    p = binding.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels)
    p.set_params(prob.cams_init, prob.pts_init)
    evaluated, _, _ = p.evaluate()
    t = _device_inputs(prob, torch)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for k in range(3):
        _call(L, prob, t, 0.0, out, k, stream)
    eps = 0.125
    _call(L, prob, t, eps, out, 3, stream)
    torch.cuda.synchronize()
    c = out.cpu().numpy()
    ref = O.cost(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels)
    ref_eps = O.cost(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels, eps_depth=eps)
    assert abs(ref_eps - ref) > 1e-3 * ref   # the depth guard changes the cost
    for k in range(3):
        assert abs(c[k] - ref) <= 1e-5 * ref, (k, c[k], ref)
        assert abs(c[k] - evaluated) <= 1e-5 * ref
        assert abs(c[k] - c[0]) <= 1e-12 * ref
    assert abs(c[3] - ref_eps) <= 1e-5 * ref_eps, (c[3], ref_eps)
    p.close()


@pytest.mark.gpu
def test_noalloc_out_of_range_index_gives_nan_and_the_next_call_recovers():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_30583_gb300 import build
    build.build()
    L = binding.lib()
    prob = synth.round_to_f32(synth.make_problem(40, 2000, ("poisson", 3.0), "uniform", seed=47))
    t = _device_inputs(prob, torch)
    bad = dict(t)
    bad["ci"] = t["ci"].clone()
    bad["ci"][1234] = prob.n_cams            # one camera index out of range
    bad_pt = dict(t)
    bad_pt["pi"] = t["pi"].clone()
    bad_pt["pi"][5] = prob.n_pts + 7         # one point index out of range
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    _call(L, prob, bad, 0.0, out, 0, stream)
    _call(L, prob, bad_pt, 0.0, out, 1, stream)
    _call(L, prob, t, 0.0, out, 2, stream)
    torch.cuda.synchronize()
    c = out.cpu().numpy()
    assert np.isnan(c[0]) and np.isnan(c[1])
    ref = O.cost(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels)
    assert abs(c[2] - ref) <= 1e-5 * ref
