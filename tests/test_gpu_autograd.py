"""The differentiable reprojection cost (torch.autograd.Function over ba_cost_forward /
ba_cost_backward) against the oracle and finite differences."""
import numpy as np
import pytest

from oracle import ba_oracle as O
from paper_2605_30583_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2605_30583_gb300 import autograd, binding, build
    build.build()
    binding.lib()
    return torch, binding, autograd


def _setup(env, prob, precision, dtype):
    torch, binding, autograd = env
    p = binding.Problem(prob.n_cams, prob.n_pts, prob.cam_idx, prob.pt_idx, prob.pixels, precision=precision)
    p.set_params(prob.cams_init, prob.pts_init)
    cams = torch.tensor(prob.cams_init, dtype=dtype, device="cuda", requires_grad=True)
    pts = torch.tensor(prob.pts_init, dtype=dtype, device="cuda", requires_grad=True)
    return p, cams, pts


@pytest.mark.parametrize("precision,dtype_name,tol", [("mixed", "float32", 1e-4), ("fp64", "float64", 1e-10)])
def test_cost_and_gradient_match_oracle(env, precision, dtype_name, tol):
    torch, binding, autograd = env
    dtype = getattr(torch, dtype_name)
    prob = synth.make_config("tiny", seed=51)
    if precision == "mixed":
        prob = synth.round_to_f32(prob)
    p, cams, pts = _setup(env, prob, precision, dtype)
    F = autograd.reprojection_cost(p, cams, pts)
    F.backward()
    lin = O.linearize(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels)
    assert abs(F.item() - lin.F) <= (1e-5 if precision == "mixed" else 1e-11) * lin.F
    g_ref = lin.g
    g = np.concatenate([cams.grad.double().cpu().numpy().ravel(), pts.grad.double().cpu().numpy().ravel()])
    assert np.linalg.norm(g - g_ref) <= tol * np.linalg.norm(g_ref), np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    # the problem's own parameters are untouched
    c, q = p.get_params()
    np.testing.assert_allclose(c, prob.cams_init, rtol=1e-6 if precision == "mixed" else 0)


def test_fp64_gradient_matches_central_differences(env):
    """Central differences of F (h = 1e-6, FP64) on random coordinates."""
    torch, binding, autograd = env
    prob = synth.make_problem(6, 60, ("poisson", 2.0), "uniform", seed=52)
    p, cams, pts = _setup(env, prob, "fp64", torch.float64)
    F = autograd.reprojection_cost(p, cams, pts)
    gc, gp = torch.autograd.grad(F, (cams, pts))
    rng = np.random.default_rng(0)
    h = 1e-6
    with torch.no_grad():
        for _ in range(12):
            if rng.random() < 0.5:
                t, g, idx = cams, gc, (int(rng.integers(prob.n_cams)), int(rng.integers(9)))
            else:
                t, g, idx = pts, gp, (int(rng.integers(prob.n_pts)), int(rng.integers(3)))
            old = t[idx].item()
            t[idx] = old + h
            Fp = autograd.reprojection_cost(p, cams, pts).item()
            t[idx] = old - h
            Fm = autograd.reprojection_cost(p, cams, pts).item()
            t[idx] = old
            fd = (Fp - Fm) / (2 * h)
            an = g[idx].item()
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-6 * abs(F.item()) * h, (idx, fd, an)


def test_gradcheck_small_problem(env):
    torch, binding, autograd = env
    prob = synth.make_problem(3, 12, ("poisson", 1.0), "uniform", seed=53)
    p, cams, pts = _setup(env, prob, "fp64", torch.float64)
    f = lambda c, q: autograd.reprojection_cost(p, c, q)
    assert torch.autograd.gradcheck(f, (cams, pts), eps=1e-6, atol=1e-4, rtol=1e-6)


def test_grad_out_scaling_and_autograd_config_size(env):
    """Config-4-sized problem (200 cameras, 50,000 points, ~300k observations)."""
    torch, binding, autograd = env
    prob = synth.round_to_f32(synth.make_config("autograd"))
    p, cams, pts = _setup(env, prob, "mixed", torch.float32)
    F = autograd.reprojection_cost(p, cams, pts)
    (2.5 * F).backward()
    ref = O.cost(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels)
    assert abs(F.item() - ref) <= 1e-5 * ref
    g1 = torch.cat([cams.grad.ravel(), pts.grad.ravel()]).double()
    cams.grad = None
    pts.grad = None
    autograd.reprojection_cost(p, cams, pts).backward()
    g0 = torch.cat([cams.grad.ravel(), pts.grad.ravel()]).double()
    assert torch.allclose(g1, 2.5 * g0, rtol=1e-5, atol=1e-3)
    # sampled points: the adjoint's point rows against the oracle, one point at a time
    rng = np.random.default_rng(1)
    for u in rng.integers(0, prob.n_pts, 5):
        sel = np.nonzero(prob.pt_idx == u)[0]
        r, Jc, Jp = O.jacobian_blocks(prob.cams_init, prob.pts_init, prob.cam_idx[sel], prob.pt_idx[sel],
                                      prob.pixels[sel])
        g_ref = np.einsum("oki,ok->i", Jp, r)
        g_gpu = pts.grad[int(u)].double().cpu().numpy()
        assert np.linalg.norm(g_gpu - g_ref) <= 1e-3 * np.linalg.norm(g_ref) + 1e-3
