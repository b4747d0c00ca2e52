"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test is chosen so that a plausible mistake in the oracle (a dropped term, a
wrong sign or index, a transposed operand, a wrong damping or gain-ratio formula)
fails at least one of them.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.spatial.transform import Rotation

from oracle import ba_oracle as O
from paper_2605_30583_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_problem(seed=7, n_cams=3, n_pts=20, noise=1.0):
    return synth.make_problem(n_cams, n_pts, ("poisson", 1.0), "uniform", seed=seed, noise_px=noise)


# ---------------------------------------------------------------- projection -----


def test_hand_projection_cases():
    """Hand-worked pixels of the Sec. VI-A residual (tests/golden/hand_projection.json)."""
    data = json.load(open(os.path.join(GOLDEN, "hand_projection.json")))
    for case in data["cases"]:
        cam = np.array(case["cam"], dtype=np.float64)
        X = np.array(case["point"], dtype=np.float64)
        RX = O.rotate(list(cam[:3]), list(X))
        P = np.array(RX) + cam[3:6]
        np.testing.assert_allclose(P, case["P"], atol=1e-14)
        u = O.project(list(cam), list(X))
        np.testing.assert_allclose(u, case["pixel"], rtol=0, atol=1e-12)
        # residual against the predicted pixel is exactly zero
        r = O.residuals(cam[None], X[None], [0], [0], np.array([case["pixel"]]))
        assert np.all(np.abs(r) <= 1e-12)


def test_first_hand_case_is_exact():
    """With w = 0 every step is exact in binary, so the pixel is bit-exact."""
    u = O.project([0.0, 0.0, 0.0, 0.0, 0.0, -4.0, 500.0, 0.1, 0.01], [1.0, 2.0, 0.0])
    assert u == (129.0283203125, 258.056640625)


def test_rotation_matches_scipy_rotvec():
    rng = np.random.default_rng(0)
    w = rng.standard_normal((500, 3))
    w[:100] *= 1e-6                                   # small-angle series branch
    w[100:200] *= np.pi / np.linalg.norm(w[100:200], axis=1, keepdims=True)  # |w| = pi
    X = rng.standard_normal((500, 3))
    ours = np.stack(O.rotate(list(w.T), list(X.T)), axis=1)
    ref = Rotation.from_rotvec(w).apply(X)
    np.testing.assert_allclose(ours, ref, rtol=0, atol=1e-13)


def test_eps_depth_shifts_depth_away_from_zero():
    """d_safe = d + eps * sign_no_zero(d): for d < 0 the shift is -eps (Sec. VI-A)."""
    cam = [0, 0, 0, 0, 0, -4, 500, 0, 0]
    u0 = O.project(cam, [1.0, 2.0, 0.0], eps_depth=0.0)
    u1 = O.project(cam, [1.0, 2.0, 0.0], eps_depth=1.0)     # d_safe = -5
    np.testing.assert_allclose(u1, (100.0, 200.0), atol=1e-12)
    assert u0 != u1
    # sign_no_zero(0) = +1
    u2 = O.project([0, 0, 0, 0, 0, 0, 1, 0, 0], [1.0, 2.0, 0.0], eps_depth=0.5)
    np.testing.assert_allclose(u2, (-2.0, -4.0), atol=1e-12)


# ---------------------------------------------------------------- Jacobian -------


def _fd_jacobian(cams, pts, ci, pi, px, h=1e-6):
    n = ci.shape[0]
    Jc = np.zeros((n, 2, 9))
    Jp = np.zeros((n, 2, 3))
    for k in range(9):
        cp, cm = cams.copy(), cams.copy()
        cp[:, k] += h
        cm[:, k] -= h
        Jc[:, :, k] = (O.residuals(cp, pts, ci, pi, px) - O.residuals(cm, pts, ci, pi, px)) / (2 * h)
    for k in range(3):
        pp, pm = pts.copy(), pts.copy()
        pp[:, k] += h
        pm[:, k] -= h
        Jp[:, :, k] = (O.residuals(cams, pp, ci, pi, px) - O.residuals(cams, pm, ci, pi, px)) / (2 * h)
    return Jc, Jp


def test_dual_jacobian_matches_central_differences():
    p = synth.make_config("tiny")
    sel = np.arange(0, p.n_obs, 7)
    ci, pi, px = p.cam_idx[sel], p.pt_idx[sel], p.pixels[sel]
    # one observation per (camera, point) row so each FD column touches one observation
    cams = p.cams_init[ci]
    pts = p.pts_init[pi]
    idx = np.arange(sel.shape[0])
    r, Jc, Jp = O.jacobian_blocks(cams, pts, idx, idx, px)
    fJc, fJp = _fd_jacobian(cams, pts, idx, idx, px)
    for A, B in ((Jc, fJc), (Jp, fJp)):
        err = np.linalg.norm(A - B, axis=(1, 2)) / np.linalg.norm(B, axis=(1, 2))
        assert err.max() < 1e-6, err.max()


def test_dual_jacobian_small_angle_and_pi():
    rng = np.random.default_rng(3)
    cams = np.tile(np.array([0, 0, 0, 0.1, -0.2, -5.0, 700.0, 0.01, -0.005]), (6, 1))
    cams[0, :3] = 0.0
    cams[1, :3] = [3e-5, -2e-5, 1e-5]          # series branch
    cams[2, :3] = [2e-4, 1e-4, -1e-4]          # just above the branch threshold
    cams[3, :3] = [0, 0, np.pi]                # 180 degrees
    cams[4, :3] = rng.standard_normal(3)
    cams[5, :3] = [1.0, 2.0, 0.5]
    pts = rng.standard_normal((6, 3)) * 0.5
    idx = np.arange(6)
    px = np.zeros((6, 2))
    r, Jc, Jp = O.jacobian_blocks(cams, pts, idx, idx, px)
    fJc, fJp = _fd_jacobian(cams, pts, idx, idx, px)
    np.testing.assert_allclose(Jc, fJc, rtol=1e-6, atol=1e-5)
    np.testing.assert_allclose(Jp, fJp, rtol=1e-6, atol=1e-5)


def test_sparse_assembly_matches_dense_fd_jacobian():
    """Column layout [9 per camera | 3 per point] and row pairs (2o, 2o+1)."""
    p = _small_problem()
    x0 = O.pack(p.cams_init, p.pts_init)
    lin = O.linearize(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels)

    def rfun(x):
        c, q = O.unpack(x, p.n_cams)
        return O.residuals(c, q, p.cam_idx, p.pt_idx, p.pixels).reshape(-1)

    h = 1e-6
    Jd = np.zeros((2 * p.n_obs, x0.shape[0]))
    for k in range(x0.shape[0]):
        e = np.zeros_like(x0)
        e[k] = h
        Jd[:, k] = (rfun(x0 + e) - rfun(x0 - e)) / (2 * h)
    J = lin.J.toarray()
    assert np.abs(J - Jd).max() <= 1e-5 * np.abs(Jd).max()
    np.testing.assert_allclose(lin.r, rfun(x0), rtol=0, atol=1e-12)
    np.testing.assert_allclose(lin.g, Jd.T @ lin.r, rtol=1e-6, atol=1e-6 * np.abs(Jd.T @ lin.r).max())
    JtJ = J.T @ J
    for c in range(p.n_cams):
        np.testing.assert_allclose(lin.Hc[c], JtJ[9 * c:9 * c + 9, 9 * c:9 * c + 9], rtol=1e-12, atol=1e-9)
    base = 9 * p.n_cams
    for q in range(p.n_pts):
        s = base + 3 * q
        np.testing.assert_allclose(lin.Hp[q], JtJ[s:s + 3, s:s + 3], rtol=1e-12, atol=1e-9)


# ---------------------------------------------------------------- PCG ------------


def test_pcgnr_matches_dense_cholesky_solve():
    p = _small_problem()
    lin = O.linearize(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels)
    mu = 0.01
    D = O.damping_diag(lin.J)
    J = lin.J.toarray()
    A = J.T @ J + mu * np.diag(D)
    h_dense = np.linalg.solve(A, -lin.g)
    Mc, Mp = O.block_jacobi(lin, D, mu)
    res = O.pcgnr(lin.J, D, mu, -lin.g, lambda v: O.apply_block_jacobi(Mc, Mp, v),
                  tol=1e-14, max_iters=10 * A.shape[0])
    assert np.linalg.norm(res.h - h_dense) <= 1e-9 * np.linalg.norm(h_dense)
    # the preconditioner blocks are the inverses of the dense diagonal blocks
    for c in range(p.n_cams):
        blk = A[9 * c:9 * c + 9, 9 * c:9 * c + 9]
        np.testing.assert_allclose(Mc[c] @ blk, np.eye(9), atol=1e-8)
    np.testing.assert_allclose(O.normal_matvec(lin, D, mu, h_dense), -lin.g, rtol=1e-8,
                               atol=1e-8 * np.abs(lin.g).max())


def test_damping_diag_is_clamped_column_norm():
    J = sp.csr_matrix(np.array([[1.0, 0.0, 2.0], [3.0, 0.0, 0.0]]))
    np.testing.assert_array_equal(O.damping_diag(J, 1e-6, 5.0), [5.0, 1e-6, 4.0])


def test_pcg_exact_preconditioner_converges_in_one_iteration():
    """A block-diagonal J^T J with the exact block inverse as preconditioner: one step."""
    rng = np.random.default_rng(1)
    B1, B2 = rng.standard_normal((4, 2)), rng.standard_normal((4, 3))
    J = sp.block_diag([sp.csr_matrix(B1), B2]).tocsr()
    D = np.ones(5)
    mu = 0.5
    A = (J.T @ J).toarray() + mu * np.eye(5)
    b = rng.standard_normal(5)
    Ainv = np.linalg.inv(A)
    res = O.pcgnr(J, D, mu, b, lambda v: Ainv @ v, tol=1e-12, max_iters=5)
    assert res.iters == 1
    np.testing.assert_allclose(res.h, Ainv @ b, rtol=1e-12)


def test_pcg_iteration_cap_and_tolerance():
    p = _small_problem()
    lin = O.linearize(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels)
    D = O.damping_diag(lin.J)
    Mc, Mp = O.block_jacobi(lin, D, 0.01)
    pre = lambda v: O.apply_block_jacobi(Mc, Mp, v)
    capped = O.pcgnr(lin.J, D, 0.01, -lin.g, pre, tol=1e-14, max_iters=3)
    assert capped.iters == 3
    tol = O.pcgnr(lin.J, D, 0.01, -lin.g, pre, tol=1e-3, max_iters=1000)
    assert tol.r_norm <= 1e-3 * tol.r0_norm
    assert tol.iters < 1000


# ---------------------------------------------------------------- LM -------------


def _linear_problem(seed=5):
    rng = np.random.default_rng(seed)
    A = sp.csr_matrix(rng.standard_normal((30, 6)))
    b = rng.standard_normal(30)

    class Lin:
        def __init__(self, x):
            self.r = A @ x - b
            self.F = 0.5 * float(self.r @ self.r)
            self.J = A
            self.g = A.T @ self.r

    def pre(lin, D, mu):
        M = np.linalg.inv((A.T @ A).toarray() + mu * np.diag(D))
        return lambda v: M @ v

    return A, b, Lin, (lambda x: 0.5 * float(np.sum((A @ x - b) ** 2))), pre


def test_lm_gain_ratio_is_one_on_linear_least_squares():
    """The quadratic model is exact for linear residuals, so rho = 1 and Madsen's rule
    gives mu <- mu * max(1/3, 1 - (2*1 - 1)^3) = mu / 3 on every accepted step."""
    A, b, Lin, cost, pre = _linear_problem()
    opts = O.LMOptions(max_lm_iters=4, pcg_rel_tol=1e-14, max_pcg_iters=50)
    res = O.lm_solve(np.zeros(6), Lin, cost, pre, opts)
    for k, h in enumerate(res.history):
        if h["model_decrease"] > 1e-9 * res.initial_cost:
            assert h["accepted"]
            assert abs(h["rho"] - 1.0) < 1e-8
    np.testing.assert_allclose([h["mu"] for h in res.history[:2]], [0.01, 0.01 / 3], rtol=1e-12)
    x_ls = np.linalg.lstsq(A.toarray(), b, rcond=None)[0]
    np.testing.assert_allclose(res.x, x_ls, rtol=1e-6, atol=1e-8)


def test_lm_rosenbrock_reaches_minimum():
    """Rosenbrock as least squares, r = (10 (x1 - x0^2), 1 - x0); minimum F = 0 at (1, 1)."""

    class Lin:
        def __init__(self, x):
            self.r = np.array([10 * (x[1] - x[0] ** 2), 1 - x[0]])
            self.F = 0.5 * float(self.r @ self.r)
            self.J = sp.csr_matrix(np.array([[-20 * x[0], 10.0], [-1.0, 0.0]]))
            self.g = self.J.T @ self.r

    def pre(lin, D, mu):
        M = np.linalg.inv((lin.J.T @ lin.J).toarray() + mu * np.diag(D))
        return lambda v: M @ v

    cost = lambda x: 0.5 * (100 * (x[1] - x[0] ** 2) ** 2 + (1 - x[0]) ** 2)
    res = O.lm_solve(np.array([-1.2, 1.0]), Lin, cost, pre,
                     O.LMOptions(max_lm_iters=200, pcg_rel_tol=1e-12, max_pcg_iters=10))
    np.testing.assert_allclose(res.x, [1.0, 1.0], atol=1e-6)
    assert res.final_cost < 1e-12


def test_lm_rejected_step_leaves_x_and_increases_mu():
    A, b, Lin, cost, pre = _linear_problem()
    # A cost function that always reports a higher cost forces every step to be rejected.
    res = O.lm_solve(np.zeros(6), Lin, lambda x: 1e30, pre, O.LMOptions(max_lm_iters=4))
    assert res.accepted == 0
    np.testing.assert_array_equal(res.x, np.zeros(6))
    mus = [h["mu"] for h in res.history]
    np.testing.assert_allclose(mus, [0.01, 0.02, 0.08, 0.64], rtol=1e-12)   # nu = 2, 4, 8


# ---------------------------------------------------------------- BA invariants --


def test_zero_residual_at_noise_free_ground_truth():
    """The generator's look-at projection and the oracle's Rodrigues projection agree."""
    p = synth.make_problem(16, 300, ("poisson", 3.0), "uniform", seed=11, noise_px=0.0)
    r = O.residuals(p.cams_gt, p.pts_gt, p.cam_idx, p.pt_idx, p.pixels)
    assert np.abs(r).max() < 1e-9
    res = O.ba_solve(p.cams_gt, p.pts_gt, p.cam_idx, p.pt_idx, p.pixels, O.LMOptions(max_lm_iters=3))
    assert res.final_cost <= res.initial_cost < 1e-15


def test_lm_monotone_cost_and_chi_square_level():
    """Accepted steps strictly decrease F; at the optimum 2F / sigma^2 follows a
    chi-square law with m - n + 7 degrees of freedom (7-DoF similarity gauge)."""
    p = synth.make_config("tiny")
    res = O.ba_solve(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels)
    costs = [h["cost"] for h in res.history] + [res.final_cost]
    for a, b_ in zip(costs[:-1], costs[1:]):
        assert b_ <= a
    for h in res.history:
        if h["accepted"]:
            assert h["cost_new"] < h["cost"]
    m = 2 * p.n_obs
    n = 9 * p.n_cams + 3 * p.n_pts
    dof = m - n + 7
    assert abs(2 * res.final_cost - dof) < 4 * np.sqrt(2 * dof)
    assert res.final_cost < 0.01 * res.initial_cost


def test_gradient_vanishes_at_solution():
    p = synth.make_config("tiny")
    res = O.ba_solve(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels)
    c, q = O.unpack(res.x, p.n_cams)
    g0 = O.linearize(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels).g
    g1 = O.linearize(c, q, p.cam_idx, p.pt_idx, p.pixels).g
    assert np.linalg.norm(g1) < 1e-6 * np.linalg.norm(g0)


# ---------------------------------------------------------------- retraction ------
# The paper's Pose3 update (Sec. VI-A) as the oracle's rotation_update="retraction":
# rotations step as R <- Exp(d) R(w), the Jacobian taken w.r.t. d at d = 0.


def _skew(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def test_retraction_jacobian_matches_central_differences():
    p = _small_problem(seed=41)
    S = np.arange(min(40, p.n_obs))
    cams, pts = p.cams_init, p.pts_init
    _, Jc, Jp = O.jacobian_blocks(cams, pts, p.cam_idx[S], p.pt_idx[S], p.pixels[S], retraction=True)
    _, Jc_add, Jp_add = O.jacobian_blocks(cams, pts, p.cam_idx[S], p.pt_idx[S], p.pixels[S])
    eps = 1e-6
    for i in range(3):
        e = np.zeros((cams.shape[0], 3))
        e[:, i] = eps
        cp, cm = cams.copy(), cams.copy()
        # perturbed rotations Exp(+-eps e_i) R(w), composed by scipy (independent of the oracle)
        cp[:, 0:3] = (Rotation.from_rotvec(e) * Rotation.from_rotvec(cams[:, 0:3])).as_rotvec()
        cm[:, 0:3] = (Rotation.from_rotvec(-e) * Rotation.from_rotvec(cams[:, 0:3])).as_rotvec()
        rp = O.residuals(cp, pts, p.cam_idx[S], p.pt_idx[S], p.pixels[S])
        rm = O.residuals(cm, pts, p.cam_idx[S], p.pt_idx[S], p.pixels[S])
        fd = (rp - rm) / (2 * eps)
        assert np.linalg.norm(fd - Jc[:, :, i]) <= 1e-6 * np.linalg.norm(fd)
    # every other column is the additive Jacobian's
    assert np.allclose(Jc[:, :, 3:], Jc_add[:, :, 3:], rtol=1e-13, atol=0)
    assert np.allclose(Jp, Jp_add, rtol=1e-13, atol=0)


def test_retraction_jacobian_maps_to_additive_through_left_jacobian():
    """d r/d w = (d r/d d) J_l(w), with the closed-form left Jacobian of SO(3)
    J_l(w) = I + (1 - cos t)/t^2 [w]x + (t - sin t)/t^3 [w]x^2."""
    p = _small_problem(seed=42)
    S = np.arange(min(40, p.n_obs))
    _, Jd, _ = O.jacobian_blocks(p.cams_init, p.pts_init, p.cam_idx[S], p.pt_idx[S], p.pixels[S], retraction=True)
    _, Jw, _ = O.jacobian_blocks(p.cams_init, p.pts_init, p.cam_idx[S], p.pt_idx[S], p.pixels[S])
    for o in range(len(S)):
        w = p.cams_init[p.cam_idx[S[o]], 0:3]
        t = np.linalg.norm(w)
        K = _skew(w)
        Jl = np.eye(3) + (1 - np.cos(t)) / t**2 * K + (t - np.sin(t)) / t**3 * (K @ K)
        assert np.allclose(Jd[o][:, 0:3] @ Jl, Jw[o][:, 0:3], rtol=1e-9, atol=1e-9 * np.abs(Jw[o]).max())


def test_retraction_step_composes_on_the_left():
    rng = np.random.default_rng(43)
    cams = rng.standard_normal((6, 9))
    h = 0.1 * rng.standard_normal((6, 9))
    out = O.retract_cams(cams, h)
    assert np.allclose(out[:, 3:], cams[:, 3:] + h[:, 3:], rtol=0, atol=1e-15)
    assert np.allclose(O.retract_cams(cams, np.zeros_like(h))[:, 0:3],
                       Rotation.from_rotvec(cams[:, 0:3]).as_rotvec(), atol=1e-14)
    # R(w') X == R(h) (R(w) X), checked with the oracle's own Rodrigues rotation
    X = list(rng.standard_normal((3, 6)))
    lhs = O.rotate(list(out[:, 0:3].T), X)
    rhs = O.rotate(list(h[:, 0:3].T), list(O.rotate(list(cams[:, 0:3].T), X)))
    assert np.allclose(np.array(lhs), np.array(rhs), atol=1e-12)


def test_lm_retraction_reaches_the_additive_optimum():
    """The minimum of F does not depend on how rotations are parametrised: run to
    convergence, both updates end at the same cost and a vanishing gradient."""
    p = _small_problem(seed=44, n_cams=4, n_pts=40)
    out = {}
    for ru in ("additive", "retraction"):
        opts = O.LMOptions(max_lm_iters=60, max_pcg_iters=400, pcg_rel_tol=1e-10, rotation_update=ru)
        out[ru] = O.ba_solve(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels, opts)
    a, b = out["additive"].final_cost, out["retraction"].final_cost
    assert abs(a - b) <= 1e-9 * a
    for r in out.values():
        c, q = O.unpack(r.x, p.n_cams)
        lin = O.linearize(c, q, p.cam_idx, p.pt_idx, p.pixels)
        lin0 = O.linearize(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels)
        assert np.linalg.norm(lin.g) <= 1e-6 * np.linalg.norm(lin0.g)


# ---------------------------------------------------------------- robust loss -----


def _with_outliers(p, frac=0.05, size=40.0, seed=0):
    import dataclasses
    rng = np.random.default_rng(seed)
    px = p.pixels.copy()
    idx = rng.choice(p.n_obs, max(1, int(frac * p.n_obs)), replace=False)
    px[idx] += size * rng.choice([-1.0, 1.0], size=(len(idx), 2))
    return dataclasses.replace(p, pixels=px)


def test_robust_losses_closed_forms():
    s = np.array([0.0, 0.25, 1.0, 4.0, 100.0])
    assert np.array_equal(O.robust_rho(s, "squared"), s)
    # Huber (d = 1): s below d^2, 2 sqrt(s) - 1 above; continuous with slope 1 at d^2
    assert np.allclose(O.robust_rho(s, "huber", 1.0), [0.0, 0.25, 1.0, 3.0, 19.0])
    assert np.allclose(O.robust_weight(s, "huber", 1.0), [1.0, 1.0, 1.0, 0.5, 0.1])
    # Cauchy (d = 2): 4 log(1 + s/4); rho(d^2) = d^2 log 2
    assert np.isclose(O.robust_rho(np.array([4.0]), "cauchy", 2.0)[0], 4.0 * np.log(2.0))
    assert np.allclose(O.robust_weight(s, "cauchy", 2.0), 1.0 / (1.0 + s / 4.0))
    # weights are the derivatives of rho: central differences
    for loss, sc in (("huber", 1.0), ("cauchy", 2.0)):
        t = np.array([0.3, 2.5, 9.0, 50.0])
        fd = (O.robust_rho(t + 1e-6, loss, sc) - O.robust_rho(t - 1e-6, loss, sc)) / 2e-6
        assert np.allclose(fd, O.robust_weight(t, loss, sc), rtol=1e-6)


@pytest.mark.parametrize("loss", ["huber", "cauchy"])
def test_robust_gradient_is_the_gradient_of_the_robust_cost(loss):
    """g = sum_o rho'(s_o) J_o^T r_o is the exact gradient of 1/2 sum rho(s_o)."""
    p = _with_outliers(_small_problem(seed=45))
    lin = O.linearize(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels, loss=loss, loss_scale=2.0)
    x0 = O.pack(p.cams_init, p.pts_init)
    rng = np.random.default_rng(1)
    for k in rng.choice(x0.size, 12, replace=False):
        e = np.zeros_like(x0)
        h = 1e-6 * max(1.0, abs(x0[k]))
        e[k] = h
        Fp = O.robust_cost(*O.unpack(x0 + e, p.n_cams), p.cam_idx, p.pt_idx, p.pixels, loss=loss, loss_scale=2.0)
        Fm = O.robust_cost(*O.unpack(x0 - e, p.n_cams), p.cam_idx, p.pt_idx, p.pixels, loss=loss, loss_scale=2.0)
        fd = (Fp - Fm) / (2 * h)
        assert abs(fd - lin.g[k]) <= 1e-5 * max(1.0, np.abs(lin.g).max() * 1e-3) + 1e-6 * abs(fd), (k, fd, lin.g[k])
    assert np.isclose(lin.F, O.robust_cost(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels, loss=loss,
                                           loss_scale=2.0))


def test_huber_with_a_huge_scale_is_the_squared_loss():
    p = _small_problem(seed=46)
    a = O.ba_solve(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels, O.LMOptions(max_lm_iters=5))
    b = O.ba_solve(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels,
                   O.LMOptions(max_lm_iters=5, loss="huber", loss_scale=1e6))
    assert a.final_cost == b.final_cost and a.pcg_iters_total == b.pcg_iters_total


@pytest.mark.parametrize("loss", ["huber", "cauchy"])
def test_robust_lm_is_monotone_and_reaches_a_stationary_point(loss):
    p = _with_outliers(_small_problem(seed=47, n_cams=4, n_pts=40), frac=0.1)
    opts = O.LMOptions(max_lm_iters=200, max_pcg_iters=400, pcg_rel_tol=1e-10, loss=loss, loss_scale=2.0)
    r = O.ba_solve(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels, opts)
    costs = [h["cost"] for h in r.history] + [r.final_cost]
    assert all(a >= b for a, b in zip(costs, costs[1:]))
    c, q = O.unpack(r.x, p.n_cams)
    g_end = O.linearize(c, q, p.cam_idx, p.pt_idx, p.pixels, loss=loss, loss_scale=2.0).g
    g0 = O.linearize(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels, loss=loss, loss_scale=2.0).g
    assert np.linalg.norm(g_end) <= 1e-6 * np.linalg.norm(g0)


# ---------------------------------------------------------------- Schur PCG -------


def _dense_damped(lin, D, mu):
    H = (lin.J.T @ lin.J).toarray()
    return H + mu * np.diag(D)


def test_schur_operator_is_the_dense_schur_complement():
    p = _small_problem(seed=48, n_cams=3, n_pts=15)
    lin = O.linearize(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels)
    D = O.damping_diag(lin.J)
    mu = 0.05
    A = _dense_damped(lin, D, mu)
    nc9 = 9 * p.n_cams
    S_dense = A[:nc9, :nc9] - A[:nc9, nc9:] @ np.linalg.solve(A[nc9:, nc9:], A[nc9:, :nc9])
    # the reduced solve equals the dense Schur system's solution
    res = O.schur_pcg(lin, D, mu, p.n_cams, tol=1e-14, max_iters=500)
    b = -lin.g[:nc9] + A[:nc9, nc9:] @ np.linalg.solve(A[nc9:, nc9:], lin.g[nc9:])
    hc = np.linalg.solve(S_dense, b)
    assert np.allclose(res.h[:nc9], hc, rtol=1e-9, atol=1e-12 * np.abs(hc).max())


def test_schur_solve_equals_the_dense_direct_solve_of_the_damped_system():
    p = _small_problem(seed=49, n_cams=3, n_pts=20)
    lin = O.linearize(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels)
    D = O.damping_diag(lin.J)
    for mu in (1e-3, 0.3):
        A = _dense_damped(lin, D, mu)
        h = np.linalg.solve(A, -lin.g)
        res = O.schur_pcg(lin, D, mu, p.n_cams, tol=1e-14, max_iters=500)
        assert np.linalg.norm(res.h - h) <= 1e-9 * np.linalg.norm(h)


def test_lm_schur_reaches_the_pcgnr_optimum():
    p = _small_problem(seed=50, n_cams=4, n_pts=40)
    out = {}
    for sv in ("pcgnr", "schur"):
        opts = O.LMOptions(max_lm_iters=60, max_pcg_iters=400, pcg_rel_tol=1e-10, solver=sv)
        out[sv] = O.ba_solve(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels, opts)
    a, b = out["pcgnr"].final_cost, out["schur"].final_cost
    assert abs(a - b) <= 1e-9 * a


# ---------------------------------------------------------------- pose factors -----


def _factors(p, noise=True, pairs="chain+skip", seed=3):
    fa, fb, meas, sq = synth.make_pose_factors(p, pairs=pairs, seed=seed, noise=noise)
    return O.PoseFactors(fa, fb, meas, sq)


def test_pose_factor_zero_at_exact_measurements():
    p = _small_problem(n_cams=6)
    f = _factors(p, noise=False)
    assert np.abs(O.pose_factor_residuals(p.cams_gt, f)).max() < 1e-9
    assert O.pose_factor_cost(p.cams_init, f) > 1.0   # the perturbed start is off


def test_pose_factor_rows_match_scipy():
    """Rotation rows = s * rotvec(R_m^T R_b R_a^T), translation rows = s * (t_b - R_b R_a^T
    t_a - t_m), both computed through scipy's rotations."""
    p = _small_problem(n_cams=6)
    rng = np.random.default_rng(5)
    cams = p.cams_init.copy()
    cams[:, 0:3] += rng.normal(0, 0.3, (6, 3))
    f = _factors(p)
    f.sqrt_info = rng.uniform(0.5, 3.0, f.sqrt_info.shape)
    r = O.pose_factor_residuals(cams, f)
    Ra, Rb = Rotation.from_rotvec(cams[f.cam_a, 0:3]), Rotation.from_rotvec(cams[f.cam_b, 0:3])
    Rm = Rotation.from_rotvec(f.meas[:, 0:3])
    rot = (Rm.inv() * Rb * Ra.inv()).as_rotvec()
    tr = cams[f.cam_b, 3:6] - (Rb * Ra.inv()).apply(cams[f.cam_a, 3:6]) - f.meas[:, 3:6]
    np.testing.assert_allclose(r, f.sqrt_info * np.concatenate([rot, tr], axis=1), atol=1e-12, rtol=1e-10)


@pytest.mark.parametrize("retraction", [False, True])
def test_pose_factor_jacobian_matches_central_differences(retraction):
    p = _small_problem(n_cams=6)
    rng = np.random.default_rng(6)
    cams = p.cams_init.copy()
    cams[:, 0:3] += rng.normal(0, 0.3, (6, 3))
    f = _factors(p)
    f.sqrt_info = rng.uniform(0.5, 3.0, f.sqrt_info.shape)
    _, Ja, Jb = O.pose_factor_blocks(cams, f, retraction=retraction)
    eps = 1e-6
    for c in range(6):
        for k in range(9):
            cp, cm = cams.copy(), cams.copy()
            if retraction and k < 3:   # left step Exp(d) R(w), through scipy's composition
                d = np.zeros(3)
                d[k] = eps
                cp[c, 0:3] = (Rotation.from_rotvec(d) * Rotation.from_rotvec(cams[c, 0:3])).as_rotvec()
                cm[c, 0:3] = (Rotation.from_rotvec(-d) * Rotation.from_rotvec(cams[c, 0:3])).as_rotvec()
            else:
                cp[c, k] += eps
                cm[c, k] -= eps
            fd = (O.pose_factor_residuals(cp, f) - O.pose_factor_residuals(cm, f)) / (2 * eps)
            an = (f.cam_a == c)[:, None] * Ja[:, :, k] + (f.cam_b == c)[:, None] * Jb[:, :, k]
            np.testing.assert_allclose(an, fd, atol=2e-6 * max(1.0, np.abs(fd).max()))


def test_pose_factor_is_invariant_to_a_world_transform():
    """X' = R_w X + t_w changes each camera to (R_c R_w^T, t_c - R_c R_w^T t_w); relative
    poses, hence the residuals, do not change."""
    p = _small_problem(n_cams=6)
    f = _factors(p)
    Rw = Rotation.from_rotvec([0.3, -0.7, 1.1])
    tw = np.array([2.0, -1.0, 0.5])
    cams = p.cams_init.copy()
    Rc = Rotation.from_rotvec(cams[:, 0:3])
    moved = cams.copy()
    moved[:, 0:3] = (Rc * Rw.inv()).as_rotvec()
    moved[:, 3:6] = cams[:, 3:6] - (Rc * Rw.inv()).apply(np.tile(tw, (6, 1)))
    np.testing.assert_allclose(O.pose_factor_residuals(moved, f), O.pose_factor_residuals(cams, f), atol=1e-9)


def test_linearize_with_factors_appends_rows():
    """F, g and the camera blocks of J^T J with factors = the observation part plus the
    factor part assembled densely from the factor blocks."""
    p = _small_problem(n_cams=5, n_pts=30)
    f = _factors(p)
    base = O.linearize(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels)
    lin = O.linearize(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels, factors=f)
    r, Ja, Jb = O.pose_factor_blocks(p.cams_init, f)
    assert abs(lin.F - base.F - 0.5 * np.sum(r * r)) < 1e-9 * lin.F
    n = lin.J.shape[1]
    Jf = np.zeros((6 * len(f.cam_a), n))
    for k, (a, b) in enumerate(zip(f.cam_a, f.cam_b)):
        Jf[6 * k:6 * k + 6, 9 * a:9 * a + 9] += Ja[k]
        Jf[6 * k:6 * k + 6, 9 * b:9 * b + 9] += Jb[k]
    np.testing.assert_allclose(lin.g, base.g + Jf.T @ r.reshape(-1), rtol=1e-10, atol=1e-8)
    Hf = Jf.T @ Jf
    for c in range(p.n_cams):
        np.testing.assert_allclose(lin.Hc[c], base.Hc[c] + Hf[9 * c:9 * c + 9, 9 * c:9 * c + 9], rtol=1e-10, atol=1e-8)


def test_lm_with_exact_factors_reaches_zero_cost():
    """Noise-free pixels and exact relative poses: the optimum has zero cost and LM gets
    there from the perturbed start."""
    p = synth.make_problem(8, 200, ("poisson", 3.0), "uniform", seed=12, noise_px=0.0)
    f = _factors(p, noise=False)
    res = O.ba_solve(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels, O.LMOptions(max_lm_iters=30), factors=f)
    assert res.initial_cost > 1e3
    assert res.final_cost < 1e-8 * res.initial_cost


def test_lm_with_factors_is_monotone_and_stationary():
    p = _small_problem(seed=9, n_cams=6, n_pts=60)
    f = _factors(p)
    res = O.ba_solve(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels,
                     O.LMOptions(max_lm_iters=60, pcg_rel_tol=1e-10, max_pcg_iters=500), factors=f)
    costs = [h["cost"] for h in res.history] + [res.final_cost]
    assert all(a >= b for a, b in zip(costs, costs[1:]))
    c, q = O.unpack(res.x, p.n_cams)
    lin = O.linearize(c, q, p.cam_idx, p.pt_idx, p.pixels, factors=f)
    assert np.linalg.norm(lin.g) < 1e-6 * np.sqrt(lin.F)


def test_block_jacobi_falls_back_to_the_inverse_diagonal():
    """A rank-deficient block (mu = 0, a point seen along one ray) is not positive
    definite: its preconditioner block is the inverse diagonal; SPD blocks are exact."""
    A = np.zeros((2, 3, 3))
    A[0] = np.diag([4.0, 2.0, 1.0]) + 0.1
    u = np.array([1.0, 2.0, 2.0])
    A[1] = np.outer(u, u)                       # rank one
    M = O._spd_inverses(A)
    np.testing.assert_allclose(M[0], np.linalg.inv(A[0]), rtol=1e-12)
    np.testing.assert_allclose(M[1], np.diag(1.0 / np.diag(A[1])), rtol=1e-12)


def test_pose_factor_hand_cases():
    """Hand-worked residuals of the relative-pose factor (tests/golden/pose_factor_hand.json)."""
    data = json.load(open(os.path.join(GOLDEN, "pose_factor_hand.json")))
    for case in data["cases"]:
        cams = np.zeros((2, 9))
        cams[0, :6] = case["cam_a"]
        cams[1, :6] = case["cam_b"]
        f = O.PoseFactors(np.array([0]), np.array([1]), np.array([case["meas"]], float),
                          np.array([case["sqrt_info"]], float))
        np.testing.assert_allclose(O.pose_factor_residuals(cams, f)[0], case["residual"], atol=1e-12)
