"""Oracle pin: the reprojection cost is invariant under a similarity transform of the
scene, and the oracle's Jacobian must say so.

A similarity X -> s Q X + u, with every camera moved along (R -> R Q^T,
t -> s t - R Q^T u), leaves every camera-frame point scaled by s and so every projection
p = -P.xy / P.z unchanged (Sec. VI-A's residual, eps_depth = 0).  Its seven tangent
vectors V (three rotations, three translations, the scale) therefore satisfy J V = 0 for
the oracle's forward-mode Jacobian at any x:
  rotation k:    point dX = e_k x X;  camera dw = -J_l(w)^-1 R e_k for the additive
                 angle-axis update (R(w + d) = Exp(J_l d) R(w)), d = -R e_k for the
                 tangent-space retraction;
  translation k: point dX = e_k;      camera dt = -R e_k;
  scale:         point dX = X;        camera dt = t.
A dropped term, a wrong sign, a transposed R or a J_l in place of its inverse in the
oracle's camera derivatives leaves J V at the size of J; the planted slips below are
caught.  With eps_depth > 0 the scale stops being a symmetry and the rigid motions stay
one.  The exact damped LM step (J^T J + mu D) h = -g is D-orthogonal to V
(mu V^T D h = -V^T g = 0), and removing a D-weighted component along V changes neither
g^T h nor J h.
"""
import numpy as np
import pytest

from oracle import ba_oracle as O
from paper_2605_30583_gb300 import synth


def _skew(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def _rot_and_left_jacobian(w):
    th = np.linalg.norm(w)
    K = _skew(w)
    A = np.sin(th) / th
    B = (1.0 - np.cos(th)) / th ** 2
    C = (th - np.sin(th)) / th ** 3
    return np.eye(3) + A * K + B * K @ K, np.eye(3) + B * K + C * K @ K


def gauge_vectors(cams, pts, retraction=False, scale=True):
    """[9 n_cams + 3 n_pts, 7]: rotations (3), translations (3), scale."""
    n_c, n_p = len(cams), len(pts)
    V = np.zeros((9 * n_c + 3 * n_p, 7))
    for c in range(n_c):
        R, Jl = _rot_and_left_jacobian(cams[c, :3])
        G = -R if retraction else -np.linalg.solve(Jl, R)
        V[9 * c: 9 * c + 3, 0:3] = G
        V[9 * c + 3: 9 * c + 6, 3:6] = -R
        if scale:
            V[9 * c + 3: 9 * c + 6, 6] = cams[c, 3:6]
    for i in range(n_p):
        X = pts[i]
        e = 9 * n_c + 3 * i
        V[e: e + 3, 0:3] = -_skew(X)          # column k: e_k x X
        V[e: e + 3, 3:6] = np.eye(3)
        if scale:
            V[e: e + 3, 6] = X
    return V


@pytest.fixture(scope="module")
def prob():
    return synth.make_problem(6, 60, ("poisson", 3.0), "uniform", seed=11)


@pytest.mark.parametrize("retraction", [False, True])
def test_similarity_tangents_are_in_the_null_space_of_the_oracle_jacobian(prob, retraction):
    _, Jc, Jp = O.jacobian_blocks(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels,
                                  retraction=retraction)
    J = O.assemble_jacobian(Jc, Jp, prob.cam_idx, prob.pt_idx, prob.n_cams, prob.n_pts).toarray()
    V = gauge_vectors(prob.cams_init, prob.pts_init, retraction)
    scale = np.linalg.norm(J, axis=1)[:, None] * np.linalg.norm(V, axis=0)[None, :]
    assert np.max(np.abs(J @ V) / scale) < 1e-12, np.max(np.abs(J @ V) / scale)
    # planted in the oracle's Jacobian: a sign slip in d r / d w_0, and point columns
    # built from R^T instead of R
    Jc_bad = Jc.copy()
    Jc_bad[:, :, 0] *= -1.0
    J_bad = O.assemble_jacobian(Jc_bad, Jp, prob.cam_idx, prob.pt_idx, prob.n_cams, prob.n_pts).toarray()
    assert np.max(np.abs(J_bad @ V) / scale) > 1e-3
    R = np.stack([_rot_and_left_jacobian(w)[0] for w in prob.cams_init[:, :3]])
    Rc = R[prob.cam_idx]
    Jp_bad = np.einsum("oij,okj,olk->oil", Jp, Rc, Rc)   # A R^T in place of A R (J_p = A R)
    J_bad = O.assemble_jacobian(Jc, Jp_bad, prob.cam_idx, prob.pt_idx, prob.n_cams, prob.n_pts).toarray()
    assert np.max(np.abs(J_bad @ V) / scale) > 1e-3


def test_rotation_parameterisations_are_not_interchangeable(prob):
    """The additive update's Jacobian (w.r.t. w) with the retraction's tangents, and the
    other way round: a mix-up of the two in the oracle would show here."""
    for jac_retraction in (False, True):
        _, Jc, Jp = O.jacobian_blocks(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels,
                                      retraction=jac_retraction)
        J = O.assemble_jacobian(Jc, Jp, prob.cam_idx, prob.pt_idx, prob.n_cams, prob.n_pts).toarray()
        V = gauge_vectors(prob.cams_init, prob.pts_init, retraction=not jac_retraction)
        scale = np.linalg.norm(J, axis=1)[:, None] * np.linalg.norm(V, axis=0)[None, :]
        assert np.max(np.abs(J @ V[:, :3]) / scale[:, :3]) > 1e-4


def test_scale_leaves_the_null_space_with_a_depth_offset(prob):
    """With eps_depth > 0 the projection p = -P.xy / (P_z + eps sign P_z) is no longer
    scale invariant: the scale vector stops being null while the rigid ones stay."""
    _, Jc, Jp = O.jacobian_blocks(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels,
                                  eps_depth=0.5)
    J = O.assemble_jacobian(Jc, Jp, prob.cam_idx, prob.pt_idx, prob.n_cams, prob.n_pts).toarray()
    V = gauge_vectors(prob.cams_init, prob.pts_init)
    rel = np.linalg.norm(J @ V, axis=0) / (np.linalg.norm(J) * np.linalg.norm(V, axis=0))
    assert np.all(rel[:6] < 1e-12) and rel[6] > 1e-6, rel


def test_projection_keeps_the_model_and_the_exact_step_is_already_projected(prob):
    lin = O.linearize(prob.cams_init, prob.pts_init, prob.cam_idx, prob.pt_idx, prob.pixels)
    J = lin.J.toarray()
    g = np.asarray(lin.g)
    D = O.damping_diag(lin.J)
    V = gauge_vectors(prob.cams_init, prob.pts_init)
    mu = 1e-3
    h = -np.linalg.solve(J.T @ J + mu * np.diag(D), g)                  # the exact damped step
    assert np.max(np.abs(V.T @ (D * h))) <= 1e-8 * np.linalg.norm(V.T @ np.abs(D * h))
    rng = np.random.default_rng(3)
    hh = h + V @ rng.standard_normal(7)                                   # a step with a gauge part
    c = np.linalg.solve(V.T @ (D[:, None] * V), V.T @ (D * hh))
    hp = hh - V @ c
    assert np.allclose(g @ hp, g @ hh, rtol=1e-9) and np.allclose(J @ hp, J @ hh, rtol=1e-7, atol=1e-9)
    assert np.allclose(hp, h, rtol=1e-6, atol=1e-9 * np.linalg.norm(h))
