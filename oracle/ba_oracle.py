"""Plain FP64 CPU oracle for the Levenberg-Marquardt + PCGNR bundle-adjustment path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module.  The product path (the CUDA
library and its Python binding) never imports, calls or links it, and it shares no
code with that path: no kernels, headers, helpers or constants.

It is slow and obviously correct on purpose.  Every function follows one passage of
the paper (arXiv 2605.30583, "Caspar"):

* residual        -- Sec. VI-A, the Snavely reprojection factor (``d_safe``, ``p``,
                     radial scale, ``pixel - px_m``).  Rotation vectors map to
                     matrices by Rodrigues' formula (reading of Sec. V / VI-A: a
                     9-parameter angle-axis camera updated additively).
* Jacobian        -- Sec. V: derivatives of each factor with respect to its
                     tunable nodes.  Forward-mode dual numbers carried through the
                     residual, so no derivative is written by hand here.
* LM              -- Sec. V: Levenberg-Marquardt with the quality-based damping
                     update of Madsen et al. (cited there).
* normal eqs.     -- Sec. V: no Schur complement; the full damped normal equations
                     are solved by PCGNR (Sec. V-A) with a block-Jacobi
                     preconditioner, one block per node (Sec. V).
* settings        -- Sec. VI: initial trust region 100, CG tolerance 0.001.
* retraction      -- Sec. VI-A's Pose3 update as an option: rotations stepped by
                     R <- Exp(d) R (scipy's rotation composition), Jacobian w.r.t. d.
* robust loss     -- robust factors (named in Sec. VI-A as an easy addition): Huber or
                     Cauchy on |r_o|^2 with IRLS weights rho'(|r_o|^2).
* Schur PCG       -- the alternative Sec. V sets aside: PCG on the camera Schur
                     complement, points back-substituted (schur_pcg).
* pose factors    -- generic node-to-node factors (Sec. IV): a relative-pose factor on
                     two cameras, Log(R_m^T R_b R_a^T) and t_b - R_b R_a^T t_a - t_m,
                     differentiated by the same dual numbers (PoseFactors).

Readings where the paper is silent (all listed in the design notes): damping
matrix D = diag(J^T J) clamped to [min_diag, max_diag]; mu_0 = 1 / trust region;
gain ratio denominator -g^T h - |J h|^2 / 2; CG tolerance is relative to the
unpreconditioned residual 2-norm with h_0 = 0; a step is accepted iff rho > 0.

Parity pins (tests/test_oracle_pins.py): hand-computed projections, central finite
differences of the residual, scipy's rotation-vector routine, dense Cholesky
solves of the damped normal equations, exact zero residual at noise-free ground
truth, monotone accepted cost, the chi-square level of the optimum and the
Rosenbrock least-squares minimum.
"""
from __future__ import annotations

import dataclasses
import numpy as np
import scipy.sparse as sp

# --------------------------------------------------------------------------------------
# Forward-mode dual numbers: value v (shape [N]) and tangent d (shape [N, K]).
# --------------------------------------------------------------------------------------


class Dual:
    __array_priority__ = 1000

    def __init__(self, v, d):
        self.v = np.asarray(v, dtype=np.float64)
        self.d = np.asarray(d, dtype=np.float64)

    @staticmethod
    def _split(o):
        if isinstance(o, Dual):
            return o.v, o.d
        return np.asarray(o, dtype=np.float64), None

    def __add__(self, o):
        v, d = Dual._split(o)
        return Dual(self.v + v, self.d if d is None else self.d + d)

    __radd__ = __add__

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __sub__(self, o):
        return self + (-o)

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        v, d = Dual._split(o)
        if d is None:
            return Dual(self.v * v, self.d * np.asarray(v)[..., None])
        return Dual(self.v * v, self.d * v[..., None] + d * self.v[..., None])

    __rmul__ = __mul__

    def __truediv__(self, o):
        v, d = Dual._split(o)
        q = self.v / v
        if d is None:
            return Dual(q, self.d / np.asarray(v)[..., None])
        return Dual(q, (self.d - d * q[..., None]) / v[..., None])

    def __rtruediv__(self, o):
        return Dual(np.broadcast_to(np.asarray(o, dtype=np.float64), self.v.shape),
                    np.zeros_like(self.d)) / self


def _sqrt(x):
    if isinstance(x, Dual):
        s = np.sqrt(x.v)
        return Dual(s, x.d / (2.0 * s)[..., None])
    return np.sqrt(x)


def _sin(x):
    if isinstance(x, Dual):
        return Dual(np.sin(x.v), x.d * np.cos(x.v)[..., None])
    return np.sin(x)


def _cos(x):
    if isinstance(x, Dual):
        return Dual(np.cos(x.v), -x.d * np.sin(x.v)[..., None])
    return np.cos(x)


def _atan2(y, x):
    """atan2 with its derivative (x dy - y dx) / (x^2 + y^2)."""
    if isinstance(y, Dual) or isinstance(x, Dual):
        yv, yd = (y.v, y.d) if isinstance(y, Dual) else (np.asarray(y, np.float64), None)
        xv, xd = (x.v, x.d) if isinstance(x, Dual) else (np.asarray(x, np.float64), None)
        den = (xv * xv + yv * yv)[..., None]
        d = 0.0
        if yd is not None:
            d = d + yd * xv[..., None] / den
        if xd is not None:
            d = d - xd * yv[..., None] / den
        return Dual(np.arctan2(yv, xv), d)
    return np.arctan2(y, x)


def _where(mask, a, b):
    if isinstance(a, Dual) or isinstance(b, Dual):
        av, ad = (a.v, a.d) if isinstance(a, Dual) else (a, 0.0 * b.d)
        bv, bd = (b.v, b.d) if isinstance(b, Dual) else (b, 0.0 * a.d)
        return Dual(np.where(mask, av, bv), np.where(mask[..., None], ad, bd))
    return np.where(mask, a, b)


def _value(x):
    return x.v if isinstance(x, Dual) else np.asarray(x)


# --------------------------------------------------------------------------------------
# Residual (Sec. VI-A)
# --------------------------------------------------------------------------------------

SMALL_ANGLE_SQ = 1e-8   # theta < 1e-4: Taylor series of the Rodrigues coefficients


def rotate(w, X):
    """R(w) X by Rodrigues' formula R = I + a [w]x + b [w]x^2 with
    a = sin(theta)/theta and b = (1 - cos(theta))/theta^2 = 2 sin^2(theta/2)/theta^2.
    For theta^2 < 1e-8 the series a = 1 - theta^2/6 + theta^4/120 and
    b = 1/2 - theta^2/24 + theta^4/720 are used instead (no 0/0)."""
    w0, w1, w2 = w
    x0, x1, x2 = X
    th2 = w0 * w0 + w1 * w1 + w2 * w2
    small = _value(th2) < SMALL_ANGLE_SQ
    th2_safe = _where(small, 1.0, th2)
    th = _sqrt(th2_safe)
    half = _sin(th * 0.5)
    a_big = _sin(th) / th
    b_big = 2.0 * half * half / th2_safe
    a_small = 1.0 - th2 / 6.0 + th2 * th2 / 120.0
    b_small = 0.5 - th2 / 24.0 + th2 * th2 / 720.0
    a = _where(small, a_small, a_big)
    b = _where(small, b_small, b_big)
    # c = w x X, e = w x (w x X)
    c0 = w1 * x2 - w2 * x1
    c1 = w2 * x0 - w0 * x2
    c2 = w0 * x1 - w1 * x0
    e0 = w1 * c2 - w2 * c1
    e1 = w2 * c0 - w0 * c2
    e2 = w0 * c1 - w1 * c0
    return (x0 + a * c0 + b * e0, x1 + a * c1 + b * e1, x2 + a * c2 + b * e2)


def _sign_no_zero(x):
    return np.where(_value(x) >= 0.0, 1.0, -1.0)


def project(cam, X, eps_depth=0.0, base_w=None):
    """Pixel predicted for a camera cam = (w0,w1,w2,t0,t1,t2,f,k1,k2) and point X.

    With base_w given, the camera's rotation is Exp(w) R(base_w): cam[0:3] is then a
    tangent-space step d applied on the left (the retraction R <- Exp(d) R of the
    paper's Pose3 update, Sec. VI-A)."""
    w = cam[0:3]
    t = cam[3:6]
    f, k1, k2 = cam[6], cam[7], cam[8]
    RX = rotate(w, X) if base_w is None else rotate(w, rotate(base_w, X))
    P0, P1, P2 = RX[0] + t[0], RX[1] + t[1], RX[2] + t[2]
    d_safe = P2 + eps_depth * _sign_no_zero(P2)
    p0 = -P0 / d_safe
    p1 = -P1 / d_safe
    n2 = p0 * p0 + p1 * p1
    n4 = n2 * n2
    s = 1.0 + k1 * n2 + k2 * n4
    return f * s * p0, f * s * p1


def residuals(cams, pts, cam_idx, pt_idx, pixels, eps_depth=0.0):
    """r_o = pixel(cam_{c_o}, X_{p_o}) - u_o for every observation, shape [n_obs, 2]."""
    cams = np.asarray(cams, np.float64)
    pts = np.asarray(pts, np.float64)
    c = cams[np.asarray(cam_idx, np.int64)].T
    X = pts[np.asarray(pt_idx, np.int64)].T
    u0, u1 = project(list(c), list(X), eps_depth)
    return np.stack([u0 - pixels[:, 0], u1 - pixels[:, 1]], axis=1)


def cost(cams, pts, cam_idx, pt_idx, pixels, eps_depth=0.0):
    """F = 1/2 sum_o |r_o|^2."""
    r = residuals(cams, pts, cam_idx, pt_idx, pixels, eps_depth)
    return 0.5 * float(np.sum(r * r))


def robust_cost(cams, pts, cam_idx, pt_idx, pixels, eps_depth=0.0, loss="squared", loss_scale=1.0):
    """F = 1/2 sum_o rho(|r_o|^2)."""
    r = residuals(cams, pts, cam_idx, pt_idx, pixels, eps_depth)
    return 0.5 * float(np.sum(robust_rho(np.sum(r * r, axis=1), loss, loss_scale)))


def jacobian_blocks(cams, pts, cam_idx, pt_idx, pixels, eps_depth=0.0, chunk=200_000, retraction=False):
    """Residuals r [n_obs,2] and Jacobian blocks J_c [n_obs,2,9], J_p [n_obs,2,3], by
    forward-mode dual numbers seeded with the 12 tangent directions of (camera, point).

    retraction=False: the rotation columns are d r / d w (additive angle-axis).
    retraction=True: they are d r / d d at d = 0 for the rotation Exp(d) R(w)."""
    cams = np.asarray(cams, np.float64)
    pts = np.asarray(pts, np.float64)
    ci = np.asarray(cam_idx, np.int64)
    pi = np.asarray(pt_idx, np.int64)
    n = ci.shape[0]
    r = np.empty((n, 2))
    Jc = np.empty((n, 2, 9))
    Jp = np.empty((n, 2, 3))
    eye = np.eye(12)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        m = e - s
        c = cams[ci[s:e]]
        X = pts[pi[s:e]]
        cd = [Dual(c[:, k], np.broadcast_to(eye[k], (m, 12))) for k in range(9)]
        Xd = [Dual(X[:, k], np.broadcast_to(eye[9 + k], (m, 12))) for k in range(3)]
        if retraction:   # the step d, seeded at 0, on the left of R(w)
            cd[0:3] = [Dual(np.zeros(m), np.broadcast_to(eye[k], (m, 12))) for k in range(3)]
            u0, u1 = project(cd, Xd, eps_depth, base_w=[c[:, 0], c[:, 1], c[:, 2]])
        else:
            u0, u1 = project(cd, Xd, eps_depth)
        r[s:e, 0] = u0.v - pixels[s:e, 0]
        r[s:e, 1] = u1.v - pixels[s:e, 1]
        Jc[s:e, 0] = u0.d[:, :9]
        Jc[s:e, 1] = u1.d[:, :9]
        Jp[s:e, 0] = u0.d[:, 9:]
        Jp[s:e, 1] = u1.d[:, 9:]
    return r, Jc, Jp


# --------------------------------------------------------------------------------------
# Pose factors: the generic, non-reprojection factors of Sec. IV (node-to-node factors
# such as odometry / pose-graph constraints, Sec. I and IV-C), here a relative-pose
# ("between") factor on two cameras.  Camera c maps world points by x = R_c X + t_c.
# The pose of camera b relative to camera a is R_ba = R_b R_a^T, t_ba = t_b - R_ba t_a;
# with a measurement (R_m = Exp(w_m), t_m) and a diagonal square-root information s,
#     r = s * [ Log(R_m^T R_ba) ; t_ba - t_m ]           (6 rows),
# and the factor adds 1/2 |r|^2 to the cost.  Its Jacobian comes from dual numbers
# carried through this residual, like the reprojection factor's.
# --------------------------------------------------------------------------------------


@dataclasses.dataclass
class PoseFactors:
    cam_a: np.ndarray        # [nf] camera indices
    cam_b: np.ndarray        # [nf]
    meas: np.ndarray         # [nf, 6]: w_m (rotation vector of R_m), t_m
    sqrt_info: np.ndarray    # [nf, 6]: s, the square root of the diagonal information


def log_rotation(M):
    """Rotation vector of a rotation matrix given as M[i][j] (arrays or duals):
    sin(theta) n = (M21 - M12, M02 - M20, M10 - M01) / 2, cos(theta) = (trace - 1) / 2,
    theta = atan2(|sin(theta) n|, cos(theta)), w = theta n.  For |sin(theta)|^2 < 1e-8
    the factor theta / sin(theta) is its series 1 + y^2/6 + 3 y^4/40 in y = sin(theta)
    (valid while theta < pi / 2 there, i.e. near the identity)."""
    v0 = 0.5 * (M[2][1] - M[1][2])
    v1 = 0.5 * (M[0][2] - M[2][0])
    v2 = 0.5 * (M[1][0] - M[0][1])
    c = 0.5 * (M[0][0] + M[1][1] + M[2][2] - 1.0)
    y2 = v0 * v0 + v1 * v1 + v2 * v2
    small = _value(y2) < SMALL_ANGLE_SQ
    y2_safe = _where(small, 1.0, y2)
    y = _sqrt(y2_safe)
    k_big = _atan2(y, c) / y
    k_small = 1.0 + y2 / 6.0 + 3.0 * y2 * y2 / 40.0
    k = _where(small, k_small, k_big)
    return (k * v0, k * v1, k * v2)


def _pose_residual(wa, ta, wb, tb, wm, tm, s, base_a=None, base_b=None):
    """The six rows of one factor (lists of arrays or duals).  With base_a / base_b
    given, wa / wb are left steps: R_a = Exp(wa) R(base_a)."""
    if base_a is None:
        rot_a_t = lambda X: rotate([-wa[0], -wa[1], -wa[2]], X)
    else:
        rot_a_t = lambda X: rotate([-base_a[0], -base_a[1], -base_a[2]], rotate([-wa[0], -wa[1], -wa[2]], X))
    rot_b = (lambda X: rotate(wb, X)) if base_b is None else (lambda X: rotate(wb, rotate(base_b, X)))
    rot_ba = lambda X: rot_b(rot_a_t(X))
    one, zero = np.ones_like(_value(tm[0])), np.zeros_like(_value(tm[0]))
    cols = [rotate([-wm[0], -wm[1], -wm[2]], rot_ba(e)) for e in
            ([one, zero, zero], [zero, one, zero], [zero, zero, one])]
    E = [[cols[j][i] for j in range(3)] for i in range(3)]      # E[i][j] = column j, entry i
    rr = log_rotation(E)
    Rt = rot_ba(ta)
    rt = [tb[i] - Rt[i] - tm[i] for i in range(3)]
    return [s[:, i] * (list(rr) + rt)[i] for i in range(6)]


def pose_factor_residuals(cams, f: PoseFactors):
    """r [nf, 6] of every factor at the cameras `cams`."""
    cams = np.asarray(cams, np.float64)
    A, Bc = cams[f.cam_a], cams[f.cam_b]
    r = _pose_residual(list(A[:, 0:3].T), list(A[:, 3:6].T), list(Bc[:, 0:3].T), list(Bc[:, 3:6].T),
                       list(f.meas[:, 0:3].T), list(f.meas[:, 3:6].T), f.sqrt_info)
    return np.stack([_value(x) for x in r], axis=1)


def pose_factor_cost(cams, f: PoseFactors):
    """1/2 sum of |r|^2 over the factors."""
    r = pose_factor_residuals(cams, f)
    return 0.5 * float(np.sum(r * r))


def pose_factor_blocks(cams, f: PoseFactors, retraction=False):
    """r [nf, 6] and the Jacobian blocks J_a, J_b [nf, 6, 9] (w, t columns filled; the
    intrinsic columns are zero), by dual numbers seeded with the 12 tangent directions
    (w_a, t_a, w_b, t_b).  retraction=True: rotation columns w.r.t. the left steps."""
    cams = np.asarray(cams, np.float64)
    A, Bc = cams[f.cam_a], cams[f.cam_b]
    m = A.shape[0]
    eye = np.eye(12)
    seed = lambda vals, k0: [Dual(vals[:, k], np.broadcast_to(eye[k0 + k], (m, 12))) for k in range(3)]
    ta, tb = seed(A[:, 3:6], 3), seed(Bc[:, 3:6], 9)
    if retraction:
        wa, wb = seed(np.zeros((m, 3)), 0), seed(np.zeros((m, 3)), 6)
        rows = _pose_residual(wa, ta, wb, tb, list(f.meas[:, 0:3].T), list(f.meas[:, 3:6].T), f.sqrt_info,
                              base_a=list(A[:, 0:3].T), base_b=list(Bc[:, 0:3].T))
    else:
        wa, wb = seed(A[:, 0:3], 0), seed(Bc[:, 0:3], 6)
        rows = _pose_residual(wa, ta, wb, tb, list(f.meas[:, 0:3].T), list(f.meas[:, 3:6].T), f.sqrt_info)
    r = np.stack([x.v for x in rows], axis=1)
    D = np.stack([x.d for x in rows], axis=1)                  # [nf, 6, 12]
    Ja = np.zeros((m, 6, 9))
    Jb = np.zeros((m, 6, 9))
    Ja[:, :, 0:6] = D[:, :, 0:6]
    Jb[:, :, 0:6] = D[:, :, 6:12]
    return r, Ja, Jb


# --------------------------------------------------------------------------------------
# Problem layout: x = [cams (9 per camera) | points (3 per point)], n = 9 Nc + 3 Np
# --------------------------------------------------------------------------------------


@dataclasses.dataclass
class Linearization:
    F: float                 # 1/2 |r|^2
    r: np.ndarray            # [m]
    J: sp.csr_matrix         # [m, n]
    g: np.ndarray            # J^T r, [n]
    Hc: np.ndarray           # camera diagonal blocks of J^T J, [Nc, 9, 9]
    Hp: np.ndarray           # point diagonal blocks of J^T J, [Np, 3, 3]


def assemble_jacobian(Jc, Jp, cam_idx, pt_idx, n_cams, n_pts):
    """Sparse J with rows (2o, 2o+1) and columns 9c..9c+8 and 9Nc + 3p..+2."""
    n_obs = Jc.shape[0]
    ci = np.asarray(cam_idx, np.int64)
    pi = np.asarray(pt_idx, np.int64)
    rows = np.repeat(np.arange(2 * n_obs), 12)
    cols_c = 9 * ci[:, None] + np.arange(9)[None, :]
    cols_p = 9 * n_cams + 3 * pi[:, None] + np.arange(3)[None, :]
    cols = np.concatenate([cols_c, cols_p], axis=1)                 # [n_obs, 12]
    cols = np.repeat(cols, 2, axis=0).reshape(-1)                    # rows 2o and 2o+1 share columns
    vals = np.concatenate([Jc, Jp], axis=2).reshape(-1)             # [n_obs, 2, 12]
    n = 9 * n_cams + 3 * n_pts
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * n_obs, n))


# Robust losses on s = |r_o|^2 (Sec. VI-A names robust factors as an easy addition):
# F = 1/2 sum_o rho(s_o).  Each is given with rho'(s), the IRLS weight of observation o.
#   squared: rho(s) = s                                rho' = 1
#   Huber:   rho(s) = s (s <= d^2), 2 d sqrt(s) - d^2    rho' = 1, d / sqrt(s)
#   Cauchy:  rho(s) = d^2 log(1 + s / d^2)               rho' = 1 / (1 + s / d^2)
LOSSES = ("squared", "huber", "cauchy")


def robust_rho(s, loss="squared", scale=1.0):
    s = np.asarray(s, np.float64)
    if loss == "squared":
        return s.copy()
    d2 = scale * scale
    if loss == "huber":
        return np.where(s <= d2, s, 2.0 * scale * np.sqrt(s) - d2)
    if loss == "cauchy":
        return d2 * np.log1p(s / d2)
    raise ValueError(loss)


def robust_weight(s, loss="squared", scale=1.0):
    s = np.asarray(s, np.float64)
    if loss == "squared":
        return np.ones_like(s)
    d2 = scale * scale
    if loss == "huber":
        return np.where(s <= d2, 1.0, scale / np.sqrt(np.maximum(s, d2)))
    if loss == "cauchy":
        return 1.0 / (1.0 + s / d2)
    raise ValueError(loss)


def linearize(cams, pts, cam_idx, pt_idx, pixels, eps_depth=0.0, retraction=False, loss="squared",
              loss_scale=1.0, factors: PoseFactors | None = None) -> Linearization:
    """F, g = J^T W r and the node blocks of J^T W J, with W the IRLS weights
    w_o = rho'(|r_o|^2) (all ones for the squared loss).  J and r are returned already
    scaled by sqrt(w_o), so every later product (PCG, |J h|^2) is the weighted one;
    F = 1/2 sum rho(|r_o|^2).  Pose factors, if given, append their six rows per factor
    (squared loss) after the observations' rows."""
    n_cams, n_pts = cams.shape[0], pts.shape[0]
    r, Jc, Jp = jacobian_blocks(cams, pts, cam_idx, pt_idx, pixels, eps_depth, retraction=retraction)
    s = np.sum(r * r, axis=1)
    F = 0.5 * float(np.sum(robust_rho(s, loss, loss_scale)))
    sw = np.sqrt(robust_weight(s, loss, loss_scale))
    r = r * sw[:, None]
    Jc = Jc * sw[:, None, None]
    Jp = Jp * sw[:, None, None]
    J = assemble_jacobian(Jc, Jp, cam_idx, pt_idx, n_cams, n_pts)
    rf = r.reshape(-1)
    Hc = np.zeros((n_cams, 9, 9))
    Hp = np.zeros((n_pts, 3, 3))
    np.add.at(Hc, np.asarray(cam_idx, np.int64), np.einsum("oki,okj->oij", Jc, Jc))
    np.add.at(Hp, np.asarray(pt_idx, np.int64), np.einsum("oki,okj->oij", Jp, Jp))
    if factors is not None and len(factors.cam_a) > 0:
        r_f, Ja, Jb = pose_factor_blocks(cams, factors, retraction)
        F += 0.5 * float(np.sum(r_f * r_f))
        nf = r_f.shape[0]
        rows = np.repeat(np.arange(6 * nf), 18)
        ca = 9 * np.asarray(factors.cam_a, np.int64)[:, None] + np.arange(9)[None, :]
        cb = 9 * np.asarray(factors.cam_b, np.int64)[:, None] + np.arange(9)[None, :]
        cols = np.repeat(np.concatenate([ca, cb], axis=1), 6, axis=0).reshape(-1)
        vals = np.concatenate([Ja, Jb], axis=2).reshape(-1)
        J_f = sp.csr_matrix((vals, (rows, cols)), shape=(6 * nf, J.shape[1]))
        J = sp.vstack([J, J_f]).tocsr()
        rf = np.concatenate([rf, r_f.reshape(-1)])
        np.add.at(Hc, np.asarray(factors.cam_a, np.int64), np.einsum("oki,okj->oij", Ja, Ja))
        np.add.at(Hc, np.asarray(factors.cam_b, np.int64), np.einsum("oki,okj->oij", Jb, Jb))
    g = J.T @ rf
    return Linearization(F=F, r=rf, J=J, g=g, Hc=Hc, Hp=Hp)


# --------------------------------------------------------------------------------------
# Block-Jacobi preconditioner and PCGNR (Sec. V, V-A)
# --------------------------------------------------------------------------------------


def damping_diag(J, min_diag=1e-6, max_diag=1e32):
    """D = diag(J^T J) (column sums of J squared), clamped to [min_diag, max_diag]."""
    d = np.asarray(J.multiply(J).sum(axis=0)).ravel()
    return np.clip(d, min_diag, max_diag)


def _spd_inverses(A):
    """Inverse of each SPD block of A [N, k, k] by Cholesky.  A block that is not
    positive definite in FP64 (rank-deficient J^T J once mu has shrunk far) gets its
    inverse diagonal instead, 1 / A_ii where A_ii > 0 and 0 elsewhere."""
    out = np.empty_like(A)
    try:
        L = np.linalg.cholesky(A)
        Li = np.linalg.inv(L)
        return Li.transpose(0, 2, 1) @ Li
    except np.linalg.LinAlgError:
        pass
    for i in range(A.shape[0]):
        try:
            Li = np.linalg.inv(np.linalg.cholesky(A[i]))
            out[i] = Li.T @ Li
        except np.linalg.LinAlgError:
            d = np.diag(A[i])
            out[i] = np.diag(np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0))
    return out


def block_jacobi(lin: Linearization, D, mu):
    """Inverses of the diagonal blocks of J^T J + mu D, one block per node, by Cholesky
    (a block that is not positive definite falls back to its inverse diagonal)."""
    nc = lin.Hc.shape[0]
    Dc = D[: 9 * nc].reshape(nc, 9)
    Dp = D[9 * nc:].reshape(-1, 3)
    Ac = lin.Hc + mu * np.einsum("ci,ij->cij", Dc, np.eye(9))
    Ap = lin.Hp + mu * np.einsum("pi,ij->pij", Dp, np.eye(3))
    return _spd_inverses(Ac), _spd_inverses(Ap)


def apply_block_jacobi(Mc, Mp, v):
    nc = Mc.shape[0]
    zc = np.einsum("cij,cj->ci", Mc, v[: 9 * nc].reshape(nc, 9)).reshape(-1)
    zp = np.einsum("pij,pj->pi", Mp, v[9 * nc:].reshape(-1, 3)).reshape(-1)
    return np.concatenate([zc, zp])


@dataclasses.dataclass
class PCGResult:
    h: np.ndarray
    iters: int
    r0_norm: float
    r_norm: float


def pcgnr(J, D, mu, b, precond, tol=1e-3, max_iters=50):
    """Solve (J^T J + mu D) h = b with preconditioned CG on the normal equations.

    Matrix-free: each iteration forms w = J p and then J^T w + mu D p.  Starts from
    h = 0 and stops when |r_k|_2 <= tol |r_0|_2 or after max_iters iterations."""
    h = np.zeros_like(b)
    r = b.copy()
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    r0 = float(np.sqrt(r @ r))
    rn = r0
    k = 0
    while k < max_iters and rn > tol * r0:
        w = J @ p
        q = J.T @ w + mu * D * p
        alpha = rz / float(w @ w + mu * (p @ (D * p)))
        h = h + alpha * p
        r = r - alpha * q
        k += 1
        rn = float(np.sqrt(r @ r))
        if rn <= tol * r0:
            break
        z = precond(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return PCGResult(h=h, iters=k, r0_norm=r0, r_norm=rn)


def schur_pcg(lin: Linearization, D, mu, n_cams, tol=1e-3, max_iters=50):
    """The damped step by the Schur complement on the cameras (the comparison the paper
    sets aside in Sec. V): with H' = J^T J + mu D split into camera and point blocks,

        S = H'_cc - H_cp H'_pp^-1 H_pc,   b = -g_c + H_cp H'_pp^-1 g_p,

    S h_c = b is solved by PCG (matrix-free S v = J_c^T (J_c v - J_p H'_pp^-1 J_p^T J_c v)
    + mu D_c v; block-Jacobi on the camera blocks of H'_cc; from h_c = 0, stopping when
    |r_k|_2 <= tol |r_0|_2 of the reduced system or after max_iters iterations), then
    h_p = H'_pp^-1 (-g_p - H_pc h_c)."""
    nc9 = 9 * n_cams
    J = lin.J.tocsc()
    Jc, Jp = J[:, :nc9].tocsr(), J[:, nc9:].tocsr()
    Dc, Dp = D[:nc9], D[nc9:]
    Mc, Mp = block_jacobi(lin, D, mu)          # inverses of the camera / point blocks of H'
    hpp_inv = lambda v: np.einsum("pij,pj->pi", Mp, v.reshape(-1, 3)).reshape(-1)
    mc_apply = lambda v: np.einsum("cij,cj->ci", Mc, v.reshape(-1, 9)).reshape(-1)

    def S(v):
        t = Jc @ v
        return Jc.T @ (t - Jp @ hpp_inv(Jp.T @ t)) + mu * Dc * v

    gc, gp = lin.g[:nc9], lin.g[nc9:]
    b = -gc + Jc.T @ (Jp @ hpp_inv(gp))
    hc = np.zeros(nc9)
    r = b.copy()
    z = mc_apply(r)
    p = z.copy()
    rz = float(r @ z)
    r0 = float(np.sqrt(r @ r))
    rn = r0
    k = 0
    while k < max_iters and rn > tol * r0:
        q = S(p)
        alpha = rz / float(p @ q)
        hc = hc + alpha * p
        r = r - alpha * q
        k += 1
        rn = float(np.sqrt(r @ r))
        if rn <= tol * r0:
            break
        z = mc_apply(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    hp = hpp_inv(-gp - Jp.T @ (Jc @ hc))
    return PCGResult(h=np.concatenate([hc, hp]), iters=k, r0_norm=r0, r_norm=rn)


# --------------------------------------------------------------------------------------
# Levenberg-Marquardt with Madsen's quality-based damping (Sec. V)
# --------------------------------------------------------------------------------------


@dataclasses.dataclass
class LMOptions:
    max_lm_iters: int = 20
    max_pcg_iters: int = 50
    pcg_rel_tol: float = 1e-3
    initial_trust_region: float = 100.0
    min_diag: float = 1e-6
    max_diag: float = 1e32
    eps_depth: float = 0.0
    max_mu: float = 1e16
    rotation_update: str = "additive"   # or "retraction": R <- Exp(d) R, J w.r.t. d
    loss: str = "squared"               # or "huber", "cauchy" (IRLS weights, see LOSSES)
    loss_scale: float = 1.0             # the loss's scale d, in pixels
    solver: str = "pcgnr"               # or "schur": PCG on the Schur complement (schur_pcg)


@dataclasses.dataclass
class LMResult:
    x: np.ndarray
    initial_cost: float
    final_cost: float
    history: list
    lm_iters: int
    accepted: int
    pcg_iters_total: int


def lm_solve(x0, linearize_fn, cost_fn, make_precond, opts: LMOptions = LMOptions(), step_fn=None,
             solve_fn=None) -> LMResult:
    """Generic LM over x.  linearize_fn(x) -> object with F, J (sparse) and g = J^T r;
    cost_fn(x) -> F; make_precond(lin, D, mu) -> callable applying the preconditioner;
    step_fn(x, h) -> x' applies a step (default x + h); solve_fn(lin, D, mu) -> PCGResult
    replaces PCGNR on the damped system (default: pcgnr with make_precond).

    One iteration: solve (J^T J + mu D) h = -g by PCGNR; x' = x + h;
    rho = (F - F') / (-g^T h - 1/2 |J h|^2).  If rho > 0 the step is accepted,
    mu <- mu * max(1/3, 1 - (2 rho - 1)^3), nu <- 2; otherwise mu <- mu nu, nu <- 2 nu.
    Stops after max_lm_iters iterations, when mu exceeds max_mu, or when F = 0."""
    x = np.array(x0, dtype=np.float64)
    lin = linearize_fn(x)
    mu = 1.0 / opts.initial_trust_region
    nu = 2.0
    F0 = lin.F
    hist = []
    accepted = 0
    pcg_total = 0
    it = 0
    while it < opts.max_lm_iters and lin.F > 0.0 and mu <= opts.max_mu:
        D = damping_diag(lin.J, opts.min_diag, opts.max_diag)
        if solve_fn is None:
            precond = make_precond(lin, D, mu)
            res = pcgnr(lin.J, D, mu, -lin.g, precond, opts.pcg_rel_tol, opts.max_pcg_iters)
        else:
            res = solve_fn(lin, D, mu)
        h = res.h
        pcg_total += res.iters
        Jh = lin.J @ h
        L = float(-(lin.g @ h) - 0.5 * (Jh @ Jh))
        x_new = x + h if step_fn is None else step_fn(x, h)
        F_new = cost_fn(x_new)
        rho = (lin.F - F_new) / L if L > 0 else -np.inf
        ok = bool(np.isfinite(F_new) and L > 0 and rho > 0)
        hist.append(dict(cost=lin.F, cost_new=F_new, mu=mu, rho=rho, pcg_iters=res.iters,
                         accepted=ok, model_decrease=L))
        it += 1
        if ok:
            x = x_new
            mu = mu * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3)
            nu = 2.0
            accepted += 1
            lin = linearize_fn(x)
        else:
            mu = mu * nu
            nu = 2.0 * nu
    return LMResult(x=x, initial_cost=F0, final_cost=lin.F, history=hist, lm_iters=it,
                    accepted=accepted, pcg_iters_total=pcg_total)


def _ba_precond(lin, D, mu):
    Mc, Mp = block_jacobi(lin, D, mu)
    return lambda v: apply_block_jacobi(Mc, Mp, v)


# --------------------------------------------------------------------------------------
# Bundle adjustment entry points
# --------------------------------------------------------------------------------------


def pack(cams, pts):
    return np.concatenate([np.asarray(cams, np.float64).reshape(-1),
                           np.asarray(pts, np.float64).reshape(-1)])


def unpack(x, n_cams):
    return x[: 9 * n_cams].reshape(n_cams, 9), x[9 * n_cams:].reshape(-1, 3)


def retract_cams(cams, h_cams):
    """Cameras after a tangent step: rotation Exp(h_w) R(w), returned as a rotation
    vector; translation, focal length and distortion updated additively."""
    from scipy.spatial.transform import Rotation
    cams = np.asarray(cams, np.float64)
    h = np.asarray(h_cams, np.float64)
    out = cams + h
    out[:, 0:3] = (Rotation.from_rotvec(h[:, 0:3]) * Rotation.from_rotvec(cams[:, 0:3])).as_rotvec()
    return out


def ba_solve(cams0, pts0, cam_idx, pt_idx, pixels, opts: LMOptions = LMOptions(),
             factors: PoseFactors | None = None) -> LMResult:
    """Bundle adjustment by LM + PCGNR over all camera and point parameters.  With
    opts.rotation_update == "retraction" each step updates the rotations by
    R <- Exp(d) R (Jacobian w.r.t. d), the rest additively.  Pose factors, if given,
    join the reprojection factors in the cost and the normal equations."""
    n_cams = cams0.shape[0]
    retraction = opts.rotation_update == "retraction"
    if opts.rotation_update not in ("additive", "retraction"):
        raise ValueError(opts.rotation_update)

    def lin_fn(x):
        c, p = unpack(x, n_cams)
        return linearize(c, p, cam_idx, pt_idx, pixels, opts.eps_depth, retraction=retraction, loss=opts.loss,
                         loss_scale=opts.loss_scale, factors=factors)

    def cost_fn(x):
        c, p = unpack(x, n_cams)
        F = robust_cost(c, p, cam_idx, pt_idx, pixels, opts.eps_depth, opts.loss, opts.loss_scale)
        return F if factors is None else F + pose_factor_cost(c, factors)

    def step_fn(x, h):
        c, p = unpack(x, n_cams)
        hc, hp = unpack(h, n_cams)
        return pack(retract_cams(c, hc), p + hp)

    if opts.solver not in ("pcgnr", "schur"):
        raise ValueError(opts.solver)
    solve_fn = None
    if opts.solver == "schur":
        solve_fn = lambda lin, D, mu: schur_pcg(lin, D, mu, n_cams, opts.pcg_rel_tol, opts.max_pcg_iters)
    return lm_solve(pack(cams0, pts0), lin_fn, cost_fn, _ba_precond, opts, step_fn if retraction else None, solve_fn)


def normal_matvec(lin: Linearization, D, mu, v):
    """(J^T J + mu D) v, the operator PCGNR applies."""
    return lin.J.T @ (lin.J @ v) + mu * D * v
