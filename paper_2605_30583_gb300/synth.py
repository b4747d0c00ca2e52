"""Seeded synthetic bundle-adjustment problems shaped like the BAL workloads.

This module is the one input generator shared by the tests, the benchmark and the
FP64 oracle's checks.  It holds none of the solver's arithmetic: no residual,
Jacobian, normal-equation or damping code.  It does need a camera model to turn
ground-truth cameras and points into measured pixels; it states that model its own
way (look-at rotation matrices, scipy rotation vectors), so a mistake in either the
oracle's projection or this one shows up as a non-zero residual at ground truth.

Camera model (Sec. VI-A of the paper, Snavely reprojection factor; 9 parameters per
camera in the BAL order): rotation vector w (3), translation t (3), focal length f,
radial terms k1, k2.  A world point X maps to the camera frame as P = R X + t, the
normalised image point is p = -P.xy / P.z (points in front of a camera have P.z < 0)
and the pixel is f * (1 + k1 |p|^2 + k2 |p|^4) * p.

Workload recipe (all randomness from numpy's PCG64 seeded per problem):
  * cameras on a ring (radius 5 unless a configuration states another) in the z = 0 plane, evenly spaced in azimuth,
    each looking at the origin along its own -z axis, with world +z as "up";
  * f ~ U(500, 1000), k1, k2 ~ N(0, 0.01^2);
  * points ~ N(0, I3), redrawn while |X| > 3 so every camera sees every point at a
    depth of at least 2 (the recipe keeps |P.z| >= 0.5 for every observation); or, for
    a ring of radius R > 8 ("band"), points at a uniform azimuth, 2-8 units inside the
    ring, height N(0, 1) clipped to 3 (the large workload: 13,000 cameras at radius 65
    keep the 1,000-camera ring's spacing, so nearest cameras see a point with the same
    parallax);
  * each point is seen by 2 + Poisson(lam) cameras (or 2 + Geometric with a given
    mean), clipped to the camera count, chosen either uniformly at random or as the
    cameras nearest to the point on the ring;
  * pixel noise N(0, 1 px^2);
  * initial guess: rotation Exp(0.01 a) R_gt with a uniform on the sphere,
    t_gt + 0.01 |t_gt| b with b uniform on the sphere, X_gt + N(0, 0.05^2 I3);
    f, k1, k2 start at their true values;
  * observation order is shuffled, so no solver can rely on the input order.
"""
from __future__ import annotations

import dataclasses
import numpy as np
from scipy.spatial.transform import Rotation

RING_RADIUS = 5.0
MAX_POINT_RADIUS = 3.0


@dataclasses.dataclass
class Problem:
    """A bundle-adjustment problem in the caller (user) layout, all FP64 on the host."""
    n_cams: int
    n_pts: int
    cam_idx: np.ndarray      # uint32 [n_obs]
    pt_idx: np.ndarray       # uint32 [n_obs]
    pixels: np.ndarray       # float64 [n_obs, 2]
    cams_init: np.ndarray    # float64 [n_cams, 9]
    pts_init: np.ndarray     # float64 [n_pts, 3]
    cams_gt: np.ndarray      # float64 [n_cams, 9]
    pts_gt: np.ndarray       # float64 [n_pts, 3]
    name: str = ""

    @property
    def n_obs(self) -> int:
        return int(self.cam_idx.shape[0])


# Configurations used by tests and the benchmark.  Sizes follow the workloads the
# paper evaluates on (BAL-like shapes); the data itself is synthetic.
CONFIGS = {
    "tiny": dict(n_cams=16, n_pts=1000, views=("poisson", 3.0), visibility="uniform", seed=1000),
    "medium": dict(n_cams=1000, n_pts=200_000, views=("poisson", 4.0), visibility="nearest", seed=1001),
    # 13,000 cameras at the medium workload's spacing (ring radius 65), points in a band
    # 2-8 units inside the ring: every point meets its nearest cameras with the medium
    # workload's parallax, as a large reconstruction's points meet theirs
    "large": dict(n_cams=13_000, n_pts=4_500_000, views=("geometric", 4.4), visibility="nearest", seed=1002,
                  ring_radius=65.0, scene="band"),
    "autograd": dict(n_cams=200, n_pts=50_000, views=("poisson", 4.0), visibility="nearest", seed=1004),
    # the large workload's local shape (camera spacing, depths, points per camera, view
    # counts, visibility) at 1/13 of its size: small enough for full profiler captures
    "large_shape": dict(n_cams=1000, n_pts=346_000, views=("geometric", 4.4), visibility="nearest", seed=1002),
}


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def ring_cameras(n_cams: int, radius: float = RING_RADIUS) -> tuple[np.ndarray, np.ndarray]:
    """World-to-camera rotation matrices and translations of the inward-looking ring."""
    az = 2.0 * np.pi * np.arange(n_cams) / n_cams
    c, s = np.cos(az), np.sin(az)
    z_cam = np.stack([c, s, np.zeros_like(c)], axis=1)          # outward radial: camera looks along -z
    y_cam = np.tile(np.array([0.0, 0.0, 1.0]), (n_cams, 1))      # world up
    x_cam = np.cross(y_cam, z_cam)
    R = np.stack([x_cam, y_cam, z_cam], axis=1)                  # rows are the camera axes
    centres = radius * z_cam
    t = -np.einsum("cij,cj->ci", R, centres)
    return R, t


def _pixels(R: np.ndarray, t: np.ndarray, intr: np.ndarray, X: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Pixel of each (camera, point) pair; R, t, intr are already gathered per pair."""
    P = np.einsum("oij,oj->oi", R, X) + t
    depth = P[:, 2]
    xy = -P[:, :2] / depth[:, None]
    rr = np.sum(xy * xy, axis=1)
    scale = intr[:, 0] * (1.0 + intr[:, 1] * rr + intr[:, 2] * rr * rr)
    return scale[:, None] * xy, depth


def _draw_points(rng: np.random.Generator, n: int, scene: str = "cloud", radius: float = RING_RADIUS) -> np.ndarray:
    if scene == "band":
        # azimuth uniform, 2-8 units inside the ring, height N(0, 1) clipped to 3
        az = rng.uniform(0.0, 2.0 * np.pi, n)
        r = radius - rng.uniform(2.0, 8.0, n)
        z = np.clip(rng.standard_normal(n), -MAX_POINT_RADIUS, MAX_POINT_RADIUS)
        return np.stack([r * np.cos(az), r * np.sin(az), z], axis=1)
    if scene != "cloud":
        raise ValueError(scene)
    X = rng.standard_normal((n, 3))
    bad = np.linalg.norm(X, axis=1) > MAX_POINT_RADIUS
    while bad.any():
        X[bad] = rng.standard_normal((int(bad.sum()), 3))
        bad = np.linalg.norm(X, axis=1) > MAX_POINT_RADIUS
    return X


def _view_counts(rng: np.random.Generator, n: int, views: tuple[str, float], n_cams: int) -> np.ndarray:
    kind, mean = views
    if kind == "poisson":
        extra = rng.poisson(mean, n)
    elif kind == "geometric":
        # numpy's geometric counts trials (support 1, 2, ...); subtract one for the
        # number of failures, whose mean is (1 - p) / p = `mean`.
        extra = rng.geometric(1.0 / (1.0 + mean), n) - 1
    else:
        raise ValueError(kind)
    return np.minimum(2 + extra, n_cams).astype(np.int64)


def _choose_cameras(rng, X, counts, n_cams, visibility) -> np.ndarray:
    """Camera index of every observation, point-major (point i's views are contiguous)."""
    n = X.shape[0]
    kmax = int(counts.max())
    if visibility == "uniform":
        keys = rng.random((n, n_cams))
        order = np.argsort(keys, axis=1)[:, :kmax]
    elif visibility == "nearest":
        # Distance to a ring camera grows with the azimuth gap, so the k nearest
        # cameras are the k ring positions closest to the point's azimuth.
        u = np.mod(np.arctan2(X[:, 1], X[:, 0]), 2.0 * np.pi) / (2.0 * np.pi / n_cams)
        start = np.round(u - (counts - 1) / 2.0).astype(np.int64)
        order = np.mod(start[:, None] + np.arange(kmax)[None, :], n_cams)
    else:
        raise ValueError(visibility)
    keep = np.arange(kmax)[None, :] < counts[:, None]
    return order[keep].astype(np.int64)


def make_problem(n_cams: int, n_pts: int, views=("poisson", 3.0), visibility="uniform",
                 seed: int = 0, noise_px: float = 1.0, perturb: bool = True, ring_radius: float = RING_RADIUS,
                 scene: str = "cloud",
                 name: str = "") -> Problem:
    rng = np.random.default_rng(seed)
    R_gt, t_gt = ring_cameras(n_cams, ring_radius)
    intr = np.stack([rng.uniform(500.0, 1000.0, n_cams),
                     0.01 * rng.standard_normal(n_cams),
                     0.01 * rng.standard_normal(n_cams)], axis=1)
    X_gt = _draw_points(rng, n_pts, scene, ring_radius)
    counts = _view_counts(rng, n_pts, views, n_cams)
    cam_idx = _choose_cameras(rng, X_gt, counts, n_cams, visibility)
    pt_idx = np.repeat(np.arange(n_pts, dtype=np.int64), counts)

    px, depth = _pixels(R_gt[cam_idx], t_gt[cam_idx], intr[cam_idx], X_gt[pt_idx])
    assert np.all(depth <= -0.5), "recipe guarantees every observed point is in front"
    if noise_px > 0:
        px = px + noise_px * rng.standard_normal(px.shape)

    rot_gt = Rotation.from_matrix(R_gt)
    cams_gt = np.concatenate([rot_gt.as_rotvec(), t_gt, intr], axis=1)
    if perturb:
        dR = Rotation.from_rotvec(0.01 * _unit_vectors(rng, n_cams))
        w0 = (dR * rot_gt).as_rotvec()
        tn = np.linalg.norm(t_gt, axis=1, keepdims=True)
        t0 = t_gt + 0.01 * tn * _unit_vectors(rng, n_cams)
        X0 = X_gt + 0.05 * rng.standard_normal(X_gt.shape)
    else:
        w0, t0, X0 = cams_gt[:, :3].copy(), t_gt.copy(), X_gt.copy()
    cams_init = np.concatenate([w0, t0, intr], axis=1)

    perm = rng.permutation(cam_idx.shape[0])
    return Problem(n_cams=n_cams, n_pts=n_pts,
                   cam_idx=cam_idx[perm].astype(np.uint32), pt_idx=pt_idx[perm].astype(np.uint32),
                   pixels=np.ascontiguousarray(px[perm]),
                   cams_init=cams_init, pts_init=X0, cams_gt=cams_gt, pts_gt=X_gt, name=name)


def make_config(name: str, **overrides) -> Problem:
    cfg = dict(CONFIGS[name])
    cfg.update(overrides)
    return make_problem(name=name, **cfg)


def make_batch(n_problems: int = 512, seed: int = 30000, cams=(5, 60), pts=(200, 5000),
               lam: float = 3.0) -> list[Problem]:
    """Independent small problems of uneven sizes: cameras ~ U[5, 60], points ~ U[200, 5000]."""
    out = []
    for i in range(n_problems):
        rng = np.random.default_rng(seed + i)
        nc = int(rng.integers(cams[0], cams[1] + 1))
        npt = int(rng.integers(pts[0], pts[1] + 1))
        out.append(make_problem(nc, npt, ("poisson", lam), "uniform", seed=seed + i,
                                name=f"batch{i}"))
    return out


def make_pose_factors(p: Problem, pairs: str = "chain", rot_sigma: float = 0.002, t_sigma: float = 0.01,
                      seed: int = 7, noise: bool = True) -> tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """Relative-pose measurements between cameras of `p`, from its ground truth plus noise.

    pairs: "chain" ties camera i to i + 1 around the ring (odometry, n_cams factors
    with the loop closed), "chain+skip" adds i to i + 2.  The measurement of (a, b) is
    the pose of b relative to a, computed here with rotation matrices: R_ab_gt =
    R_b R_a^T and t_ab_gt = t_b - R_ab_gt t_a, then perturbed by a left rotation
    Exp(rot_sigma n) (n ~ N(0, I3)) and N(0, t_sigma^2 I3) on the translation.
    Returns cam_a, cam_b (uint32), meas [nf, 6] (rotation vector, translation) and
    sqrt_info [nf, 6] = (1 / rot_sigma, 1 / t_sigma) per row.  noise=False returns the
    exact relative poses (same weights)."""
    rng = np.random.default_rng(seed)
    n = p.n_cams
    a = np.arange(n)
    b = (a + 1) % n
    if pairs == "chain+skip":
        a = np.concatenate([a, np.arange(n)])
        b = np.concatenate([b, (np.arange(n) + 2) % n])
    elif pairs != "chain":
        raise ValueError(pairs)
    keep = a != b
    a, b = a[keep], b[keep]
    Rm = Rotation.from_rotvec(p.cams_gt[:, 0:3]).as_matrix()
    R_ab = np.einsum("kij,klj->kil", Rm[b], Rm[a])                     # R_b R_a^T
    t_ab = p.cams_gt[b, 3:6] - np.einsum("kij,kj->ki", R_ab, p.cams_gt[a, 3:6])
    scale = 1.0 if noise else 0.0
    dR = Rotation.from_rotvec(scale * rot_sigma * rng.standard_normal((a.size, 3))).as_matrix()
    meas_R = np.einsum("kij,kjl->kil", dR, R_ab)
    meas = np.concatenate([Rotation.from_matrix(meas_R).as_rotvec(),
                           t_ab + scale * t_sigma * rng.standard_normal((a.size, 3))], axis=1)
    sqrt_info = np.tile(np.array([1.0 / rot_sigma] * 3 + [1.0 / t_sigma] * 3), (a.size, 1))
    return a.astype(np.uint32), b.astype(np.uint32), meas, sqrt_info


def round_to_f32(p: Problem) -> Problem:
    """Same problem with every real input rounded to FP32, so an FP32 device path and an
    FP64 reference see bit-identical inputs."""
    f = lambda a: a.astype(np.float32).astype(np.float64)
    return dataclasses.replace(p, pixels=f(p.pixels), cams_init=f(p.cams_init), pts_init=f(p.pts_init))
