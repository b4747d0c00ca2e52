"""The oracle's pins catch plausible mistakes: each mutation below is planted in a
copy of the oracle (on the CPU, in a temporary tree) and the pin suite must fail on it.

The mutations are the mistakes a restatement of the method could make: a dropped
Rodrigues or distortion term, a wrong sign or index, a wrong damping, gain-ratio or
Madsen constant, a transposed block, an inverted CG coefficient, a retraction applied
on the wrong side, a pose factor with its measurement, sign or camera block wrong.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "rodrigues_second_order_term": ("x0 + a * c0 + b * e0", "x0 + a * c0"),
    "projection_sign": ("p0 = -P0 / d_safe", "p0 = P0 / d_safe"),
    "dropped_k2": ("s = 1.0 + k1 * n2 + k2 * n4", "s = 1.0 + k1 * n2"),
    "half_angle_factor": ("b_big = 2.0 * half * half / th2_safe", "b_big = half * half / th2_safe"),
    "gain_ratio_half": ("L = float(-(lin.g @ h) - 0.5 * (Jh @ Jh))", "L = float(-(lin.g @ h) - (Jh @ Jh))"),
    "madsen_third": ("max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3)", "max(1.0 / 2.0, 1.0 - (2.0 * rho - 1.0) ** 3)"),
    "damping_without_D": ("q = J.T @ w + mu * D * p", "q = J.T @ w + mu * p"),
    "nu_growth": ("nu = 2.0 * nu", "nu = 3.0 * nu"),
    "point_columns_permuted": ("cols_p = 9 * n_cams + 3 * pi", "cols_p = 9 * n_cams + 3 * pi[::-1]"),
    "cg_beta_inverted": ("beta = rz_new / rz", "beta = rz / rz_new"),
    "depth_guard_sign": ("d_safe = P2 + eps_depth * _sign_no_zero(P2)", "d_safe = P2 - eps_depth * _sign_no_zero(P2)"),
    "retraction_composed_on_the_right": ("(Rotation.from_rotvec(h[:, 0:3]) * Rotation.from_rotvec(cams[:, 0:3]))",
                                         "(Rotation.from_rotvec(cams[:, 0:3]) * Rotation.from_rotvec(h[:, 0:3]))"),
    "retraction_step_on_the_right": ("rotate(w, rotate(base_w, X))", "rotate(base_w, rotate(w, X))"),
    "huber_weight_power": ("scale / np.sqrt(np.maximum(s, d2))", "scale / np.maximum(s, d2)"),
    "cauchy_weight_squared": ("return 1.0 / (1.0 + s / d2)", "return 1.0 / (1.0 + s / d2) ** 2"),
    "schur_rhs_sign": ("b = -gc + Jc.T @ (Jp @ hpp_inv(gp))", "b = -gc - Jc.T @ (Jp @ hpp_inv(gp))"),
    "schur_backsub_sign": ("hp = hpp_inv(-gp - Jp.T @ (Jc @ hc))", "hp = hpp_inv(-gp + Jp.T @ (Jc @ hc))"),
    "pose_measurement_not_inverted": ("cols = [rotate([-wm[0], -wm[1], -wm[2]], rot_ba(e)) for e in",
                                      "cols = [rotate([wm[0], wm[1], wm[2]], rot_ba(e)) for e in"),
    "pose_translation_sign": ("rt = [tb[i] - Rt[i] - tm[i] for i in range(3)]",
                              "rt = [tb[i] + Rt[i] - tm[i] for i in range(3)]"),
    "pose_block_to_wrong_camera": ("np.add.at(Hc, np.asarray(factors.cam_b, np.int64), np.einsum(\"oki,okj->oij\", Jb, Jb))",
                                   "np.add.at(Hc, np.asarray(factors.cam_a, np.int64), np.einsum(\"oki,okj->oij\", Jb, Jb))"),
    "pose_cost_dropped_from_candidate": ("return F if factors is None else F + pose_factor_cost(c, factors)",
                                         "return F"),
    "fallback_diagonal_not_inverted": ("out[i] = np.diag(np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0))",
                                       "out[i] = np.diag(np.where(d > 0, d, 0.0))"),
}


@pytest.fixture(scope="module")
def tree(tmp_path_factory):
    """A copy of what the pin suite needs: the oracle, the generator, the pins, goldens."""
    d = tmp_path_factory.mktemp("mut")
    shutil.copytree(os.path.join(ROOT, "oracle"), d / "oracle", ignore=shutil.ignore_patterns("__pycache__", "*.so"))
    pkg = d / "paper_2605_30583_gb300"
    pkg.mkdir()
    (pkg / "__init__.py").write_text("")
    shutil.copy(os.path.join(ROOT, "paper_2605_30583_gb300", "synth.py"), pkg / "synth.py")
    (d / "tests").mkdir()
    shutil.copy(os.path.join(ROOT, "tests", "test_oracle_pins.py"), d / "tests" / "test_oracle_pins.py")
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), d / "tests" / "golden")
    (d / "tests" / "conftest.py").write_text(
        "import os, sys\nsys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))\n")
    return d


def _run_pins(d):
    env = dict(os.environ, PYTHONPATH=str(d), PYTHONDONTWRITEBYTECODE="1")
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                           str(d / "tests" / "test_oracle_pins.py")],
                          cwd=str(d), env=env, capture_output=True, text=True)


def test_unmutated_copy_passes(tree):
    r = _run_pins(tree)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(tree, name):
    path = tree / "oracle" / "ba_oracle.py"
    src = open(os.path.join(ROOT, "oracle", "ba_oracle.py")).read()
    a, b = MUTATIONS[name]
    assert src.count(a) >= 1, f"mutation site for {name} not found"
    path.write_text(src.replace(a, b))
    try:
        r = _run_pins(tree)
        assert r.returncode != 0, f"mutation {name} passed every pin"
    finally:
        path.write_text(src)
