"""bench.py's accounting, on the CPU: the algorithmic byte model behind `roofline`, the
time-to-cost rule, and the medium workload's counts the design notes quote."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _P:
    def __init__(self, n_cams, n_pts, n_obs):
        self.n_cams, self.n_pts, self.n_obs = n_cams, n_pts, n_obs


def test_operator_bytes_per_unit():
    # 4 B per observation key; 48 B per point (X, p, D read, q written); 64 + 48 + 96 B per
    # camera (record, direction record, accumulator read-modify-write)
    nb, nf = bench.matvec_model(_P(1, 0, 0))
    assert nb == 208 and nf == 0
    assert bench.matvec_model(_P(0, 1, 0))[0] == 48
    assert bench.matvec_model(_P(0, 0, 1)) == (4, 120)


def test_pcg_iteration_bytes_add_the_vector_update_and_preconditioner():
    # per unknown 44 B; per point block 24 B of M^-1; per camera block 324 B
    nb_c = bench.pcg_iter_model(_P(1, 0, 0))[0]
    assert nb_c == 208 + 44 * 9 + 324
    nb_p = bench.pcg_iter_model(_P(0, 1, 0))[0]
    assert nb_p == 48 + 44 * 3 + 24


def test_medium_workload_counts():
    # 1,000 cameras, 200,000 points, 1,199,169 observations: 46,524,676 B per PCG iteration
    nb, _ = bench.pcg_iter_model(_P(1000, 200_000, 1_199_169))
    assert nb == 46_524_676


def test_time_to_cost_takes_the_first_accepted_step_at_the_target():
    hist = [dict(accepted=True, cost_new=10.0, t_ns=1_000_000),
            dict(accepted=False, cost_new=1.0, t_ns=2_000_000),     # rejected: does not count
            dict(accepted=True, cost_new=4.0, t_ns=3_000_000),
            dict(accepted=True, cost_new=3.0, t_ns=4_000_000)]
    assert bench.time_to_cost(hist, 5.0) == 3.0
    assert bench.time_to_cost(hist, 2.0) is None
    assert bench.time_to_cost(hist, None) is None


def test_tile_operator_bytes_per_unit():
    # 4 B per key; 60 B per point (direction, D, X read; p, q written); 364 B per camera
    assert bench.operator_model(_P(0, 0, 1)) == (4, 120)
    assert bench.operator_model(_P(0, 1, 0))[0] == 60
    assert bench.operator_model(_P(1, 0, 0))[0] == 364


def test_tile_pcg_iteration_bytes():
    # per point 72 (operator) + 84 (update) + 24 (M^-1); per camera 364 + 684
    assert bench.pcg_iter_tile_model(_P(0, 1, 0)) == 180
    assert bench.pcg_iter_tile_model(_P(1, 0, 0)) == 1048
    assert bench.pcg_iter_tile_model(_P(0, 0, 1)) == 4


def test_lm_iteration_bytes():
    # per observation 32 B (linearisation 20, evaluation 12); per point 48 + 48 + 3 x 44;
    # per camera 240 + 516 + 9 x 44
    assert bench.lm_iter_model(_P(0, 0, 1)) == 32
    assert bench.lm_iter_model(_P(0, 1, 0)) == 48 + 48 + 132
    assert bench.lm_iter_model(_P(1, 0, 0)) == 240 + 516 + 396


def test_oracle_subsample_keeps_every_strided_point_with_all_its_observations():
    import numpy as np
    from paper_2605_30583_gb300 import synth
    prob = synth.make_config("tiny")
    sub = bench.oracle_subsample(prob, 4)
    keep = np.arange(prob.n_pts)[::4]
    assert sub.n_pts == len(keep) and sub.n_cams == prob.n_cams
    assert sub.n_obs == int(np.isin(prob.pt_idx, keep).sum())
    # observation by observation the same measurements, points renumbered in order
    sel = np.isin(prob.pt_idx, keep)
    assert np.array_equal(sub.pixels, prob.pixels[sel])
    assert np.array_equal(keep[sub.pt_idx], prob.pt_idx[sel])
    assert np.array_equal(sub.pts_init, prob.pts_init[keep])
    assert np.all(np.bincount(sub.pt_idx, minlength=sub.n_pts) >= 2)


def test_fp64_form_iteration_model():
    # per observation 192 B of stored Jacobian + 8 B of indices, 228 FP64 flops; per point
    # 3 unknowns x (32 + 56) B + 48 B of block inverse; per camera 9 x 88 + 648 B
    assert bench.fp64_iter_model(_P(0, 0, 1)) == (200, 228)
    assert bench.fp64_iter_model(_P(0, 1, 0)) == (312, 60)
    assert bench.fp64_iter_model(_P(1, 0, 0)) == (1440, 180)
