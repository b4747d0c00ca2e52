"""Host-side checks of the batched entry points (no GPU work: creation validates and
lays out the batch on the host only)."""
import ctypes

import numpy as np
import pytest

from paper_2605_30583_gb300 import synth


@pytest.fixture(scope="module")
def L():
    from paper_2605_30583_gb300 import binding, build
    build.build()
    return binding


def _arrays(probs):
    cam_off = np.concatenate([[0], np.cumsum([p.n_cams for p in probs])]).astype(np.int32)
    pt_off = np.concatenate([[0], np.cumsum([p.n_pts for p in probs])]).astype(np.int32)
    obs_off = np.concatenate([[0], np.cumsum([p.n_obs for p in probs])]).astype(np.int64)
    ci = np.concatenate([p.cam_idx for p in probs]).astype(np.uint32)
    pi = np.concatenate([p.pt_idx for p in probs]).astype(np.uint32)
    px = np.ascontiguousarray(np.concatenate([p.pixels for p in probs]))
    return cam_off, pt_off, obs_off, ci, pi, px


def _create(L, n, cam_off, pt_off, obs_off, ci, pi, px):
    h = ctypes.c_void_p()
    st = L.lib().ba_batch_create(n, L._ptr(cam_off), L._ptr(pt_off), L._ptr(obs_off), L._ptr(ci), L._ptr(pi),
                                 L._ptr(px), ctypes.byref(h))
    return st, h


def test_batch_create_and_workspace_size(L):
    probs = synth.make_batch(5, seed=50000, cams=(5, 9), pts=(200, 300))
    arrs = _arrays(probs)
    st, h = _create(L, len(probs), *arrs)
    assert st == 0 and h.value
    size = ctypes.c_size_t()
    assert L.lib().ba_batch_workspace_size(h, ctypes.byref(size)) == 0
    n_obs = int(arrs[2][-1])
    n_vec = sum(9 * p.n_cams + 3 * p.n_pts for p in probs)
    # at least the observation records and the nine solver vectors
    assert size.value >= 16 * n_obs + 9 * 4 * n_vec
    # calls that need a bound workspace fail cleanly before binding
    o = L.default_options()
    assert L.lib().ba_batch_solve(h, ctypes.byref(o), None) == 7
    L.lib().ba_batch_destroy(h)


def test_batch_create_rejects_bad_inputs(L):
    probs = synth.make_batch(3, seed=50001, cams=(5, 9), pts=(200, 300))
    cam_off, pt_off, obs_off, ci, pi, px = _arrays(probs)
    # local camera index out of range in problem 1
    bad = ci.copy()
    bad[obs_off[1]] = probs[1].n_cams
    assert _create(L, 3, cam_off, pt_off, obs_off, bad, pi, px)[0] == 1
    assert b"out of range" in L.lib().ba_last_error()
    # a point observed only once: keep a single observation of point 0 of problem 2
    own = obs_off[2] + np.flatnonzero(pi[obs_off[2]:] == 0)
    keep = np.ones(len(ci), bool)
    keep[own[1:]] = False
    obs2 = obs_off.copy()
    obs2[3] -= len(own) - 1
    assert _create(L, 3, cam_off, pt_off, obs2, ci[keep], pi[keep], np.ascontiguousarray(px[keep]))[0] == 1
    assert b"fewer than twice" in L.lib().ba_last_error()
    # offsets must start at zero
    c2 = cam_off.copy()
    c2[0] = 1
    assert _create(L, 3, c2, pt_off, obs_off, ci, pi, px)[0] == 1
    # no problems
    assert _create(L, 0, cam_off, pt_off, obs_off, ci, pi, px)[0] == 1


def test_batch_create_rejects_oversized_problem(L):
    n_cams = 1025   # BA_BATCH_MAX_CAMS + 1
    ci = np.repeat(np.arange(n_cams, dtype=np.uint32), 2)
    pi = np.repeat(np.arange(n_cams, dtype=np.uint32), 2)
    px = np.zeros((2 * n_cams, 2))
    st, _ = _create(L, 1, np.array([0, n_cams], np.int32), np.array([0, n_cams], np.int32),
                    np.array([0, 2 * n_cams], np.int64), ci, pi, px)
    assert st == 1 and b"limits" in L.lib().ba_last_error()
