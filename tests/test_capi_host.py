"""Host-side checks of the C ABI: the library loads, exports every symbol the public
header declares, and validates its inputs without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2605_30583_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_30583_gb300 import build
    build.build()
    return binding.lib()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "gbba.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ba_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(binding.SIGNATURES), set(names) ^ set(binding.SIGNATURES)


def test_options_defaults_follow_the_paper(lib):
    o = binding.default_options()
    assert o.initial_trust_region == 100.0 and o.pcg_rel_tol == 1e-3      # Sec. VI settings
    assert o.max_lm_iters == 20 and o.max_pcg_iters == 50 and o.use_graph == 1
    # the build's own defaults: double-float residuals, LM stops once mu passes 1e16
    assert o.residual_precision == 1 and o.max_mu == 1e16 and o.wait_timeout_ms == 2000
    assert lib.ba_abi_version() == 2


def _create(n_cams, n_pts, ci, pi, px, prec=0):
    h = ctypes.c_void_p()
    ci = np.ascontiguousarray(ci, np.uint32)
    pi = np.ascontiguousarray(pi, np.uint32)
    px = np.ascontiguousarray(px, np.float64)
    st = binding.lib().ba_problem_create(n_cams, n_pts, len(ci), ci.ctypes.data, pi.ctypes.data,
                                          px.ctypes.data, prec, ctypes.byref(h))
    return st, h


def test_create_rejects_bad_indices_and_single_views(lib):
    px = np.zeros((4, 2))
    st, h = _create(2, 2, [0, 1, 2, 0], [0, 0, 1, 1], px)
    assert st == 1 and not h.value
    assert b"out of range" in lib.ba_last_error()
    st, h = _create(2, 2, [0, 1, 0, 1], [0, 0, 1, 0], px)      # point 1 seen once
    assert st == 1 and b"at least 2" in lib.ba_last_error()
    st, h = _create(0, 2, [0, 1, 0, 1], [0, 0, 1, 1], px)
    assert st == 1
    st, h = _create(2, 2, [0, 1, 0, 1], [0, 0, 1, 1], px, prec=7)
    assert st == 1


def test_create_and_workspace_size_without_gpu(lib):
    st, h = _create(3, 2, [0, 1, 2, 0], [0, 0, 1, 1], np.zeros((4, 2)))
    assert st == 0 and h.value
    n = ctypes.c_size_t()
    assert lib.ba_workspace_size(h, ctypes.byref(n)) == 0 and n.value > 0
    # calls that need a bound workspace report a state error, not a crash
    c = np.zeros((3, 9))
    p = np.zeros((2, 3))
    assert lib.ba_set_params(h, c.ctypes.data, p.ctypes.data) == 7
    o = binding.default_options()
    assert lib.ba_solve(h, ctypes.byref(o), None, None, 0) == 7
    lib.ba_problem_destroy(h)


def test_workspace_grows_with_problem_and_fp64_is_larger(lib):
    sizes = {}
    for prec in (0, 1):
        st, h = _create(4, 3, [0, 1, 2, 3, 0, 1], [0, 0, 1, 1, 2, 2], np.zeros((6, 2)), prec)
        n = ctypes.c_size_t()
        lib.ba_workspace_size(h, ctypes.byref(n))
        sizes[prec] = n.value
        lib.ba_problem_destroy(h)
    assert sizes[1] > sizes[0]


def test_pose_factor_validation_without_gpu(lib):
    """ba_set_pose_factors checks indices, values and the form before any device work,
    and the workspace grows with the factors."""
    px = np.zeros((4, 2))
    st, h = _create(3, 2, [0, 1, 2, 0], [0, 0, 1, 1], px)
    assert st == 0
    size0 = ctypes.c_size_t()
    assert lib.ba_workspace_size(h, ctypes.byref(size0)) == 0
    a = np.array([0, 1], np.uint32)
    b = np.array([1, 2], np.uint32)
    meas = np.zeros((2, 6))
    ok = lib.ba_set_pose_factors(h, 2, a.ctypes.data, b.ctypes.data, meas.ctypes.data, None)
    assert ok == 0
    size1 = ctypes.c_size_t()
    assert lib.ba_workspace_size(h, ctypes.byref(size1)) == 0
    assert size1.value > size0.value
    bad = np.array([1, 3], np.uint32)                               # camera 3 does not exist
    assert lib.ba_set_pose_factors(h, 2, a.ctypes.data, bad.ctypes.data, meas.ctypes.data, None) == 1
    same = np.array([0, 1], np.uint32)                              # a factor tying camera 0 to itself
    assert lib.ba_set_pose_factors(h, 2, a.ctypes.data, same.ctypes.data, meas.ctypes.data, None) == 1
    nan = meas.copy()
    nan[1, 4] = np.nan
    assert lib.ba_set_pose_factors(h, 2, a.ctypes.data, b.ctypes.data, nan.ctypes.data, None) == 1
    neg = -np.ones((2, 6))
    assert lib.ba_set_pose_factors(h, 2, a.ctypes.data, b.ctypes.data, meas.ctypes.data, neg.ctypes.data) == 1
    assert lib.ba_set_pose_factors(h, 0, None, None, None, None) == 0   # removes them
    size2 = ctypes.c_size_t()
    assert lib.ba_workspace_size(h, ctypes.byref(size2)) == 0 and size2.value == size0.value
    lib.ba_problem_destroy(h)
    st, h = _create(3, 2, [0, 1, 2, 0], [0, 0, 1, 1], px, prec=1)   # plain FP64 form
    assert lib.ba_set_pose_factors(h, 2, a.ctypes.data, b.ctypes.data, meas.ctypes.data, None) == 6
    lib.ba_problem_destroy(h)


def _struct_fields(name):
    """Field names of `typedef struct { ... } name;` in the public header, in order."""
    src = open(os.path.join(ROOT, "include", "gbba.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef struct(?:\s+\w+)?\s*\{([^}]*)\}\s*" + name + r"\s*;", src)
    assert m, name
    names = []
    for decl in re.findall(r"\b(?:int32_t|int64_t|uint32_t|double|float)\s+([a-z_0-9,\s]+);", m.group(1)):
        names += [n.strip() for n in decl.split(",")]
    return names


@pytest.mark.parametrize("cname,pyname", [("ba_options", "Options"), ("ba_stats", "Stats"),
                                          ("ba_iter_stat", "IterStat"), ("ba_batch_trial", "BatchTrial")])
def test_ctypes_mirrors_follow_the_header(lib, cname, pyname):
    """The binding's ctypes structures list the header's fields in the header's order
    (the layout the library reads), and have the C size."""
    cls = getattr(binding, pyname, None)
    if cls is None:
        pytest.skip(f"binding has no {pyname}")
    assert [f[0] for f in cls._fields_] == _struct_fields(cname)


def test_create_rejects_non_finite_pixels(lib):
    """Non-finite measurements are refused at creation, before any device work."""
    for bad in (np.nan, np.inf, -np.inf):
        px = np.zeros((4, 2))
        px[2, 1] = bad
        st, h = _create(2, 2, [0, 1, 0, 1], [0, 0, 1, 1], px)
        assert st == 1 and not h.value
        assert b"non-finite pixel" in lib.ba_last_error()


def test_bind_rejects_a_workspace_one_byte_short(lib):
    """ba_bind_workspace checks the size before it touches the device: a workspace one
    byte smaller than ba_workspace_size is refused with BA_ERR_WORKSPACE_TOO_SMALL (the
    pointer is never dereferenced, so a 256-byte aligned stand-in address serves)."""
    st, h = _create(3, 2, [0, 1, 2, 0], [0, 0, 1, 1], np.zeros((4, 2)))
    assert st == 0
    n = ctypes.c_size_t()
    assert lib.ba_workspace_size(h, ctypes.byref(n)) == 0
    fake = ctypes.c_void_p(1 << 20)
    assert lib.ba_bind_workspace(h, fake, n.value - 1, None) == 3
    assert b"needs" in lib.ba_last_error()
    assert lib.ba_bind_workspace(h, ctypes.c_void_p((1 << 20) + 16), n.value, None) == 1   # misaligned
    lib.ba_problem_destroy(h)


def test_wait_timeout_default(lib):
    o = binding.default_options()
    assert o.wait_timeout_ms == 2000


def test_create_reports_the_first_bad_observation_of_a_large_problem(lib):
    """ba_problem_create checks and copies the observations on several host threads for
    large problems; the error it reports is still the first one in observation order:
    the lowest bad observation, else the lowest point observed fewer than twice (with
    its count)."""
    n_pts, n_cams = 300_000, 50
    n_obs = 4 * 2 ** 20   # several threads' worth of observations
    rng = np.random.default_rng(3)
    pi = np.concatenate([np.repeat(np.arange(n_pts), 2), rng.integers(0, n_pts, n_obs - 2 * n_pts)])
    ci = rng.integers(0, n_cams, n_obs)
    px = rng.standard_normal((n_obs, 2))
    st, h = _create(n_cams, n_pts, ci, pi, px)
    assert st == 0 and h.value
    lib.ba_problem_destroy(h)
    for o_bad in (n_obs - 3, 2_500_000, 1_300_000):      # the lowest of them is reported
        ci[o_bad] = n_cams
    px[3_000_000, 0] = np.nan
    st, h = _create(n_cams, n_pts, ci, pi, px)
    assert st == 1 and not h.value
    assert b"observation 1300000 has camera" in lib.ba_last_error(), lib.ba_last_error()
    ci[[n_obs - 3, 2_500_000, 1_300_000]] = 0
    st, h = _create(n_cams, n_pts, ci, pi, px)
    assert st == 1 and b"observation 3000000 has a non-finite pixel" in lib.ba_last_error()
    px[3_000_000, 0] = 0.0
    # points 7 and 123,457 lose all but one / all of their observations
    for q, keep in ((123_457, 0), (7, 1)):
        idx = np.flatnonzero(pi == q)
        pi[idx[keep:]] = (q + 1) % n_pts
    st, h = _create(n_cams, n_pts, ci, pi, px)
    assert st == 1 and b"point 7 is observed 1 time(s)" in lib.ba_last_error(), lib.ba_last_error()
    pi[pi == 8] = 7    # point 7 seen again; point 8 now unobserved
    st, h = _create(n_cams, n_pts, ci, pi, px)
    assert st == 1 and b"point 8 is observed 0 time(s)" in lib.ba_last_error(), lib.ba_last_error()
