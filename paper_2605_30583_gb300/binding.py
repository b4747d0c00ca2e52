"""ctypes binding of libgbba (include/gbba.h).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  PyTorch supplies the device workspace (one uint8 tensor) and the stream.
If the library has not been built, loading fails with an error: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbba.so")

BA_PREC_MIXED = 0
BA_PREC_FP64 = 1
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "workspace too small", 4: "numeric failure",
          5: "timeout", 6: "not implemented", 7: "call out of order"}


class BAError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{STATUS.get(status, status)}] {message}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("max_lm_iters", ctypes.c_int32), ("max_pcg_iters", ctypes.c_int32),
                ("pcg_rel_tol", ctypes.c_double), ("initial_trust_region", ctypes.c_double),
                ("min_diag", ctypes.c_double), ("max_diag", ctypes.c_double), ("max_mu", ctypes.c_double),
                ("eps_depth", ctypes.c_double), ("use_graph", ctypes.c_int32), ("pcg_kernel", ctypes.c_int32),
                ("rotation_update", ctypes.c_int32), ("loss", ctypes.c_int32), ("loss_scale", ctypes.c_double),
                ("solver", ctypes.c_int32), ("wait_timeout_ms", ctypes.c_int32),
                ("residual_precision", ctypes.c_int32)]


class IterStat(ctypes.Structure):
    _fields_ = [("cost", ctypes.c_double), ("cost_new", ctypes.c_double), ("mu", ctypes.c_double),
                ("rho", ctypes.c_double), ("model_decrease", ctypes.c_double), ("pcg_iters", ctypes.c_int32),
                ("accepted", ctypes.c_int32), ("t_ns", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("initial_cost", ctypes.c_double), ("final_cost", ctypes.c_double), ("lm_iters", ctypes.c_int32),
                ("accepted", ctypes.c_int32), ("pcg_iters_total", ctypes.c_int32), ("status", ctypes.c_int32),
                ("solve_ns", ctypes.c_int64)]


class BatchTrial(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("ms", ctypes.c_float)]


BA_TUNE_IGNORE_CACHE = 1
BA_SCHED_STAGE_POINTS = 1

P = ctypes.c_void_p
I32, I64, U32P, DP, SZ = ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint32), ctypes.c_void_p, ctypes.c_size_t

# name -> (restype, argtypes); the complete exported surface of gbba.h
SIGNATURES = {
    "ba_last_error": (ctypes.c_char_p, []),
    "ba_status_string": (ctypes.c_char_p, [I32]),
    "ba_abi_version": (I32, []),
    "ba_options_default": (I32, [ctypes.POINTER(Options)]),
    "ba_problem_create": (I32, [I32, I32, I64, P, P, P, I32, ctypes.POINTER(P)]),
    "ba_problem_destroy": (None, [P]),
    "ba_workspace_size": (I32, [P, ctypes.POINTER(SZ)]),
    "ba_set_pose_factors": (I32, [P, I32, P, P, P, P]),
    "ba_selftest_wait_timeout": (I32, [P, I32, I32, P, ctypes.POINTER(I32), ctypes.POINTER(I32)]),
    "ba_selftest_rcp64": (I32, [P, P, I64, P]),
    "ba_bind_workspace": (I32, [P, P, SZ, P]),
    "ba_set_params": (I32, [P, P, P]),
    "ba_get_params": (I32, [P, P, P]),
    "ba_set_params_device": (I32, [P, P, P, I32]),
    "ba_get_params_device": (I32, [P, P, P, I32]),
    "ba_evaluate": (I32, [P, ctypes.POINTER(ctypes.c_double), P, P]),
    "ba_solve": (I32, [P, ctypes.POINTER(Options), ctypes.POINTER(Stats), ctypes.POINTER(IterStat), I32]),
    "ba_get_stats": (I32, [P, ctypes.POINTER(Stats), ctypes.POINTER(IterStat), I32]),
    "ba_apply_normal": (I32, [P, ctypes.c_double, P, P, ctypes.POINTER(ctypes.c_double)]),
    "ba_repeat_normal": (I32, [P, I32]),
    "ba_profile_kernels": (I32, [P, I32, P, I32]),
    "ba_cost_forward": (I32, [P, P, P, I32, P]),
    "ba_cost_backward": (I32, [P, P, P, I32, P, P, P]),
    "ba_cost_noalloc": (I32, [I32, I32, I64, P, P, P, P, P, ctypes.c_double, P, P]),
    "ba_batch_create": (I32, [I32, P, P, P, P, P, P, ctypes.POINTER(P)]),
    "ba_batch_destroy": (None, [P]),
    "ba_batch_workspace_size": (I32, [P, ctypes.POINTER(SZ)]),
    "ba_batch_bind_workspace": (I32, [P, P, SZ, P]),
    "ba_batch_set_params": (I32, [P, P, P]),
    "ba_batch_get_params": (I32, [P, P, P]),
    "ba_batch_solve": (I32, [P, ctypes.POINTER(Options), ctypes.POINTER(Stats)]),
    "ba_batch_get_costs": (I32, [P, P, P]),
    "ba_batch_set_schedule": (I32, [P, I32, I32, I32]),
    "ba_batch_get_schedule": (I32, [P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32),
                                    ctypes.POINTER(I32)]),
    "ba_batch_autotune": (I32, [P, ctypes.POINTER(Options), I32, ctypes.POINTER(BatchTrial), I32,
                                ctypes.POINTER(I32)]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library.  Raises if libgbba.so has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != 0:
        raise BAError(status, lib().ba_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def selftest_wait_timeout(grid: int = 4, timeout_ms: int = 50):
    """Runs the bounded-wait self-test (ba_selftest_wait_timeout) on the current CUDA
    stream; returns (CTAs that gave up, error word)."""
    torch = _torch()
    scratch = torch.zeros(16, dtype=torch.uint8, device="cuda")
    gave, err = ctypes.c_int32(), ctypes.c_int32()
    check(lib().ba_selftest_wait_timeout(scratch.data_ptr(), int(grid), int(timeout_ms),
                                         torch.cuda.current_stream().cuda_stream, ctypes.byref(gave),
                                         ctypes.byref(err)))
    return int(gave.value), int(err.value)


def selftest_rcp64(x):
    """1/x through the FP64 reciprocal of the block inversions (ba_selftest_rcp64) for a
    CUDA float64 tensor x; returns a new tensor."""
    torch = _torch()
    x = x.contiguous()
    assert x.is_cuda and x.dtype == torch.float64
    y = torch.empty_like(x)
    check(lib().ba_selftest_rcp64(x.data_ptr(), y.data_ptr(), x.numel(), torch.cuda.current_stream().cuda_stream))
    return y


def default_options(**kw) -> Options:
    o = Options()
    check(lib().ba_options_default(ctypes.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


@dataclasses.dataclass
class SolveResult:
    initial_cost: float
    final_cost: float
    lm_iters: int
    accepted: int
    pcg_iters_total: int
    status: int
    solve_ns: int
    history: list


def _torch():
    import torch
    return torch


class Problem:
    """One bundle-adjustment problem bound to a device workspace.

    cam_idx, pt_idx: integer arrays [n_obs]; pixels: float64 [n_obs, 2] (host arrays).
    precision: "mixed" (FP32 bulk, FP64 sums) or "fp64" (plain all-FP64 form).
    pose_factors: optional (cam_a, cam_b, meas [nf, 6], sqrt_info [nf, 6] or None), the
    relative-pose factors of ba_set_pose_factors (mixed form only)."""

    def __init__(self, n_cams, n_pts, cam_idx, pt_idx, pixels, precision="mixed", stream=None, pose_factors=None):
        torch = _torch()
        self.n_cams, self.n_pts = int(n_cams), int(n_pts)
        ci = np.ascontiguousarray(cam_idx, dtype=np.uint32)
        pi = np.ascontiguousarray(pt_idx, dtype=np.uint32)
        px = np.ascontiguousarray(pixels, dtype=np.float64)
        self.n_obs = int(ci.shape[0])
        self.precision = BA_PREC_FP64 if precision == "fp64" else BA_PREC_MIXED
        self.dtype = torch.float64 if self.precision == BA_PREC_FP64 else torch.float32
        h = ctypes.c_void_p()
        check(lib().ba_problem_create(self.n_cams, self.n_pts, self.n_obs, _ptr(ci), _ptr(pi), _ptr(px),
                                      self.precision, ctypes.byref(h)))
        self._h = h
        self.n_factors = 0
        if pose_factors is not None:
            fa, fb, meas, sq = pose_factors
            fa = np.ascontiguousarray(fa, dtype=np.uint32)
            fb = np.ascontiguousarray(fb, dtype=np.uint32)
            meas = np.ascontiguousarray(meas, dtype=np.float64).reshape(-1, 6)
            sq = None if sq is None else np.ascontiguousarray(sq, dtype=np.float64).reshape(-1, 6)
            self.n_factors = int(fa.shape[0])
            st = lib().ba_set_pose_factors(h, self.n_factors, _ptr(fa), _ptr(fb), _ptr(meas),
                                           _ptr(sq) if sq is not None else None)
            if st != 0:
                self._h = None   # destroyed here; close() must not destroy it again
                lib().ba_problem_destroy(h)
                check(st)
        nbytes = ctypes.c_size_t()
        check(lib().ba_workspace_size(h, ctypes.byref(nbytes)))
        self.workspace_bytes = int(nbytes.value)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        # torch's caching allocator returns 512-byte aligned blocks
        self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device="cuda")
        check(lib().ba_bind_workspace(h, self.workspace.data_ptr(), self.workspace_bytes,
                                      self.stream.cuda_stream))

    # -- parameters ------------------------------------------------------------------
    def set_params(self, cams, pts):
        torch = _torch()
        if isinstance(cams, torch.Tensor):
            c, p = cams.contiguous(), pts.contiguous()
            assert c.is_cuda and p.is_cuda and c.dtype == p.dtype
            check(lib().ba_set_params_device(self._h, c.data_ptr(), p.data_ptr(),
                                             1 if c.dtype == torch.float64 else 0))
            self._keep = (c, p)
        else:
            c = np.ascontiguousarray(cams, dtype=np.float64).reshape(self.n_cams, 9)
            p = np.ascontiguousarray(pts, dtype=np.float64).reshape(self.n_pts, 3)
            check(lib().ba_set_params(self._h, _ptr(c), _ptr(p)))

    def get_params(self):
        c = np.empty((self.n_cams, 9))
        p = np.empty((self.n_pts, 3))
        check(lib().ba_get_params(self._h, _ptr(c), _ptr(p)))
        return c, p

    def get_params_device(self, dtype=None):
        torch = _torch()
        dtype = dtype or self.dtype
        c = torch.empty((self.n_cams, 9), dtype=dtype, device="cuda")
        p = torch.empty((self.n_pts, 3), dtype=dtype, device="cuda")
        check(lib().ba_get_params_device(self._h, c.data_ptr(), p.data_ptr(), 1 if dtype == torch.float64 else 0))
        return c, p

    # -- evaluation ------------------------------------------------------------------
    def evaluate(self, residuals=False, jacobian=False):
        torch = _torch()
        r = torch.empty((self.n_obs, 2), dtype=self.dtype, device="cuda") if residuals else None
        J = torch.empty((self.n_obs, 2, 12), dtype=self.dtype, device="cuda") if jacobian else None
        cost = ctypes.c_double()
        check(lib().ba_evaluate(self._h, ctypes.byref(cost), r.data_ptr() if r is not None else None,
                                J.data_ptr() if J is not None else None))
        return cost.value, r, J

    def apply_normal(self, mu, v):
        torch = _torch()
        v = v.to(device="cuda", dtype=self.dtype).contiguous()
        out = torch.empty_like(v)
        vav = ctypes.c_double()
        check(lib().ba_apply_normal(self._h, float(mu), v.data_ptr(), out.data_ptr(), ctypes.byref(vav)))
        return out, vav.value

    KERNELS = ("camera_records", "linearize", "precond", "matvec", "update", "candidate", "eval_candidate",
               "commit", "pcg_persistent", "pcg_persistent_iters", "cg_round", "residual")

    def profile_kernels(self, reps=20) -> dict:
        out = np.zeros(len(self.KERNELS))
        check(lib().ba_profile_kernels(self._h, int(reps), _ptr(out), len(out)))
        return dict(zip(self.KERNELS, out.tolist()))

    def repeat_normal(self, launches):
        check(lib().ba_repeat_normal(self._h, int(launches)))

    # -- solve -----------------------------------------------------------------------
    def solve(self, options: Options | None = None, wait=True, **kw) -> SolveResult | None:
        o = options if options is not None else default_options(**kw)
        if not wait:
            check(lib().ba_solve(self._h, ctypes.byref(o), None, None, 0))
            return None
        st = Stats()
        cap = max(1, int(o.max_lm_iters))
        hist = (IterStat * cap)()
        check(lib().ba_solve(self._h, ctypes.byref(o), ctypes.byref(st), hist, cap))
        return self._result(st, hist)

    def stats(self, cap=1024) -> SolveResult:
        st = Stats()
        hist = (IterStat * cap)()
        check(lib().ba_get_stats(self._h, ctypes.byref(st), hist, cap))
        return self._result(st, hist)

    @staticmethod
    def _result(st, hist) -> SolveResult:
        n = st.lm_iters
        h = [dict(cost=x.cost, cost_new=x.cost_new, mu=x.mu, rho=x.rho, model_decrease=x.model_decrease,
                  pcg_iters=x.pcg_iters, accepted=bool(x.accepted), t_ns=x.t_ns) for x in list(hist)[:n]]
        return SolveResult(st.initial_cost, st.final_cost, st.lm_iters, st.accepted, st.pcg_iters_total,
                           st.status, st.solve_ns, h)

    def close(self):
        if getattr(self, "_h", None):
            lib().ba_problem_destroy(self._h)
            self._h = None
            self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent problems solved by one persistent launch (ba_batch_*).

    problems: sequence of objects with n_cams, n_pts, cam_idx, pt_idx (local indices)
    and pixels [n_obs, 2]; they are concatenated in the given order."""

    def __init__(self, problems, stream=None):
        torch = _torch()
        self.n_problems = len(problems)
        nc = np.array([p.n_cams for p in problems], dtype=np.int64)
        npt = np.array([p.n_pts for p in problems], dtype=np.int64)
        no = np.array([len(p.cam_idx) for p in problems], dtype=np.int64)
        self.cam_off = np.concatenate([[0], np.cumsum(nc)]).astype(np.int32)
        self.pt_off = np.concatenate([[0], np.cumsum(npt)]).astype(np.int32)
        self.obs_off = np.concatenate([[0], np.cumsum(no)]).astype(np.int64)
        ci = np.ascontiguousarray(np.concatenate([p.cam_idx for p in problems]), dtype=np.uint32)
        pi = np.ascontiguousarray(np.concatenate([p.pt_idx for p in problems]), dtype=np.uint32)
        px = np.ascontiguousarray(np.concatenate([p.pixels for p in problems]), dtype=np.float64)
        self.total_cams, self.total_pts, self.n_obs = int(self.cam_off[-1]), int(self.pt_off[-1]), int(ci.shape[0])
        h = ctypes.c_void_p()
        check(lib().ba_batch_create(self.n_problems, _ptr(self.cam_off), _ptr(self.pt_off), _ptr(self.obs_off),
                                    _ptr(ci), _ptr(pi), _ptr(px), ctypes.byref(h)))
        self._h = h
        nbytes = ctypes.c_size_t()
        check(lib().ba_batch_workspace_size(h, ctypes.byref(nbytes)))
        self.workspace_bytes = int(nbytes.value)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device="cuda")
        check(lib().ba_batch_bind_workspace(h, self.workspace.data_ptr(), self.workspace_bytes,
                                            self.stream.cuda_stream))

    def set_params(self, cams, pts):
        """cams [total_cams, 9], pts [total_pts, 3] (host, concatenated per problem)."""
        c = np.ascontiguousarray(cams, dtype=np.float64).reshape(self.total_cams, 9)
        p = np.ascontiguousarray(pts, dtype=np.float64).reshape(self.total_pts, 3)
        check(lib().ba_batch_set_params(self._h, _ptr(c), _ptr(p)))

    def get_params(self):
        c = np.empty((self.total_cams, 9))
        p = np.empty((self.total_pts, 3))
        check(lib().ba_batch_get_params(self._h, _ptr(c), _ptr(p)))
        return c, p

    def solve(self, options: Options | None = None, wait=True, **kw):
        """Solves every problem; returns a list of SolveResult (no history) if wait."""
        o = options if options is not None else default_options(**kw)
        if not wait:
            check(lib().ba_batch_solve(self._h, ctypes.byref(o), None))
            return None
        st = (Stats * self.n_problems)()
        check(lib().ba_batch_solve(self._h, ctypes.byref(o), st))
        return [SolveResult(s.initial_cost, s.final_cost, s.lm_iters, s.accepted, s.pcg_iters_total, s.status,
                            s.solve_ns, []) for s in st]

    def costs(self):
        a = np.empty(self.n_problems)
        b = np.empty(self.n_problems)
        check(lib().ba_batch_get_costs(self._h, _ptr(a), _ptr(b)))
        return a, b

    def set_schedule(self, threads, ctas_per_sm=0, stage_points=False):
        check(lib().ba_batch_set_schedule(self._h, int(threads), int(ctas_per_sm),
                                          BA_SCHED_STAGE_POINTS if stage_points else 0))

    def schedule(self):
        t, c, f, g = I32(), I32(), I32(), I32()
        check(lib().ba_batch_get_schedule(self._h, ctypes.byref(t), ctypes.byref(c), ctypes.byref(f),
                                          ctypes.byref(g)))
        return dict(threads=t.value, ctas_per_sm=c.value, stage_points=bool(f.value & BA_SCHED_STAGE_POINTS),
                    grid=g.value)

    def autotune(self, options: Options | None = None, ignore_cache=False, **kw):
        """Times the candidate schedules and keeps the fastest; returns the trials."""
        o = options if options is not None else default_options(**kw)
        cap = 64
        tr = (BatchTrial * cap)()
        n = I32()
        check(lib().ba_batch_autotune(self._h, ctypes.byref(o), BA_TUNE_IGNORE_CACHE if ignore_cache else 0, tr, cap,
                                      ctypes.byref(n)))
        return [dict(threads=t.threads, ctas_per_sm=t.ctas_per_sm,
                     stage_points=bool(t.flags & BA_SCHED_STAGE_POINTS), grid=t.grid, ms=t.ms)
                for t in tr[: n.value]]

    def close(self):
        if getattr(self, "_h", None):
            lib().ba_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
