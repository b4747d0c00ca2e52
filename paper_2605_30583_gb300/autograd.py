"""torch.autograd.Function over the total reprojection cost of a bound problem.

F(cams, pts) = 1/2 sum_o |r_o|^2 (Sec. VI-A residual).  Forward calls ba_cost_forward;
backward calls the hand-written adjoint kernel (ba_cost_backward), which recomputes
the residuals and returns grad_out * J^T r for cameras and points.  Inputs are CUDA
tensors in caller layout, cams [n_cams, 9] and pts [n_pts, 3], float32 or float64;
the result is a float64 scalar.  The problem's own parameters are not changed.
"""
from __future__ import annotations

import torch

from . import binding


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return 1
    if t.dtype == torch.float32:
        return 0
    raise TypeError(f"cams/pts must be float32 or float64, got {t.dtype}")


class ReprojectionCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cams: torch.Tensor, pts: torch.Tensor, problem: binding.Problem) -> torch.Tensor:
        if not (cams.is_cuda and pts.is_cuda) or cams.dtype != pts.dtype:
            raise ValueError("cams and pts must be CUDA tensors of one dtype")
        if tuple(cams.shape) != (problem.n_cams, 9) or tuple(pts.shape) != (problem.n_pts, 3):
            raise ValueError("cams must be [n_cams, 9] and pts [n_pts, 3]")
        c, p = cams.contiguous(), pts.contiguous()
        out = torch.empty((), dtype=torch.float64, device=cams.device)
        binding.check(binding.lib().ba_cost_forward(problem._h, c.data_ptr(), p.data_ptr(), _dtype_code(c),
                                                    out.data_ptr()))
        ctx.save_for_backward(c, p)
        ctx.problem = problem
        return out

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        c, p = ctx.saved_tensors
        g = grad_out.detach().to(dtype=torch.float64, device=c.device).contiguous().reshape(())
        gc = torch.empty_like(c)
        gp = torch.empty_like(p)
        binding.check(binding.lib().ba_cost_backward(ctx.problem._h, c.data_ptr(), p.data_ptr(), _dtype_code(c),
                                                     g.data_ptr(), gc.data_ptr(), gp.data_ptr()))
        return gc, gp, None


def reprojection_cost(problem: binding.Problem, cams: torch.Tensor, pts: torch.Tensor) -> torch.Tensor:
    """Differentiable F = 1/2 sum |r|^2 of `problem` at (cams, pts)."""
    return ReprojectionCost.apply(cams, pts, problem)
