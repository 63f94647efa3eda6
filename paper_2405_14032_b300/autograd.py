"""torch.autograd wrappers of the matrix-free derivative kernels.

``constraints(h, x, pd, qd)`` returns c(x, Pd, Qd) and ``objective(h, x)`` the
cost f(x) as differentiable torch tensors: backward runs J^T y and the load
adjoint (``mpopf_vjp``), double backward runs W v (``mpopf_hvp``) and J v
(``mpopf_jvp``), so gradients with respect to x and to the per-period loads
flow without J or W ever being materialised.  Argument marshalling only; all
arithmetic runs in libmpopf's kernels.
"""
from __future__ import annotations

import torch

from . import mpopf


class _ConsVJP(torch.autograd.Function):
    """(J(x)^T y, (dc/dPd)^T y, (dc/dQd)^T y) as a differentiable function of (x, y)."""

    @staticmethod
    def forward(ctx, x, y, h):
        gx, gpd, gqd = h.vjp(x, y)
        ctx.save_for_backward(x, y)
        ctx.h = h
        return gx, gpd, gqd

    @staticmethod
    def backward(ctx, ggx, ggpd, ggqd):
        x, y = ctx.saved_tensors
        h = ctx.h
        if ggx is None:
            ggx = torch.zeros_like(x)
        ggx = ggx.contiguous()
        # d/dx <ggx, J(x)^T y> = (sum_i y_i grad^2 c_i) ggx: W v with lambda = y, sigma = 0
        gx = h.hvp(x, y, 0.0, ggx) if ctx.needs_input_grad[0] else None
        gy = None
        if ctx.needs_input_grad[1]:
            if ggpd is None and ggqd is None:
                gy = h.jvp(x, ggx)
            else:
                zero = torch.zeros(h.T * h.n_load, dtype=torch.float64, device=x.device)
                dp = zero if ggpd is None else ggpd.contiguous()
                dq = zero if ggqd is None else ggqd.contiguous()
                gy = h.jvp(x, ggx, dpd=dp, dqd=dq)
        return gx, gy, None


class _Constraints(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, pd, qd, h):
        h.set_loads(pd.contiguous(), qd.contiguous())
        c = h.eval(mpopf.OUT_CONS, x)["c"]
        ctx.save_for_backward(x)
        ctx.h = h
        ctx.load_shape = pd.shape
        return c

    @staticmethod
    def backward(ctx, gc):
        (x,) = ctx.saved_tensors
        gx, gpd, gqd = _ConsVJP.apply(x, gc.contiguous(), ctx.h)
        return gx, gpd.view(ctx.load_shape), gqd.view(ctx.load_shape), None


class _ObjGrad(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, h):
        g = h.eval(mpopf.OUT_GRAD, x)["grad"]
        ctx.save_for_backward(x)
        ctx.h = h
        return g

    @staticmethod
    def backward(ctx, gg):
        (x,) = ctx.saved_tensors
        h = ctx.h
        lam0 = torch.zeros(h.m, dtype=torch.float64, device=x.device)
        return h.hvp(x, lam0, 1.0, gg.contiguous()), None


class _Objective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, h):
        f = h.eval(mpopf.OUT_OBJ, x)["f"]
        ctx.save_for_backward(x)
        ctx.h = h
        return f.reshape(())

    @staticmethod
    def backward(ctx, gf):
        (x,) = ctx.saved_tensors
        return gf * _ObjGrad.apply(x, ctx.h), None


def constraints(h: mpopf.Handle, x: torch.Tensor, pd: torch.Tensor, qd: torch.Tensor) -> torch.Tensor:
    """c(x, Pd, Qd) [m]; pd, qd are the per-period loads [T][D] (this call
    also makes them the handle's loads)."""
    return _Constraints.apply(x, pd, qd, h)


def objective(h: mpopf.Handle, x: torch.Tensor) -> torch.Tensor:
    """f(x) (0-dim)."""
    return _Objective.apply(x, h)
