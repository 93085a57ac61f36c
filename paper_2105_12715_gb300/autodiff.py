"""torch.autograd.Function around the unrolled restarted-PDHG map.

forward: (c, b) -> (xbar, ybar), the running average after `iters` recorded
iterations of restarted PDHG (lp_solve_recorded).  backward: the library's
hand-written adjoint (lp_backward).  Restart decisions and clamp/projection
activity are those of the recorded forward solve.

The tensors go to the library as they are: c, b, the incoming gradients and
the outputs are passed by pointer (the C ABI takes host or device arrays), so
CUDA tensors never round-trip through host memory.  The matrix, bounds and
row senses come from the LP's data object.
"""
from __future__ import annotations

import torch

from . import lp as _lp
from .lpgen import LPData


def _f64(t):
    return t.detach().to(torch.float64).contiguous()


def _replace_cb(data, c, b):
    d = LPData(**{**data.__dict__})
    d.c = c
    d.b = b
    return d


class UnrolledRestartedPDHG(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, b, data, iters, options):
        cd, bd = _f64(c), _f64(b)
        g = _lp.LP(_replace_cb(data, cd, bd), **options)
        _lp.lp_solve_recorded(g.h, iters, g.stream)
        xbar = torch.empty(g.n, dtype=torch.float64, device=c.device)
        ybar = torch.empty(g.m, dtype=torch.float64, device=b.device)
        _lp.lp_get_state(g.h, xbar=xbar, ybar=ybar, stream=g.stream)
        ctx.handle = g
        ctx.devices = (c.device, b.device)
        return xbar, ybar

    @staticmethod
    def backward(ctx, gx, gy):
        g = ctx.handle
        dev_c, dev_b = ctx.devices
        dc = torch.empty(g.n, dtype=torch.float64, device=dev_c)
        db = torch.empty(g.m, dtype=torch.float64, device=dev_b)
        gxd = None if gx is None else _f64(gx)
        gyd = None if gy is None else _f64(gy)
        _lp.lp_backward(g.h, gxd, gyd, dc, db, g.stream)
        g.close()
        return dc, db, None, None, None


def unrolled_pdhg(c, b, data, iters, **options):
    """(xbar, ybar) after `iters` unrolled iterations; differentiable in c and b."""
    return UnrolledRestartedPDHG.apply(c, b, data, iters, options)


class UnrolledRestartedPDHGBatch(torch.autograd.Function):
    """The same map for a batch of LPs solved together (lp_batch_solve_recorded /
    lp_batch_backward): c and b are the problems' vectors concatenated."""

    @staticmethod
    def forward(ctx, c, b, problems, iters, options):
        g = _lp.LPBatch(problems, c=_f64(c), b=_f64(b), **options)
        g.solve_recorded(iters)
        xbar = torch.empty(g.n, dtype=torch.float64, device=c.device)
        ybar = torch.empty(g.m, dtype=torch.float64, device=b.device)
        _lp.lp_batch_get_state(g.h, xbar=xbar, ybar=ybar, stream=g.stream)
        ctx.handle = g
        ctx.devices = (c.device, b.device)
        return xbar, ybar

    @staticmethod
    def backward(ctx, gx, gy):
        g = ctx.handle
        dev_c, dev_b = ctx.devices
        dc = torch.empty(g.n, dtype=torch.float64, device=dev_c)
        db = torch.empty(g.m, dtype=torch.float64, device=dev_b)
        gxd = None if gx is None else _f64(gx)
        gyd = None if gy is None else _f64(gy)
        _lp.lp_batch_backward(g.h, gxd, gyd, dc, db, g.stream)
        g.close()
        return dc, db, None, None, None


def unrolled_pdhg_batch(c, b, problems, iters, **options):
    """Batched (xbar, ybar) of every problem after `iters` unrolled iterations,
    concatenated; differentiable in the concatenated c and b."""
    return UnrolledRestartedPDHGBatch.apply(c, b, problems, iters, options)
