"""torch.autograd.Function around the unrolled restarted-PDHG map.

forward: (c, b) -> (xbar, ybar), the running average after `iters` recorded
iterations of restarted PDHG (lp_solve_recorded).  backward: the library's
hand-written adjoint (lp_backward).  Restart decisions and clamp/projection
activity are those of the recorded forward solve.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lp as _lp
from .lpgen import LPData


def _replace_cb(data, c, b):
    d = LPData(**{**data.__dict__})
    d.c = c
    d.b = b
    return d


class UnrolledRestartedPDHG(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, b, data, iters, options):
        cn = c.detach().to("cpu", torch.float64).numpy()
        bn = b.detach().to("cpu", torch.float64).numpy()
        g = _lp.LP(_replace_cb(data, cn, bn), **options)
        _lp.lp_solve_recorded(g.h, iters, g.stream)
        st = g.state()
        ctx.handle = g
        return (torch.from_numpy(st["xbar"]).to(c.device), torch.from_numpy(st["ybar"]).to(b.device))

    @staticmethod
    def backward(ctx, gx, gy):
        g = ctx.handle
        dc = np.empty(g.n)
        db = np.empty(g.m)
        gxn = None if gx is None else gx.detach().to("cpu", torch.float64).contiguous().numpy()
        gyn = None if gy is None else gy.detach().to("cpu", torch.float64).contiguous().numpy()
        _lp.lp_backward(g.h, gxn, gyn, dc, db, g.stream)
        g.close()
        return (torch.from_numpy(dc).to(gx.device), torch.from_numpy(db).to(gx.device),
                None, None, None)


def unrolled_pdhg(c, b, data, iters, **options):
    """(xbar, ybar) after `iters` unrolled iterations; differentiable in c and b."""
    return UnrolledRestartedPDHG.apply(c, b, data, iters, options)


class UnrolledRestartedPDHGBatch(torch.autograd.Function):
    """The same map for a batch of LPs solved together (lp_batch_solve_recorded /
    lp_batch_backward): c and b are the problems' vectors concatenated."""

    @staticmethod
    def forward(ctx, c, b, problems, iters, options):
        cn = c.detach().to("cpu", torch.float64).numpy()
        bn = b.detach().to("cpu", torch.float64).numpy()
        probs, co, ro = [], 0, 0
        for d in problems:
            probs.append(_replace_cb(d, cn[co:co + d.n], bn[ro:ro + d.m]))
            co += d.n
            ro += d.m
        g = _lp.LPBatch(probs, **options)
        g.solve_recorded(iters)
        st = g.state()
        ctx.handle = g
        return (torch.from_numpy(st["xbar"]).to(c.device), torch.from_numpy(st["ybar"]).to(b.device))

    @staticmethod
    def backward(ctx, gx, gy):
        g = ctx.handle
        gxn = None if gx is None else gx.detach().to("cpu", torch.float64).contiguous().numpy()
        gyn = None if gy is None else gy.detach().to("cpu", torch.float64).contiguous().numpy()
        dc, db = g.backward(gxn, gyn)
        g.close()
        dev = gx.device if gx is not None else gy.device
        return torch.from_numpy(dc).to(dev), torch.from_numpy(db).to(dev), None, None, None


def unrolled_pdhg_batch(c, b, problems, iters, **options):
    """Batched (xbar, ybar) of every problem after `iters` unrolled iterations,
    concatenated; differentiable in the concatenated c and b."""
    return UnrolledRestartedPDHGBatch.apply(c, b, problems, iters, options)
