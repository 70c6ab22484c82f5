"""torch.autograd.Function for the differentiation form of Online FISTA.

`unrolled_loss(ctx, lam, tau, d, track, c0, c_true, steps)` returns
L = ||c_T - c_true||^2 after `steps` unrolled inner steps of Algorithm 1 on
the context's accumulated Gram and data vector.  Its backward pass uses the
library's adjoint kernels (osar_unroll_grad, checkpointed every ~sqrt(steps)
steps) for dL/dlambda and dL/dtau, and dL/dd_s = G_s dL/db for the pulse data
(osar_simulate_pulse applied to dL/db).  The context must hold the
statistics of the pulses `d` along `track` (push them first); `d` enters the
graph only through those statistics.  Complex gradients follow torch's
convention dL/dRe + i dL/dIm.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import osar as _osar


class UnrolledFistaLoss(torch.autograd.Function):
    @staticmethod
    def forward(fctx, lam, tau, d, ctx, track, c0, c_true, steps, ckpt_every, t0):
        res = ctx.unroll_grad(int(steps), int(ckpt_every), float(lam), float(tau),
                              c0, c_true, float(t0))
        fctx.osar = ctx
        fctx.track = np.asarray(track, dtype=np.float64)
        fctx.res = res
        fctx.d_shape = tuple(d.shape)
        return torch.tensor(res["loss"], dtype=torch.float64)

    @staticmethod
    def backward(fctx, grad):
        g = float(grad)
        res = fctx.res
        d_lam = torch.tensor(g * res["d_lambda"], dtype=torch.float64)
        d_tau = torch.tensor(g * res["d_tau"], dtype=torch.float64)
        d_d = None
        if fctx.needs_input_grad[2]:
            rows = [fctx.osar.data_grad(gm, res["d_b"]) for gm in fctx.track]
            d_d = torch.from_numpy(np.stack(rows) * g).reshape(fctx.d_shape)
        return d_lam, d_tau, d_d, None, None, None, None, None, None, None


def unrolled_loss(ctx: "_osar.Osar", lam, tau, d, track, c0, c_true, steps: int,
                  ckpt_every: int | None = None, t0: float = 1.0):
    """Differentiable L(lambda, tau, d); see the module docstring."""
    ckpt = ckpt_every or max(1, int(round(math.sqrt(steps))))
    return UnrolledFistaLoss.apply(lam, tau, d, ctx, track, c0, c_true, steps,
                                   ckpt, t0)
